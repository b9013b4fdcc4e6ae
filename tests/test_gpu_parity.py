"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

FP64 path bar: max |Q_gpu - Q_oracle| <= 1e-12 * max |Q_oracle| over the compared cells.
Inputs are seeded (wef_inputs); the core is either a random stand-in (the contraction
is what is tested) or the oracle's own quadrature core."""
import numpy as np
import pytest

import wef_inputs as wi
from oracle import core as ocore
from oracle import dense, gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not __import__("os").path.exists(W.LIB_PATH):
        from paper_2605_28475_gb300 import build

        build.build()


def _gpu_eval(op, f, precision="fp64"):
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    q = op.evaluate(fd, precision=precision)
    torch.cuda.synchronize()
    return q.cpu().numpy()


def _oracle(km, lm, R, f):
    op = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
    return op.evaluate(f.reshape(f.shape[0], -1)).reshape(f.shape)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize(
    "km,lm,ncells",
    [(0, 0, 5), (1, 2, 1), (2, 3, 70), (4, 4, 33), (3, 5, 64), (4, 6, 40), (8, 8, 37), (6, 10, 9)],
)
def test_fp64_random_core(km, lm, ncells):
    """Several tiles of 32 cells and a ragged tail, random core and random cells."""
    nt = len(gaunt.channels(lm))
    R = wi.random_core(nt, km, seed=km * 100 + lm)
    f = wi.random_cells(km, lm, ncells, seed=lm)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f)
    assert _rel(Q, _oracle(km, lm, R, f)) <= FP64_TOL


def test_fp64_maxwell_config1_oracle_core():
    """Maxwell molecules, Kmax = Lmax = 4, one perturbed-Maxwellian cell, core from the oracle's quadrature."""
    km = lm = 4
    R = ocore.core(km, lm, 0.0)
    f = wi.perturbed_maxwellian(km, lm, 1, seed=1)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f)
    Qo = _oracle(km, lm, R, f)
    assert _rel(Q, Qo) <= FP64_TOL
    assert np.max(np.abs(Q)) > 1e-6


def test_invariants_and_maxwellian():
    """Exact zeros at the mass, momentum and energy outputs; Q(M, M) = 0 (Sec. 4.4)."""
    km, lm = 4, 4
    nq = (lm + 1) ** 2
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=3)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    f = wi.random_cells(km, lm, 50, seed=4)
    f[0] = 0.0
    f[0, 0, 0] = 1.0
    Q = _gpu_eval(op, f)
    assert np.all(Q[:, 0, 0:4] == 0.0) and np.all(Q[:, 1, 0] == 0.0)
    assert np.all(Q[0] == 0.0)
    assert np.max(np.abs(Q[1:])) > 0


def test_deterministic_rerun():
    km, lm = 6, 6
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=5)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    f = wi.random_cells(km, lm, 100, seed=6)
    assert np.array_equal(_gpu_eval(op, f), _gpu_eval(op, f))


@pytest.mark.parametrize("km,lm,ncells,nsample", [(8, 8, 4096, 12)])
def test_fp64_full_size_sampled(km, lm, ncells, nsample):
    """Full batch size at K=L=8 (4096 cells) in the benchmark's launch configuration; seeded
    two-Maxwellian cells; oracle on sampled cells.  K=L=12 is covered, for every precision,
    by test_full_size_kl12_sampled."""
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=7)
    f = wi.two_maxwellians(km, lm, ncells, seed=3, pool=512)
    op = W.Operator(km, lm, 1.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f)
    idx = np.random.default_rng(0).choice(ncells, nsample, replace=False)
    idx[-1] = ncells - 1
    Qo = _oracle(km, lm, R, f[idx])
    assert _rel(Q[idx], Qo) <= FP64_TOL


def test_error_paths():
    op = W.Operator(2, 2, 0.0)
    f = torch.zeros(4, 3, 9, dtype=torch.float64, device="cuda")
    with pytest.raises(W.WefError) as e:
        op.evaluate(f)
    assert e.value.status == W.WEF_ENOCORE
    op.upload_core(np.zeros((len(gaunt.channels(2)), 3, 3, 3)))
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    q = torch.empty_like(f)
    with pytest.raises(W.WefError) as e:
        W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), 4, 0, ws.data_ptr() + 8, 4000, 0)
    assert e.value.status == W.WEF_EINVAL
    with pytest.raises(W.WefError):
        W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), 4, 0, ws.data_ptr(), 16, 0)


# ------------------------------------------------------------------ mixed precision (tcgen05)
# Normwise bound max|Q - Q_oracle| / max|Q_oracle| for the radial stage in BF16 / TF32 with
# FP32 accumulation (Phi and the core rounded to 8 / 10 mantissa bits).
MIXED_TOL = {"bf16": 3e-2, "tf32": 5e-3}


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("km,lm,ncells", [(1, 2, 1), (2, 3, 70), (4, 4, 33), (4, 6, 40), (8, 8, 37), (16, 2, 45), (12, 12, 3)])
def test_mixed_random_core(prec, km, lm, ncells):
    nt = len(gaunt.channels(lm))
    R = wi.random_core(nt, km, seed=km * 100 + lm + 1)
    f = wi.random_cells(km, lm, ncells, seed=lm + 1)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, prec)
    W.wef_device_status(op.h)
    err = _rel(Q, _oracle(km, lm, R, f))
    print(f"{prec} K={km} L={lm} n={ncells} normwise err {err:.3e}")
    assert err <= MIXED_TOL[prec]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_invariants_exact(prec):
    km, lm = 4, 4
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=3)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    f = wi.random_cells(km, lm, 50, seed=4)
    f[0] = 0.0
    f[0, 0, 0] = 1.0
    Q = _gpu_eval(op, f, prec)
    assert np.all(Q[:, 0, 0:4] == 0.0) and np.all(Q[:, 1, 0] == 0.0)
    assert np.all(Q[0] == 0.0)


# ------------------------------------------------------------------ radial-first (FP32 radial, FP64 angular)
RF_TOL = 2e-5  # normwise; FP32 radial contractions (f and the core rounded to FP32)


@pytest.mark.parametrize("km,lm,ncells", [(0, 0, 3), (1, 2, 1), (2, 3, 70), (4, 4, 33), (4, 6, 40), (8, 8, 37),
                                          (16, 2, 45), (12, 12, 3), (16, 16, 2)])
def test_radial_first_random_core(km, lm, ncells):
    nt = len(gaunt.channels(lm))
    R = wi.random_core(nt, km, seed=km * 100 + lm + 2)
    f = wi.random_cells(km, lm, ncells, seed=lm + 2)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, "rf32")
    err = _rel(Q, _oracle(km, lm, R, f))
    print(f"rf32 K={km} L={lm} n={ncells} normwise err {err:.3e}")
    assert err <= RF_TOL


def test_radial_first_invariants_and_rerun():
    km, lm = 4, 4
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=3)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    f = wi.random_cells(km, lm, 50, seed=4)
    f[0] = 0.0
    f[0, 0, 0] = 1.0
    Q = _gpu_eval(op, f, "rf32")
    assert np.all(Q[:, 0, 0:4] == 0.0) and np.all(Q[:, 1, 0] == 0.0)
    assert np.all(Q[0] == 0.0)
    assert np.array_equal(Q, _gpu_eval(op, f, "rf32"))


# The workload of the headline benchmark (hard spheres, Kmax = Lmax = 12, 16384 seeded
# two-Maxwellian cells) in its launch configuration, every precision against one oracle
# evaluation of 64 sampled cells (the first, the last and 62 drawn at random).
KL12_SAMPLES = 64


@pytest.fixture(scope="module")
def kl12_full():
    km = lm = 12
    ncells = 16384
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=7)
    f = wi.two_maxwellians(km, lm, ncells, seed=3, pool=512)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, ncells - 1], rng.choice(np.arange(1, ncells - 1), KL12_SAMPLES - 2,
                                                                   replace=False)]))
    assert idx.size == KL12_SAMPLES
    return km, lm, R, f, idx, _oracle(km, lm, R, f[idx])


@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32", "rf32"])
def test_full_size_kl12_sampled(kl12_full, prec):
    km, lm, R, f, idx, Qo = kl12_full
    op = W.Operator(km, lm, 1.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, prec)
    W.wef_device_status(op.h)  # no bounded wait gave up
    err = _rel(Q[idx], Qo)
    print(f"{prec} full-size ({idx.size} sampled cells) normwise err {err:.3e}")
    assert err <= {"fp64": FP64_TOL, "rf32": RF_TOL}.get(prec, MIXED_TOL.get(prec))


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("rf32", RF_TOL), ("tf32", MIXED_TOL["tf32"])])
def test_maximum_size_sampled_rows(prec, tol):
    """The largest operator the ABI accepts (Kmax = 16, Lmax = 20, N = 7497 per cell): every
    path against the oracle on sampled output rows (the invariant rows, the last one and a
    seeded sample), two cells plus a ragged third."""
    km, lm, ncells = 16, 20, 3
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=29)
    f = wi.random_cells(km, lm, ncells, seed=30)
    op = W.Operator(km, lm, 1.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, prec).reshape(ncells, -1)
    N = op.N
    rows = sorted(set([0, 1, 2, 3, op.NQ, N - 1] + list(np.random.default_rng(1).choice(N, 10, replace=False))))
    o = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
    Qo = o.evaluate_rows(f.reshape(ncells, -1), rows)
    err = _rel(Q[:, rows], Qo)
    print(f"{prec} K=17 L=20 sampled-row normwise err {err:.3e}")
    assert err <= tol
    assert np.all(Q[:, [0, 1, 2, 3, op.NQ]] == 0.0)
