"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Bar (tests/_parity.py): for every compared cell, the infinity norm of Q_gpu - Q_oracle over
its output rows, divided by max(|Q_oracle| of the cell, EPS * the largest sum of |terms|
of its rows), is at most 1e-12 on the FP64 path and a stated multiple of the unit
roundoff of the radial operands on the mixed paths.  Inputs are seeded (wef_inputs); the
core is a random stand-in (the contraction is what is tested), the oracle's own quadrature
core, or at the headline size the hard-sphere core of the library's host quadrature (an
input to both sides, pinned to the oracle's core at small sizes in tests/test_abi.py)."""
import numpy as np
import pytest

import wef_inputs as wi
from _parity import FP64_TOL, cell_errors, summary, tolerance
from oracle import core as ocore
from oracle import dense, gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402



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


def _oracle(km, lm, R, f, rows=None):
    """Q and the sums of |terms| T of the dense oracle, [ncells, K, NQ] (or [ncells, rows])."""
    op = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
    Q, T = op.evaluate_rows_with_terms(f.reshape(f.shape[0], -1), rows)
    if rows is None:
        return Q.reshape(f.shape), T.reshape(f.shape)
    return Q, T


def _check(Q, oracle, prec, what, physical=False):
    """Assert the per-cell guarded error of Q against (Qo, T) and print it."""
    Qo, T = oracle
    s = summary(cell_errors(Q, Qo, T))
    tol = tolerance(prec, physical)
    print(f"PARITY {prec} {what}: per-cell max {s['max']:.3e} median {s['median']:.3e} over {s['cells']} cells "
          f"(bound {tol:.2e})")
    assert s["max"] <= tol, (prec, what, s)


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
    _check(Q, _oracle(km, lm, R, f), "fp64", f"random core K={km + 1} L={lm} n={ncells}")


def test_fp64_maxwell_config1_oracle_core():
    """Maxwell molecules, Kmax = Lmax = 4, one perturbed-Maxwellian cell, core from the oracle's quadrature."""
    km = lm = 4
    R = ocore.core(km, lm, 0.0)
    f = wi.perturbed_maxwellian(km, lm, 1, seed=1)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f)
    _check(Q, _oracle(km, lm, R, f), "fp64", "Maxwell K=L=4 oracle core, 1 cell")
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
    _check(Q[idx], _oracle(km, lm, R, f[idx]), "fp64", f"K=L=8 x {ncells} cells, {nsample} sampled")


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
    _check(Q, _oracle(km, lm, R, f), prec, f"random core K={km + 1} L={lm} n={ncells}")


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
# (13, 6): K = 14 with three q2 groups at two CTAs per SM; (14, 8) and (15, 12): one CTA per SM
# from K = 15 on at small Lmax; (6, 12): shared-memory accumulators (the columns of K = 7 at
# Lmax = 12 do not fit five CTAs' shares of tensor memory)
@pytest.mark.parametrize("km,lm,ncells", [(0, 0, 3), (1, 2, 1), (2, 3, 70), (4, 4, 33), (4, 6, 40), (8, 8, 37),
                                          (16, 2, 45), (12, 12, 3), (16, 16, 2), (13, 6, 29), (14, 8, 33),
                                          (15, 12, 5), (6, 12, 17)])
def test_radial_first_random_core(km, lm, ncells):
    nt = len(gaunt.channels(lm))
    R = wi.random_core(nt, km, seed=km * 100 + lm + 2)
    f = wi.random_cells(km, lm, ncells, seed=lm + 2)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, "rf32")
    _check(Q, _oracle(km, lm, R, f), "rf32", f"random core K={km + 1} L={lm} n={ncells}")


# radial-first with the first radial stage on the tcgen05 tensor cores (split TF32): the
# radial-function counts it is compiled for, ragged tails, a shell wider than the program's
# q2 blocks (Lmax = 16), and agreement with the CUDA-core radial-first path
@pytest.mark.parametrize("km,lm,ncells", [(8, 8, 37), (10, 10, 45), (12, 12, 33), (12, 4, 70), (8, 3, 5)])
def test_radial_first_tensor_core_stage1(km, lm, ncells):
    nt = len(gaunt.channels(lm))
    R = wi.random_core(nt, km, seed=km * 100 + lm + 9)
    f = wi.random_cells(km, lm, ncells, seed=lm + 9)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, "rftc")
    W.wef_device_status(op.h)  # no bounded wait gave up
    _check(Q, _oracle(km, lm, R, f), "rftc", f"random core K={km + 1} L={lm} n={ncells}")
    assert np.all(Q[:, 0, 0:4] == 0.0) and np.all(Q[:, 1, 0] == 0.0)
    assert np.array_equal(Q, _gpu_eval(op, f, "rftc"))  # deterministic
    d = np.abs(Q - _gpu_eval(op, f, "rf32")).max() / np.abs(Q).max()
    assert d < 2.0 ** -20, d  # both paths are FP32-accurate in the radial products


def test_radial_first_tensor_core_wide_shell():
    """Kmax = 12 with Lmax = 16: the largest shells' accumulators (33 q1) take one CTA per SM."""
    km, lm, ncells = 12, 16, 3
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=31)
    f = wi.random_cells(km, lm, ncells, seed=32)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, "rftc").reshape(ncells, -1)
    rows = sorted(set([0, 1, 2, 3, op.NQ, op.N - 1] + list(np.random.default_rng(2).choice(op.N, 10, replace=False))))
    _check(Q[:, rows], _oracle(km, lm, R, f, rows), "rftc", "K=13 L=16 sampled rows")


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
# evaluation of sampled cells (the first, the last and the others drawn at random): with the
# hard-sphere core of the library's quadrature (the physics whose error the paper's accuracy
# argument concerns) on 64 cells, and with a random stand-in core on 16.
def _kl12_case(R, nsample, seed):
    km = lm = 12
    ncells = 16384
    f = wi.two_maxwellians(km, lm, ncells, seed=3, pool=1024)
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, ncells - 1], rng.choice(np.arange(1, ncells - 1), nsample - 2,
                                                                   replace=False)]))
    assert idx.size == nsample
    return km, lm, R, f, idx, _oracle(km, lm, R, f[idx])


@pytest.fixture(scope="module")
def kl12_hs():
    op = W.Operator(12, 12, 1.0)
    R = op.build_core()  # host quadrature (Sec. 4.3, App. A-B), hard spheres, paddings 20/20
    op.close()
    return _kl12_case(R, 64, 0)


@pytest.fixture(scope="module")
def kl12_random():
    return _kl12_case(wi.random_core(len(gaunt.channels(12)), 12, seed=7), 16, 1)


@pytest.mark.parametrize("core", ["kl12_hs", "kl12_random"])
@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32", "rf32", "rftc"])
def test_full_size_kl12_sampled(request, core, prec):
    km, lm, R, f, idx, oracle = request.getfixturevalue(core)
    op = W.Operator(km, lm, 1.0)
    op.upload_core(R)
    Q = _gpu_eval(op, f, prec)
    W.wef_device_status(op.h)  # no bounded wait gave up
    _check(Q[idx], oracle, prec, f"{core} 16384 cells, {idx.size} sampled", physical=core == "kl12_hs")
    assert np.all(Q[:, 0, 0:4] == 0.0) and np.all(Q[:, 1, 0] == 0.0)  # invariants, every cell


@pytest.mark.parametrize("prec", ["fp64", "rf32", "tf32"])
def test_maximum_size_sampled_rows(prec):
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
    _check(Q[:, rows], _oracle(km, lm, R, f, rows), prec, "K=17 L=20 sampled rows")
    assert np.all(Q[:, [0, 1, 2, 3, op.NQ]] == 0.0)
