"""Device time integration and linearization: RK4 on df/dt = Q(f, f) and L d by polarization
of the bilinear form.  Pinned by the Krook-Wu moment system (Maxwell molecules, isotropic
data, Sec. 5.2.1), the dense oracle's linearized operator, and the Wang Chang-Uhlenbeck
spectrum of Table 3 (Sec. 5.2.2)."""
import math

import numpy as np
import pytest
from scipy import special

import wef_inputs as wi
from conftest import golden
from oracle import basis, dense, gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _krook_wu_rhs(c, km):
    """Q of isotropic data, Maxwell molecules, B = 1/(4 pi): with a_n = c_n N_n0 / (sqrt(4 pi) n!),
    da_n/dt = sum_{j+k=n} a_j a_k j! k! / (n+1)! - a_0 a_n (Sec. 5.2.1)."""
    f = math.factorial
    N = [basis.radial_norm(n, 0) for n in range(km + 1)]
    a = [c[n] * N[n] / (math.sqrt(4 * math.pi) * f(n)) for n in range(km + 1)]
    da = [sum(a[j] * a[n - j] * f(j) * f(n - j) / f(n + 1) for j in range(n + 1)) - a[0] * a[n] for n in range(km + 1)]
    return np.array([da[n] * math.sqrt(4 * math.pi) * f(n) / N[n] for n in range(km + 1)])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("rf32", 2e-6)])
def test_rk4_relaxation_matches_moment_system(prec, tol):
    """Isotropic relaxation of Maxwell molecules: the device RK4 of the full spectral system
    (Lmax = 2, so anisotropic channels take part) equals an RK4 of the closed moment system with
    the same step; mass and energy components stay bit-for-bit constant and f stays isotropic."""
    km, lm = 5, 2
    op = W.Operator(km, lm, 0.0)
    op.upload_core(op.build_core())
    nq = (lm + 1) ** 2
    rng = np.random.default_rng(11)
    ncells = 70  # several tiles and a ragged tail; every cell its own initial state
    c0 = np.zeros((ncells, km + 1))
    c0[:, 0] = 1.0
    c0[:, 2:] = 0.1 * rng.standard_normal((ncells, km - 1))
    f = np.zeros((ncells, km + 1, nq))
    f[:, :, 0] = c0
    fd = torch.from_numpy(f).cuda()
    dt, nsteps = 0.05, 40
    op.integrate(fd, dt, nsteps, precision=prec)
    torch.cuda.synchronize()
    out = fd.cpu().numpy()
    for i in range(ncells):
        y = c0[i].copy()
        for _ in range(nsteps):
            k1 = _krook_wu_rhs(y, km)
            k2 = _krook_wu_rhs(y + 0.5 * dt * k1, km)
            k3 = _krook_wu_rhs(y + 0.5 * dt * k2, km)
            k4 = _krook_wu_rhs(y + dt * k3, km)
            y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        assert np.max(np.abs(out[i, :, 0] - y)) < tol
        assert abs(out[i, 2, 0] - c0[i, 2]) > 1e-4  # something relaxed
    assert np.max(np.abs(out[:, :, 1:])) < tol  # stays isotropic
    assert np.array_equal(out[:, 0, 0], c0[:, 0]) and np.array_equal(out[:, 1, 0], c0[:, 1])


def test_rk4_conserves_anisotropic():
    """Random anisotropic data, hard spheres: mass, momentum and energy components are unchanged
    to the bit by any number of steps (the projection zeroes them in every stage)."""
    km, lm = 3, 4
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=3)
    op = W.Operator(km, lm, 1.0)
    op.upload_core(R)
    f = torch.from_numpy(wi.random_cells(km, lm, 45, seed=4)).cuda()
    f0 = f.clone()
    op.integrate(f, 0.01, 7)
    torch.cuda.synchronize()
    for k, q in [(0, 0), (0, 1), (0, 2), (0, 3), (1, 0)]:
        assert torch.equal(f[:, k, q], f0[:, k, q])
    assert not torch.equal(f, f0)


def test_rk4_zero_steps_and_empty():
    op = W.Operator(2, 2, 0.0)
    op.upload_core(op.build_core())
    f = torch.from_numpy(wi.random_cells(2, 2, 5, seed=1)).cuda()
    f0 = f.clone()
    op.integrate(f, 0.1, 0)
    assert torch.equal(f, f0)
    e = torch.empty((0, 3, 9), dtype=torch.float64, device="cuda")
    op.integrate(e, 0.1, 3)
    with pytest.raises(W.WefError):
        W.wef_integrate(op.h, f.data_ptr(), 5, 0.1, 1, 0, f.data_ptr(), 8, torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("prec", ["fp64", "rf32"])
def test_linearized_apply_matches_oracle(prec):
    """Cell i holds base state c0_i and direction e_(i mod N): out_i = column of L(c0_i),
    L[a1, a2] = C[a1, c0, a2] + C[a1, a2, c0] from the dense oracle.  (The BF16/TF32 paths are
    not used for L: the polarization difference magnifies their relative error by |c0| / |d|.)"""
    km, lm = 2, 3
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=17)
    op = W.Operator(km, lm, 0.0)
    op.upload_core(R)
    N = (km + 1) * (lm + 1) ** 2
    ncells = N + 9
    rng = np.random.default_rng(5)
    c0 = rng.standard_normal((ncells, N))
    d = np.zeros((ncells, N))
    d[np.arange(ncells), np.arange(ncells) % N] = 1.0
    out = op.linearized_apply(torch.from_numpy(c0).cuda(), torch.from_numpy(d).cuda(), precision=prec)
    torch.cuda.synchronize()
    o = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
    S = [o.slice(a) for a in range(N)]
    ref = np.stack([np.array([S[a][i % N] @ c0[i] + c0[i] @ S[a][:, i % N] for a in range(N)]) for i in range(ncells)])
    tol = {"fp64": 1e-11, "rf32": 3e-5}[prec]
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= tol * np.max(np.abs(ref))


def _wcu_closed_form(k, l):
    """Maxwell molecules, B = 1/(4 pi), unit density: the (k, l) Laguerre-harmonic function is an
    eigenfunction of L with lambda_kl = 1/2 int_{-1}^{1} [c^n P_l(c) + s^n P_l(s) - 1 - delta] dx,
    n = 2k + l, c = sqrt((1+x)/2), s = sqrt((1-x)/2), delta = 1 for k = l = 0 (Sec. 5.2.2)."""
    x, w = np.polynomial.legendre.leggauss(60)
    cc, ss = np.sqrt((1 + x) / 2), np.sqrt((1 - x) / 2)
    n = 2 * k + l
    val = cc**n * special.eval_legendre(l, cc) + ss**n * special.eval_legendre(l, ss) - 1.0 - (1.0 if k == l == 0 else 0.0)
    return 0.5 * np.sum(w * val)


def test_wcu_spectrum_on_device():
    """L at the reference Maxwellian assembled column by column on the device (Kmax = 4,
    Lmax = 6, Maxwell molecules): each (l, m) block is diagonal with lambda_kl, and the sorted
    spectrum normalised by the first relaxation mode is Table 3's."""
    km, lm = 4, 6
    op = W.Operator(km, lm, 0.0)
    op.upload_core(op.build_core())
    K, NQ = km + 1, (lm + 1) ** 2
    N = K * NQ
    c0 = np.zeros((N, N))
    c0[:, 0] = 1.0
    L = op.linearized_apply(torch.from_numpy(c0).cuda(), torch.eye(N, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    L = L.cpu().numpy().T  # column a2 = L e_a2
    ev = []
    for l in range(lm + 1):
        for m in range(-l, l + 1):
            idx = [k * NQ + l * l + l + m for k in range(K)]
            B = L[np.ix_(idx, idx)]
            for k in range(K):
                lam = 0.0 if (l == 0 and k < 2) or (l == 1 and k == 0) else _wcu_closed_form(k, l)
                assert B[k, k] == pytest.approx(lam, abs=1e-12)
            assert np.max(np.abs(B - np.diag(np.diag(B)))) < 1e-12
            ev += list(np.diag(B))
    off = L.copy()
    for l in range(lm + 1):
        for m in range(-l, l + 1):
            idx = [k * NQ + l * l + l + m for k in range(K)]
            off[np.ix_(idx, idx)] = 0.0
    assert np.max(np.abs(off)) < 1e-12  # no coupling between different (l, m)
    ev = np.sort(np.array(ev))[::-1]
    lam6 = abs(ev[5])
    for first, last, ratio, bound in golden("table3_wcu.txt"):
        seg = ev[int(first) - 1:int(last)] / lam6
        assert np.max(np.abs(seg - float(ratio))) <= max(float(bound), 1e-15) * 100
