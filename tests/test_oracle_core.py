"""Pins of the oracle's kinematic core quadrature (§3, §4.3, §4.4, §5.1, §5.2, §5.3).

Each pin is fixed by something other than the oracle: closed forms (Krook-Wu
moment system, exact stress relaxation and moment closure of Maxwell molecules,
Wang Chang-Uhlenbeck eigenvalues), values the paper prints (Table 3, Table 5),
exact brute-force 8D evaluations of the weak form (Maxwell molecules in (v, w);
any power law in centre-of-mass and relative velocity), the padding convergence
of §5.1, and the analytic conservation laws that the raw quadrature must already
satisfy to rounding before the §4.4 zeroing."""
import math

import numpy as np
import pytest
from scipy import special

import wef_inputs as wi
from conftest import golden
from oracle import basis, core, dense, gaunt


# ----------------------------------------------------------------- Maxwell molecules
def test_krook_wu_isotropic_maxwell():
    """Isotropic inputs, Maxwell molecules (B = 1/4pi): with a_n = c_n N_n0 / (sqrt(4pi) n!)
    the Fourier-transformed equation gives the closed triangular system
    da_n/dt = sum_{j+k=n} a_j a_k j! k! / (n+1)! - a_0 a_n, exact at any truncation (§5.2.1)."""
    km = 5
    R = dense.conservation_zeroing(core.core(km, 0, 0.0), 0)
    op = dense.DenseOperator(km, 0, R)
    rng = np.random.default_rng(7)
    for _ in range(3):
        c = 0.2 * rng.standard_normal(km + 1)
        c[0] = 1.0
        N = [basis.radial_norm(n, 0) for n in range(km + 1)]
        f = math.factorial
        a = [c[n] * N[n] / (math.sqrt(4 * math.pi) * f(n)) for n in range(km + 1)]
        da = [sum(a[j] * a[n - j] * f(j) * f(n - j) / f(n + 1) for j in range(n + 1)) - a[0] * a[n] for n in range(km + 1)]
        Qex = np.array([da[n] * math.sqrt(4 * math.pi) * f(n) / N[n] for n in range(km + 1)])
        Q = op.evaluate(c[None, :])[0]
        assert np.allclose(Q, Qex, rtol=0, atol=1e-14)


@pytest.fixture(scope="module")
def maxwell_33():
    """The dense Maxwell-molecule operator at Kmax = Lmax = 3 (oracle core, zeroed)."""
    return dense.DenseOperator(3, 3, dense.conservation_zeroing(core.core(3, 3, 0.0), 3))


def test_maxwell_stress_and_heat_flux_relaxation_nonlinear(maxwell_33):
    """Maxwell molecules (§5.2): the traceless pressure tensor relaxes exactly at the first
    l = 2 rate, whatever else f contains (and, at zero momentum, the heat flux at the first
    l = 1 relaxation rate, 2/3 of it).  In the basis, phi_000 = 1 and phi_{0,(1,m)} =
    v_(y,z,x), so c_000 is the density and c_{0,(1,.)} the momentum density p, and the
    k = 0, l = 2 rows of the full nonlinear operator are
        Q_{0,(2,m)} = lambda_{0,2} (c_000 c_{0,(2,m)} - N_02 |p|^2 Y_2m(p / |p|)),
    the Galerkin form of d(rho P_ij)/dt = -nu rho (P_ij - p delta_ij) with P the central
    second moment.  Checked on random f with every mode (Kmax = Lmax = 3) against the
    closed-form lambda_{0,2}: all other products of modes must cancel in these rows."""
    op = maxwell_33
    K, NQ = op.K, op.NQ
    lam = _wcu_closed_form(0, 2)
    rng = np.random.default_rng(5)
    for _ in range(3):
        c = 0.3 * rng.standard_normal((K, NQ))
        c[0, 0] = 1.3
        Q = op.evaluate(c.reshape(1, -1)).reshape(K, NQ)
        p = np.array([c[0, 3], c[0, 1], c[0, 2]])  # (x, y, z) from m = 1, -1, 0
        Y2 = basis.real_sh_all(2, (p / np.linalg.norm(p))[None, :])[0, 4:9]
        expect = lam * (c[0, 0] * c[0, 4:9] - basis.radial_norm(0, 2) * (p @ p) * Y2)
        assert np.max(np.abs(Q[0, 4:9] - expect)) < 1e-13 * np.max(np.abs(expect))
    # the heat flux (k = 1, l = 1 rows): at zero momentum it relaxes linearly at lambda_{1,1},
    # two thirds of the stress rate (the Prandtl number 2/3 of Maxwell molecules)
    lam11 = _wcu_closed_form(1, 1)
    assert lam11 / lam == pytest.approx(2.0 / 3.0, rel=1e-13)
    for _ in range(3):
        c = 0.3 * rng.standard_normal((K, NQ))
        c[0, 0], c[0, 1:4] = 1.1, 0.0
        Q = op.evaluate(c.reshape(1, -1)).reshape(K, NQ)
        expect = lam11 * c[0, 0] * c[1, 1:4]
        assert np.max(np.abs(Q[1, 1:4] - expect)) < 1e-13 * np.max(np.abs(expect))


def test_maxwell_moment_closure_on_projected_maxwellians(maxwell_33):
    """Maxwell molecules (§5.2): the collision rate of a degree-n moment depends only on
    moments of degree <= n.  The projection of a drifting Maxwellian M_{U,T} (any U, T)
    reproduces every moment of degree <= min(Lmax, 2 Kmax + 1) = 3 exactly, so the rows
    2k + l <= 3 of Q vanish to rounding (Q(M, M) = 0), while the higher rows do not."""
    op = maxwell_33
    lq = np.array([basis.lm_of_q(q)[0] for q in range(op.NQ)])
    deg = 2 * np.arange(op.K)[:, None] + lq[None, :]
    for U, T in (([0.3, -0.2, 0.1], 1.4), ([0.0, 0.0, 0.5], 0.6)):
        c = wi.maxwellian_coefficients(3, 3, np.array([0.8]), np.array([U]), np.array([T]))
        Q = op.evaluate(c.reshape(1, -1)).reshape(op.K, op.NQ)
        high = np.abs(Q[deg > 3]).max()
        assert high > 1e-6
        assert np.abs(Q[deg <= 3]).max() < 1e-11 * high


def _wcu_closed_form(k, l):
    """lambda_kl = 1/2 int_{-1}^{1} [c^{2k+l} P_l(c) + s^{2k+l} P_l(s) - 1 - delta_k0 delta_l0] dx,
    c = sqrt((1+x)/2), s = sqrt((1-x)/2): Maxwell molecules, B = 1/(4 pi), unit density."""
    x, w = np.polynomial.legendre.leggauss(60)
    cc, ss = np.sqrt((1 + x) / 2), np.sqrt((1 - x) / 2)
    n = 2 * k + l
    val = cc**n * special.eval_legendre(l, cc) + ss**n * special.eval_legendre(l, ss) - 1.0 - (1.0 if k == l == 0 else 0.0)
    return 0.5 * np.sum(w * val)


@pytest.fixture(scope="module")
def maxwell_linear_blocks():
    """Radial blocks L^{(l)}[k1, k2] of the linearized operator at c_000 = 1 (§5.3.1), Kmax=4, Lmax=6."""
    km, lm = 4, 6
    chans = [ch for ch in gaunt.channels(lm) if ch[1] == 0 or ch[2] == 0]
    R = core.core(km, lm, 0.0, chans=chans)
    g0 = 1.0 / math.sqrt(4 * math.pi)  # G[(l,m),(0,0),(l,m)]
    blocks = {}
    for l in range(lm + 1):
        B = (R[chans.index((l, 0, l))][:, 0, :] + R[chans.index((l, l, 0))][:, :, 0]) * g0
        if l == 0:
            B[0, :] = 0.0
            B[1, :] = 0.0
        if l == 1:
            B[0, :] = 0.0
        blocks[l] = B
    return blocks


def test_wcu_spectrum_table3(maxwell_linear_blocks):
    """Table 3: eigenvalues normalised by the first relaxation mode, ascending |lambda|;
    modes 1-5 are the collision invariants (0), then -1, -1.5, -1.75, -1.8 with their degeneracies."""
    ev = []
    for l, B in maxwell_linear_blocks.items():
        lam = np.linalg.eigvals(B)
        assert np.max(np.abs(lam.imag)) < 1e-13
        ev += list(np.repeat(lam.real, 2 * l + 1))
    ev = np.sort(np.array(ev))[::-1]  # 0 first, then decreasing
    assert np.all(ev < 1e-13)  # H-theorem: non-positive spectrum
    lam6 = abs(ev[5])
    for first, last, ratio, bound in golden("table3_wcu.txt"):
        seg = ev[int(first) - 1:int(last)] / lam6
        assert np.max(np.abs(seg - float(ratio))) <= max(float(bound), 1e-15) * 10


def test_wcu_closed_form_diagonal(maxwell_linear_blocks):
    """For Maxwell molecules the Laguerre x spherical-harmonic functions are eigenfunctions:
    each block is diagonal with the closed-form eigenvalues lambda_kl."""
    for l, B in maxwell_linear_blocks.items():
        for k in range(B.shape[0]):
            assert B[k, k] == pytest.approx(_wcu_closed_form(k, l), abs=1e-13)
        assert np.max(np.abs(B - np.diag(np.diag(B)))) < 1e-13


def test_bruteforce_8d_maxwell():
    """The weak form of §2.3 evaluated directly in 8D (Gauss-Hermite in v and w, an exact
    sphere rule for u'), exact for Maxwell molecules at small (Kmax, Lmax) because the
    integrand is a polynomial times the Gaussian weight; compared with C = R * G of the
    oracle core (raw, before any zeroing) entry by entry."""
    km, lm = 1, 2
    K, NQ = km + 1, (lm + 1) ** 2
    N = K * NQ
    lq = np.array([basis.lm_of_q(q)[0] for q in range(NQ)])
    op = dense.DenseOperator(km, lm, core.core(km, lm, 0.0))
    C_fact = np.stack([op.slice(a) for a in range(N)])

    def phi(p):
        r = np.linalg.norm(p, axis=-1)
        Y = basis.real_sh_all(lm, p / np.maximum(r, 1e-300)[..., None])
        Rr = basis.radial_all(K, lm, r)[..., lq]  # [..., K, NQ]
        return (Rr * Y[..., None, :]).reshape(p.shape[:-1] + (N,))

    x, w = np.polynomial.hermite_e.hermegauss(7)
    w = w / math.sqrt(2 * math.pi)
    grid = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    gw = np.einsum("i,j,k->ijk", w, w, w).reshape(-1)
    sph, sw = gaunt.sphere_rule(2 * km + lm + 1)
    sw = sw / (4 * math.pi)  # B = 1/(4 pi)
    phiw = phi(grid)  # phi at all w (and v) nodes
    C = np.zeros((N, N, N))
    for i, v in enumerate(grid):
        V = 0.5 * (v + grid)  # [Pw, 3]
        u = np.linalg.norm(v - grid, axis=1)
        vp = V[:, None, :] + 0.5 * u[:, None, None] * sph[None, :, :]
        gain = np.einsum("s,psa->pa", sw, phi(vp))
        loss = phiw[i][None, :] * sw.sum()
        C += gw[i] * np.einsum("p,pa,b,pc->abc", gw, gain - loss, phiw[i], phiw)
    assert np.max(np.abs(C - C_fact)) < 1e-13 * np.max(np.abs(C))


@pytest.mark.parametrize("km,lm", [(1, 2), (2, 1)])
@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0])
def test_bruteforce_8d_any_gamma(gamma, km, lm):
    """The same weak form for any power law u^gamma, exact at small (Kmax, Lmax).

    Centre of mass V = (v + w)/2 and relative velocity g = v - w (unit Jacobian) split the
    Maxwellian pair weight into e^{-|V|^2} e^{-|g|^2/4}, and u^gamma = |g|^gamma becomes part
    of the radial weight of g.  Every test function is a polynomial in (V, g, |g| sigma), so
    after exact sphere rules over g/|g| and sigma (which annihilate the odd powers of |g|) the
    radial integrand is an even polynomial in |g|: with s = |g|^2/4 the generalized
    Gauss-Laguerre rule of weight s^{(1+gamma)/2} e^{-s} integrates it exactly.  Independent of
    the oracle's Duffy-patched (z, x, y) quadrature; this pins the VHS core (gamma = 0.5) and
    the hard-sphere core (gamma = 1) entry by entry, raw, before any zeroing."""
    K, NQ = km + 1, (lm + 1) ** 2
    N = K * NQ
    lq = np.array([basis.lm_of_q(q)[0] for q in range(NQ)])
    op = dense.DenseOperator(km, lm, core.core(km, lm, gamma))
    C_fact = np.stack([op.slice(a) for a in range(N)])

    def phi(p):
        r = np.linalg.norm(p, axis=-1)
        Y = basis.real_sh_all(lm, p / np.maximum(r, 1e-300)[..., None])
        Rr = basis.radial_all(K, lm, r)[..., lq]  # [..., K, NQ]
        return (Rr * Y[..., None, :]).reshape(p.shape[:-1] + (N,))

    deg = 2 * (2 * km + lm)  # degree of phi_b(v) phi_c(w) in g
    # V: weight pi^{-3/2} e^{-|V|^2}, i.e. x / sqrt 2 with x standard normal per axis; the
    # integrand has degree deg + 2 km + lm in V
    x, wx = np.polynomial.hermite_e.hermegauss((deg + 2 * km + lm) // 2 + 1)
    wx = wx / math.sqrt(2 * math.pi)
    Vn = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3) / math.sqrt(2.0)
    Vw = np.einsum("i,j,k->ijk", wx, wx, wx).reshape(-1)
    # g = 2 sqrt(s) ghat: (4 pi)^{-3/2} e^{-|g|^2/4} |g|^gamma dg
    #   = (4 pi)^{-3/2} 2^{2+gamma} s^{(1+gamma)/2} e^{-s} ds dghat
    s, ws = special.roots_genlaguerre((deg + 2 * km + lm) // 2 + 1, 0.5 * (1.0 + gamma))
    ws = ws * 2.0 ** (2.0 + gamma) * (4 * math.pi) ** -1.5
    gh, wgh = gaunt.sphere_rule(deg + 2 * km + lm + 1)
    g = (2.0 * np.sqrt(s))[:, None, None] * gh[None, :, :]  # [S, G, 3]
    gw = (ws[:, None] * wgh[None, :]).reshape(-1)
    g = g.reshape(-1, 3)
    r = np.linalg.norm(g, axis=1)
    sph, sw = gaunt.sphere_rule(2 * km + lm + 1)
    sw = sw / (4 * math.pi)  # B = u^gamma / (4 pi); u^gamma is in the g weight
    C = np.zeros((N, N, N))
    for V, wV in zip(Vn, Vw):
        v, w = V + 0.5 * g, V - 0.5 * g
        pv, pw = phi(v), phi(w)
        vp = V[None, None, :] + 0.5 * r[:, None, None] * sph[None, :, :]
        gain = np.einsum("s,psa->pa", sw, phi(vp))
        loss = pv * sw.sum()
        G = (gain - loss) * (wV * gw)[:, None]
        C += ((G[:, :, None] * pv[:, None, :]).reshape(len(gw), N * N).T @ pw).reshape(N, N, N)
    assert np.max(np.abs(C - C_fact)) < 1e-13 * np.max(np.abs(C))


# ----------------------------------------------------------------- hard spheres
def test_chapman_enskog_viscosity_table5():
    """Table 5: f_mu = L_00 [L^{-1}]_00 of the l = 2 block for hard spheres; Kmax = 1 is 205/202."""
    g0 = 1.0 / math.sqrt(4 * math.pi)
    for km, ref in golden("table5_viscosity.txt"):
        km = int(km)
        R = core.core(km, 2, 1.0, chans=[(2, 0, 2), (2, 2, 0)])
        B = (R[0][:, 0, :] + R[1][:, :, 0]) * g0
        fmu = B[0, 0] * np.linalg.inv(B)[0, 0]
        assert fmu == pytest.approx(float(ref), abs=6e-7)
        if km == 1:
            assert fmu == pytest.approx(205.0 / 202.0, rel=1e-13)


def test_raw_core_conserves_before_zeroing():
    """§4.4: the slices that the null-space correction zeroes differ from zero only by quadrature
    error.  Checked on the raw hard-sphere core (the part symmetric in (a2, a3), which is all
    that Q sees), together with the detailed-balance slice R^(000)_{k1,0,0}."""
    km, lm = 3, 3
    ch = gaunt.channels(lm)
    idx = gaunt.channel_index(lm)
    R = core.core(km, lm, 1.0)
    scale = np.max(np.abs(R))
    res = 0.0
    for (l1, l2, l3), c in idx.items():
        sym = R[c] + R[idx[(l1, l3, l2)]].transpose(0, 2, 1)
        if l1 == 0:
            res = max(res, np.max(np.abs(sym[0])), np.max(np.abs(sym[1])))
        if l1 == 1:
            res = max(res, np.max(np.abs(sym[0])))
    res = max(res, np.max(np.abs(R[idx[(0, 0, 0)]][:, 0, 0])))
    assert res < 1e-13 * scale


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_padding_convergence(gamma):
    """The convergence study of §5.1 (relative l-infinity core error at Kmax = Lmax = 4 against
    the Duffy padding): the error falls exponentially to machine precision, alike for Maxwell
    molecules and hard spheres.  Checked on every seventh channel against padding 24: the
    unpadded rule is off by more than 1e-5, padding 10 is below 1e-6, padding 20 (the
    library default) below 1e-12."""
    km = lm = 4
    chans = gaunt.channels(lm)[::7]
    ref = core.core(km, lm, gamma, pad_rad=24, pad_ang=24, chans=chans)
    err = {}
    for p in (0, 10, 20):
        R = core.core(km, lm, gamma, pad_rad=p, pad_ang=p, chans=chans)
        err[p] = np.max(np.abs(R - ref)) / np.max(np.abs(ref))
    assert err[0] > 1e-5 and err[10] < 1e-6 and err[20] < 1e-12
    assert err[0] > err[10] > err[20]
