"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Holds no arithmetic of the collision operator: no Gaunt coefficients, no
kinematic core, no contraction.  It draws coefficient vectors f[cell, k, q]
(q = l^2 + l + m, k = 0..Kmax) shaped like the paper's workloads (§5: perturbed
and shifted Maxwellians) and random stand-in cores for parity tests.

To draw Maxwellian coefficients it needs the Galerkin basis itself
(phi_klm = R_kl Y_lm with the conventions below, which every other part of this
repository shares); that basis is written out here on its own:
R_kl(v) = N_kl v^l L_k^{(l+1/2)}(v^2/2), N_kl^2 = 2^{1-l} pi^{3/2} k!/Gamma(k+l+3/2);
real spherical harmonics without Condon-Shortley phase, cos-type for m > 0,
sin-type for m < 0.

Recipes (seeded numpy PCG64 streams):
* perturbed_maxwellian: c_000 = 1, plus 1e-2 * 2^-(k+l) * N(0,1) on every (k,l,m) mode.
* two_maxwellians: each cell rho1 M(U1,T1) + rho2 M(U2,T2) projected onto the basis,
  rho1 ~ U[0.25, 0.75], rho2 = 1 - rho1, U_i uniform in the ball |U| <= 0.5,
  T1 = r^-1/2, T2 = r^1/2 with r log-uniform in [0.5, 2] (so T2/T1 = r).
* random_core: R[c, k1, k2, k3] ~ N(0, 1) * 0.1, a stand-in core for contraction parity.
"""
import math

import numpy as np

__all__ = ["perturbed_maxwellian", "two_maxwellians", "maxwellian_coefficients", "random_core", "random_cells"]


def _nq(lmax):
    return (lmax + 1) ** 2


def perturbed_maxwellian(kmax, lmax, ncells, seed=1):
    """f[cell, k, q]: unit Maxwellian (c_000 = 1) plus 1e-2 * 2^-(k+l) N(0,1) on every mode."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K, NQ = kmax + 1, _nq(lmax)
    lq = np.array([int(math.isqrt(q)) for q in range(NQ)])
    amp = 1e-2 * 2.0 ** (-(np.arange(K)[:, None] + lq[None, :]))
    f = amp[None] * rng.standard_normal((ncells, K, NQ))
    f[:, 0, 0] += 1.0
    return f


def random_cells(kmax, lmax, ncells, seed=0, scale=1.0):
    """f[cell, k, q] ~ N(0, scale^2): generic inputs for bilinear-form parity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal((ncells, kmax + 1, _nq(lmax)))


def random_core(n_channels, kmax, seed=0, scale=0.1):
    """A stand-in core R[c, k1, k2, k3] ~ N(0, scale^2) for contraction parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = kmax + 1
    return scale * rng.standard_normal((n_channels, K, K, K))


# ---------------------------------------------------------------- basis (inputs only)
def _lgamma(x):
    return math.lgamma(x)


def _radial_norm(k, l):
    return math.exp(0.5 * ((1 - l) * math.log(2.0) + 1.5 * math.log(math.pi) + _lgamma(k + 1) - _lgamma(k + l + 1.5)))


def _laguerre_table(K, a, x):
    """L_k^{(a)}(x) for k < K by the three-term recurrence; x any array."""
    out = [np.ones_like(x)]
    if K > 1:
        out.append(1.0 + a - x)
    for k in range(1, K - 1):
        out.append(((2 * k + 1 + a - x) * out[k] - (k + a) * out[k - 1]) / (k + 1))
    return out


def _legendre_table(L, t):
    out = [np.ones_like(t), t]
    for l in range(1, L):
        out.append(((2 * l + 1) * t * out[l] - l * out[l - 1]) / (l + 1))
    return out[: L + 1]


def _real_sh_unit(lmax, n):
    """Real spherical harmonics Y_q(n) for unit vectors n[..., 3] -> [..., NQ]."""
    x, y, z = n[..., 0], n[..., 1], np.clip(n[..., 2], -1.0, 1.0)
    s = np.sqrt(np.clip(1.0 - z * z, 0.0, None))
    ph = np.arctan2(y, x)
    out = np.zeros(n.shape[:-1] + (_nq(lmax),))
    pmm = np.ones_like(z)
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
        p_prev, p = None, pmm
        for l in range(m, lmax + 1):
            if l == m + 1:
                p_prev, p = p, (2 * m + 1) * z * pmm
            elif l > m + 1:
                p_prev, p = p, ((2 * l - 1) * z * p - (l + m - 1) * p_prev) / (l - m)
            nrm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(_lgamma(l - m + 1) - _lgamma(l + m + 1)))
            if m == 0:
                out[..., l * l + l] = nrm * p
            else:
                out[..., l * l + l + m] = math.sqrt(2.0) * nrm * p * np.cos(m * ph)
                out[..., l * l + l - m] = math.sqrt(2.0) * nrm * p * np.sin(m * ph)
    return out


def maxwellian_coefficients(kmax, lmax, rho, U, T):
    """c[k, q] of rho * M(U, T) for arrays rho[n], U[n, 3], T[n] -> [n, K, NQ].

    c_a = integral of M(U,T)(v) phi_a(v) dv (orthonormality under the reference
    Maxwellian).  Computed for the drift along z (only m = 0 survives) with a
    product rule that is exact for the polynomial integrand (Gauss-Hermite in
    v_z, Gauss-Laguerre in rho_perp^2 / (2T)), then turned to the direction of U
    by the addition theorem: c_klm = c_kl0 sqrt(4 pi / (2l+1)) Y_lm(U_hat)."""
    rho = np.asarray(rho, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(-1, 3)
    T = np.asarray(T, dtype=np.float64)
    K, NQ = kmax + 1, _nq(lmax)
    n_h = kmax + (lmax + 1) // 2 + 2
    n_l = kmax + (lmax + 1) // 2 + 2
    xi, wxi = np.polynomial.hermite_e.hermegauss(n_h)
    wxi = wxi / math.sqrt(2.0 * math.pi)
    sl, wsl = np.polynomial.laguerre.laggauss(n_l)
    Um = np.linalg.norm(U, axis=1)
    st = np.sqrt(T)
    vz = Um[:, None, None] + st[:, None, None] * xi[None, :, None]  # [n, h, 1]
    rp2 = 2.0 * T[:, None, None] * sl[None, None, :]  # [n, 1, l]
    v2 = vz * vz + rp2  # [n, h, l]
    v = np.sqrt(v2)
    cth = np.where(v > 0, vz / np.where(v > 0, v, 1.0), 1.0)
    w = wxi[None, :, None] * wsl[None, None, :]
    zon = np.zeros((rho.size, K, lmax + 1))
    Pl = _legendre_table(lmax, cth)
    for l in range(lmax + 1):
        Lk = _laguerre_table(K, l + 0.5, 0.5 * v2)
        yl0 = math.sqrt((2 * l + 1) / (4 * math.pi)) * v**l * Pl[l]
        for k in range(K):
            zon[:, k, l] = np.sum(w * _radial_norm(k, l) * Lk[k] * yl0, axis=(1, 2))
    Uh = np.where(Um[:, None] > 0, U / np.where(Um > 0, Um, 1.0)[:, None], np.array([0.0, 0.0, 1.0]))
    Y = _real_sh_unit(lmax, Uh)  # [n, NQ]
    lq = np.array([int(math.isqrt(q)) for q in range(NQ)])
    fac = np.sqrt(4.0 * np.pi / (2 * lq + 1))
    return rho[:, None, None] * zon[:, :, lq] * (fac * Y)[:, None, :]


def two_maxwellians(kmax, lmax, ncells, seed=2, chunk=2048, pool=None):
    """f[cell, k, q] for the two-Maxwellian mixtures described in the module docstring.

    With `pool` = P, the (U, T) pairs are drawn for P cells only and every cell
    takes the pair of a uniformly drawn pool member with its own rho1 (the
    coefficients are linear in the Maxwellians, so each cell is still an exact
    projected two-Maxwellian mixture); this bounds the cost of large batches."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if pool is not None and pool < ncells:
        comp = _pool_components(kmax, lmax, pool, seed=seed + 1000003, chunk=chunk)
        idx = rng.integers(0, pool, ncells)
        rho1 = rng.uniform(0.25, 0.75, ncells)
        return rho1[:, None, None] * comp[0][idx] + (1.0 - rho1)[:, None, None] * comp[1][idx]
    rho1 = rng.uniform(0.25, 0.75, ncells)
    r = np.exp(rng.uniform(np.log(0.5), np.log(2.0), ncells))

    def ball(n):
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return d * (0.5 * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0))[:, None]

    U1, U2 = ball(ncells), ball(ncells)
    T1, T2 = r**-0.5, r**0.5
    out = np.empty((ncells, kmax + 1, _nq(lmax)))
    for s in range(0, ncells, chunk):
        e = min(ncells, s + chunk)
        out[s:e] = maxwellian_coefficients(kmax, lmax, rho1[s:e], U1[s:e], T1[s:e]) + maxwellian_coefficients(
            kmax, lmax, 1.0 - rho1[s:e], U2[s:e], T2[s:e]
        )
    return out


def _pool_components(kmax, lmax, n, seed, chunk=2048):
    """The two unit-density Maxwellian components of `two_maxwellians(..., n, seed)`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rng.uniform(0.25, 0.75, n)  # rho1 of the pool (not used)
    r = np.exp(rng.uniform(np.log(0.5), np.log(2.0), n))

    def ball(m):
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return d * (0.5 * rng.uniform(0.0, 1.0, m) ** (1.0 / 3.0))[:, None]

    U1, U2 = ball(n), ball(n)
    T1, T2 = r**-0.5, r**0.5
    ones = np.ones(n)
    a = np.empty((n, kmax + 1, _nq(lmax)))
    b = np.empty_like(a)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        a[s:e] = maxwellian_coefficients(kmax, lmax, ones[s:e], U1[s:e], T1[s:e])
        b[s:e] = maxwellian_coefficients(kmax, lmax, ones[s:e], U2[s:e], T2[s:e])
    return a, b
