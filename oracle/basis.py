"""Galerkin basis of the oracle: phi_{klm}(v) = R_kl(|v|) Y_lm(v_hat)  (§2.2).

Conventions (readings where the paper is silent):

* Radial functions.  R_kl(v) = N_kl v^l L_k^{(l+1/2)}(v^2/2) with
  N_kl^2 = 2^{1-l} pi^{3/2} k! / Gamma(k+l+3/2).  This is the normalisation
  that makes the basis orthonormal under the reference Maxwellian
  M(v) = (2 pi)^{-3/2} exp(-v^2/2), i.e. the identity mass matrix of §2.3.
  It gives phi_000 = 1.
* Real spherical harmonics (§4.1 maps the complex basis to the real one).
  Y_l0 = n_l0 P_l(cos t); Y_lm = sqrt2 n_lm P_l^m(cos t) cos(m p) for m > 0;
  Y_lm = sqrt2 n_l|m| P_l^|m|(cos t) sin(|m| p) for m < 0, where P_l^m carries
  no Condon-Shortley phase and n_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!.
  Angular index q = l^2 + l + m (0-based), i.e. the paper's q - 1.
"""
import numpy as np
from scipy import special


def radial_norm(k, l):
    """N_kl from the orthonormality of §2.3 (identity mass matrix)."""
    logn2 = (1 - l) * np.log(2.0) + 1.5 * np.log(np.pi) + special.gammaln(k + 1) - special.gammaln(k + l + 1.5)
    return np.exp(0.5 * logn2)


def radial(k, l, v):
    """R_kl(v) = N_kl v^l L_k^{(l+1/2)}(v^2/2)."""
    v = np.asarray(v, dtype=np.float64)
    return radial_norm(k, l) * v**l * special.eval_genlaguerre(k, l + 0.5, 0.5 * v * v)


def q_index(l, m):
    """0-based angular index q = l^2 + l + m (§4.1)."""
    return l * l + l + m


def lm_of_q(q):
    l = int(np.floor(np.sqrt(q + 0.5)))
    return l, q - l * l - l


def real_sh(l, m, xyz):
    """Real spherical harmonic Y_lm at unit vectors xyz[..., 3]."""
    xyz = np.asarray(xyz, dtype=np.float64)
    ct = np.clip(xyz[..., 2], -1.0, 1.0)
    ph = np.arctan2(xyz[..., 1], xyz[..., 0])
    am = abs(m)
    lognorm = 0.5 * (np.log(2 * l + 1) - np.log(4 * np.pi) + special.gammaln(l - am + 1) - special.gammaln(l + am + 1))
    # scipy's lpmv includes the Condon-Shortley phase (-1)^m; remove it.
    plm = (-1.0) ** am * special.lpmv(am, l, ct)
    base = np.exp(lognorm) * plm
    if m == 0:
        return base
    if m > 0:
        return np.sqrt(2.0) * base * np.cos(am * ph)
    return np.sqrt(2.0) * base * np.sin(am * ph)


def real_sh_all(L, xyz):
    """All Y_q, q = 0..(L+1)^2-1, stacked on a new last axis.

    Same functions as `real_sh`, evaluated together by the standard upward
    recurrences for associated Legendre functions (no Condon-Shortley phase):
    P_m^m = (2m-1)!! s^m, P_{m+1}^m = (2m+1) x P_m^m,
    (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m."""
    xyz = np.asarray(xyz, dtype=np.float64)
    x = np.clip(xyz[..., 2], -1.0, 1.0)
    s = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
    ph = np.arctan2(xyz[..., 1], xyz[..., 0])
    out = np.empty(((L + 1) ** 2,) + xyz.shape[:-1])  # q first: contiguous writes
    pmm = np.ones_like(x)
    for m in range(L + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
            cm, sm = np.sqrt(2.0) * np.cos(m * ph), np.sqrt(2.0) * np.sin(m * ph)
        plm2, plm1 = None, pmm
        for l in range(m, L + 1):
            if l == m:
                p = pmm
            elif l == m + 1:
                p = (2 * m + 1) * x * pmm
            else:
                p = ((2 * l - 1) * x * plm1 - (l + m - 1) * plm2) / (l - m)
            if l > m:
                plm2, plm1 = plm1, p
            norm = np.exp(0.5 * (np.log(2 * l + 1) - np.log(4 * np.pi) + special.gammaln(l - m + 1) - special.gammaln(l + m + 1)))
            if m == 0:
                out[l * l + l] = norm * p
            else:
                np_ = norm * p
                out[l * l + l + m] = np_ * cm
                out[l * l + l - m] = np_ * sm
    return np.moveaxis(out, 0, -1)


def radial_all(K, L, v):
    """R_kl(v) for k = 0..K-1, l = 0..L stacked as [..., K, L+1].

    Same functions as `radial`, evaluated by the three-term recurrence
    (k+1) L_{k+1}^a = (2k+1+a-x) L_k^a - (k+a) L_{k-1}^a with a = l + 1/2, x = v^2/2."""
    v = np.asarray(v, dtype=np.float64)
    x = 0.5 * v * v
    out = np.empty((K, L + 1) + v.shape)  # (k, l) first: contiguous writes
    for l in range(L + 1):
        a = l + 0.5
        vl = v**l
        lkm1 = np.ones_like(v)
        lk = 1.0 + a - x
        for k in range(K):
            if k == 0:
                cur = lkm1
            elif k == 1:
                cur = lk
            else:
                cur = ((2 * k - 1 + a - x) * lk - (k - 1 + a) * lkm1) / k
                lkm1, lk = lk, cur
            out[k, l] = radial_norm(k, l) * vl * cur
    return np.moveaxis(out, (0, 1), (-2, -1))
