"""Angular geometry of the oracle: channels and the real Gaunt tensor (§4.1, §4.2).

The real Gaunt tensor is computed here by numerical integration of three real
spherical harmonics over the unit sphere, with a product rule (Gauss-Legendre
in cos(theta) x trapezoid in phi) that is exact for the degree-3*Lmax
trigonometric polynomials involved.  This is a different method from the
closed-form Wigner 3-j route of §3.2/§4.1, so it checks that route.

Reading (§3.2 writes G = 8 pi^2 x 3j, but Table 1 prints values of the real
Gaunt integral): the COO weight is g = integral of Y_q1 Y_q2 Y_q3 over the
sphere, and the core R carries the rest of the normalisation.
"""
import numpy as np
from scipy import special

from . import basis


def channels(lmax):
    """Valid (l1, l2, l3) triplets in the enumeration order of §4.6:
    l1 outermost, then l2, then l3 ascending; triangle rule, even l1+l2+l3,
    l3 <= Lmax (§4.1 selection rules)."""
    out = []
    for l1 in range(lmax + 1):
        for l2 in range(lmax + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                if (l1 + l2 + l3) % 2 == 0:
                    out.append((l1, l2, l3))
    return out


def channel_index(lmax):
    """Map (l1, l2, l3) -> 0-based channel index c (the paper's c - 1)."""
    return {t: i for i, t in enumerate(channels(lmax))}


def sphere_rule(degree):
    """Nodes (unit vectors) and weights exact for polynomials of total degree
    `degree` on S^2: Gauss-Legendre in cos(theta) times the trapezoid rule in phi."""
    nt = degree // 2 + 1
    nphi = degree + 1
    ct, wt = special.roots_legendre(nt)
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1.0 - ct * ct)
    xyz = np.stack(
        [np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)), np.outer(ct, np.ones(nphi))], axis=-1
    ).reshape(-1, 3)
    w = np.outer(wt, np.full(nphi, 2.0 * np.pi / nphi)).reshape(-1)
    return xyz, w


def gaunt_dense(lmax, tol=1e-13):
    """G[q1, q2, q3] = integral over S^2 of Y_q1 Y_q2 Y_q3 (real SH of basis.py).

    Entries below `tol` in magnitude are exact zeros of the selection rules
    (§4.1) polluted by rounding; they are set to 0."""
    xyz, w = sphere_rule(3 * lmax)
    Y = basis.real_sh_all(lmax, xyz)  # [P, NQ]
    nq = Y.shape[1]
    Yw = Y * w[:, None]
    G = np.empty((nq, nq, nq))
    for q1 in range(nq):
        G[q1] = (Yw * Y[:, q1][:, None]).T @ Y
    G[np.abs(G) < tol] = 0.0
    return G


def coo(lmax, G=None):
    """COO table of the nonzero real Gaunt entries in the order of Table 1:
    column-major over (q1, q2, q3), i.e. q3 slowest and q1 fastest.

    Returns (q1, q2, q3, c, g) as arrays, all indices 0-based."""
    if G is None:
        G = gaunt_dense(lmax)
    cidx = channel_index(lmax)
    lq = np.array([basis.lm_of_q(q)[0] for q in range(G.shape[0])])
    nz = np.nonzero(G.transpose(2, 1, 0))  # iterate q3, q2, q1 with q1 fastest
    q3, q2, q1 = nz
    g = G[q1, q2, q3]
    c = np.array([cidx[(lq[a], lq[b], lq[d])] for a, b, d in zip(q1, q2, q3)], dtype=np.int64)
    return q1.astype(np.int64), q2.astype(np.int64), q3.astype(np.int64), c, g


def channel_norm(lmax, G=None):
    """S_c = sum over all m-triples of G^2 for each channel (the squared norm of
    the invariant tensor of the channel); used to normalise the core."""
    if G is None:
        G = gaunt_dense(lmax)
    cidx = channel_index(lmax)
    S = np.zeros(len(cidx))
    q1, q2, q3, c, g = coo(lmax, G)
    np.add.at(S, c, g * g)
    return S
