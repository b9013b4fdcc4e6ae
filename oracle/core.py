"""The reduced kinematic core R^{(c)}_{k1 k2 k3} by 5D singular quadrature.

Follows §3.2-3.3 (reduction to five intrinsic variables and the gain/loss
filters), §4.3 (rotated speeds, 2D Duffy split, tensor-product rules, Table 2
point counts plus padding) and Appendix A (scattering angles innermost, loss
subtracted inside the scattering integral) in that order.  Plain numpy; the
scattering sphere is integrated by an explicit (cos chi, epsilon) rule.

Definition evaluated (real-basis form of the §3.2/§3.3 formulas):

    R^{(c)}_{k1k2k3} = (8 pi^2 / S_c) * int_{5D} B(u, cos chi) R_{k2 l2}(v) R_{k3 l3}(w)
        [ R_{k1 l1}(|v'|) P_gain^c(v'_hat, w_hat) - R_{k1 l1}(v) P_loss^c(w_hat) ]
        M(v) M(w) v^2 w^2 sin(beta) sin(chi) dv dw dbeta dchi deps

with P_gain^c = sum_{m1,m3} G[(l1 m1),(l2 0),(l3 m3)] Y_{l1 m1}(v'_hat) Y_{l2 0}(z_hat) Y_{l3 m3}(w_hat),
P_loss^c the same with v'_hat -> z_hat, and S_c = sum_m G^2 over the channel
(the squared norm of the channel's invariant tensor).  The SO(3) integral of
three Wigner matrices gives 8 pi^2 times the projector onto that invariant.

Readings (where the paper is silent or inconsistent):
* collision kernel B = u^gamma / (4 pi)  (isotropic; gamma=0 Maxwell, 1 hard spheres);
* z = t^2 / 2 with t = (v + w)/sqrt2, so that M(v)M(w) = (2pi)^-3 e^{-z} e^{-z x^2} and the
  generalized Gauss-Laguerre weight z^{gamma/2} e^{-z} of §4.3.3 / Appendix A
  absorbs both the Maxwellian and the z-part of u^gamma;  u = 2 sqrt(z) sqrt(x^2 + (1-x^2) y^2);
* Jacobian re-derived: dv dw = dz dx, v^2 w^2 = z^2 (1-x^2)^2, sin(beta) dbeta = 4 y dy,
  Duffy factors x (patch 1) and y (patch 2);
* the v < w half-plane is integrated by the mirrored map x -> -x with the same patches;
* padding N_rad_pad = N_ang_pad = 20 by default (the paper's range is 10-20).
"""
import math

import numpy as np
from scipy import special

from . import basis, gaunt


def point_counts(kmax, lmax, pad_rad=20, pad_ang=20):
    """Table 2 minimum point counts (Appendix B) plus the selective padding."""
    return dict(
        z=math.ceil((3 * kmax + 1.5 * lmax + 3) / 2) + pad_rad,
        x1=4 * kmax + 3 * lmax + 4 + pad_rad,
        h1=kmax + math.ceil(1.5 * lmax) + 1 + pad_ang,
        y2=4 * kmax + 3 * lmax + 4 + pad_ang,
        h2=3 * kmax + math.floor(1.5 * lmax) + 3 + pad_rad,
        chi=kmax + math.ceil(0.5 * lmax) + 1,
        eps=2 * kmax + lmax + 1,
    )


def _gl01(n):
    x, w = special.roots_legendre(n)
    return 0.5 * (x + 1.0), 0.5 * w


def outer_points(kmax, lmax, gamma, pad_rad=20, pad_ang=20):
    """All (z, x, y) nodes of both Duffy patches and both half-planes with the
    weight of everything except the channel normalisation and the integrand
    proper: returns z, x (signed), y, W."""
    n = point_counts(kmax, lmax, pad_rad, pad_ang)
    zz, wz = special.roots_genlaguerre(n["z"], 0.5 * gamma)
    pts = []
    # Patch 1 (x > y): y = x h.
    xa, wxa = _gl01(n["x1"])
    ha, wha = _gl01(n["h1"])
    X, H = np.meshgrid(xa, ha, indexing="ij")
    WX = np.outer(wxa, wha) * X  # Duffy Jacobian x
    Y = X * H
    sing = X**gamma * (1.0 + (1.0 - X * X) * H * H) ** (0.5 * gamma)
    pts.append((X.ravel(), Y.ravel(), (WX * sing).ravel()))
    # Patch 2 (y > x): x = y h.
    ya, wya = _gl01(n["y2"])
    hb, whb = _gl01(n["h2"])
    Yb, Hb = np.meshgrid(ya, hb, indexing="ij")
    WY = np.outer(wya, whb) * Yb  # Duffy Jacobian y
    Xb = Yb * Hb
    singb = Yb**gamma * (1.0 + (1.0 - Yb * Yb) * Hb * Hb) ** (0.5 * gamma)
    pts.append((Xb.ravel(), Yb.ravel(), (WY * singb).ravel()))
    xs = np.concatenate([p[0] for p in pts])
    ys = np.concatenate([p[1] for p in pts])
    ws = np.concatenate([p[2] for p in pts])
    # both half-planes: x >= 0 (v > w) and the mirror x -> -x (v < w)
    xs = np.concatenate([xs, -xs])
    ys = np.concatenate([ys, ys])
    ws = np.concatenate([ws, ws])
    Z = np.repeat(zz, xs.size)
    WZ = np.repeat(wz, xs.size)
    X = np.tile(xs, zz.size)
    Yy = np.tile(ys, zz.size)
    Wxy = np.tile(ws, zz.size)
    # remaining scalar factors: 2^gamma (from u^gamma), residual Gaussian e^{-z x^2},
    # v^2 w^2 = z^2 (1-x^2)^2, sin(beta) dbeta = 4 y dy, M(v)M(w) prefactor (2 pi)^-3.
    W = WZ * Wxy * 2.0**gamma * np.exp(-Z * X * X) * Z**2 * (1.0 - X * X) ** 2 * 4.0 * Yy * (2.0 * np.pi) ** -3
    return Z, X, Yy, W, n


def core(kmax, lmax, gamma, pad_rad=20, pad_ang=20, chans=None, chunk=256):
    """R[c, k1, k2, k3] for the channels `chans` (default: all, in §4.6 order)."""
    K = kmax + 1
    NQ = (lmax + 1) ** 2
    all_ch = gaunt.channels(lmax)
    chans = all_ch if chans is None else list(chans)
    G = gaunt.gaunt_dense(lmax)
    S = gaunt.channel_norm(lmax, G)
    cidx = gaunt.channel_index(lmax)
    lq = np.array([basis.lm_of_q(q)[0] for q in range(NQ)])
    Z, X, Yv, W, n = outer_points(kmax, lmax, gamma, pad_rad, pad_ang)
    # scattering sphere around u_hat: Gauss-Legendre in cos(chi), trapezoid in eps
    cchi, wchi = special.roots_legendre(n["chi"])
    eps = 2.0 * np.pi * np.arange(n["eps"]) / n["eps"]
    weps = np.full(n["eps"], 2.0 * np.pi / n["eps"])
    CC, EE = np.meshgrid(cchi, eps, indexing="ij")
    SC = np.sqrt(1.0 - CC * CC)
    ws = (np.outer(wchi, weps) / (4.0 * np.pi)).ravel()  # b(cos chi) = 1/(4 pi)
    cchi_s, schi_s, ce_s, se_s = CC.ravel(), SC.ravel(), np.cos(EE).ravel(), np.sin(EE).ravel()
    zhat = np.array([0.0, 0.0, 1.0])
    Yz = basis.real_sh_all(lmax, zhat)  # Y_q(z_hat)
    out = np.zeros((len(chans), K, K, K))
    for s0 in range(0, Z.size, chunk):
        z, x, y, w = Z[s0:s0 + chunk], X[s0:s0 + chunk], Yv[s0:s0 + chunk], W[s0:s0 + chunk]
        P = z.size
        v = np.sqrt(z) * (1.0 + x)
        wm = np.sqrt(z) * (1.0 - x)
        cb = 1.0 - 2.0 * y * y
        sb = 2.0 * y * np.sqrt(np.clip(1.0 - y * y, 0.0, None))
        vvec = np.stack([np.zeros(P), np.zeros(P), v], axis=1)
        wvec = np.stack([wm * sb, np.zeros(P), wm * cb], axis=1)
        uvec = vvec - wvec
        u = np.linalg.norm(uvec, axis=1)
        uh = uvec / u[:, None]
        e2 = np.array([0.0, 1.0, 0.0])
        e1 = np.cross(np.broadcast_to(e2, uh.shape), uh)
        Vc = 0.5 * (vvec + wvec)
        # post-collision velocity v' = V + (u/2) u'_hat for every sphere node
        up = (cchi_s[None, :, None] * uh[:, None, :]
              + schi_s[None, :, None] * (ce_s[None, :, None] * e1[:, None, :] + se_s[None, :, None] * e2[None, None, :]))
        vp = Vc[:, None, :] + 0.5 * u[:, None, None] * up
        vpn = np.linalg.norm(vp, axis=2)
        vph = vp / vpn[..., None]
        Ygain = basis.real_sh_all(lmax, vph)  # [P, S, NQ]
        Rgain = basis.radial_all(K, lmax, vpn)  # [P, S, K, L+1]
        # azimuthally / polar integrated gain filter pieces, T[p, k1, q1]
        T = np.empty((P, K, NQ))
        for l in range(lmax + 1):
            sh = slice(l * l, (l + 1) ** 2)
            T[:, :, sh] = np.matmul(np.swapaxes(Rgain[:, :, :, l] * ws[None, :, None], 1, 2), Ygain[:, :, sh])
        Rv = basis.radial_all(K, lmax, v)  # [P, K, L+1]
        Rw = basis.radial_all(K, lmax, wm)
        Yw = basis.real_sh_all(lmax, wvec / np.maximum(wm, 1e-300)[:, None])  # [P, NQ]
        # loss term integrated over the same scattering rule: sum_s w_s b = 1
        lossw = ws.sum()
        for ci, (l1, l2, l3) in enumerate(chans):
            sh1 = slice(l1 * l1, (l1 + 1) ** 2)
            sh3 = slice(l3 * l3, (l3 + 1) ** 2)
            q20 = l2 * l2 + l2
            Gs = G[sh1, q20, sh3] * Yz[q20]  # [n1, n3]
            gain = T[:, :, sh1]
            loss = lossw * Rv[:, :, l1][:, :, None] * Yz[sh1][None, None, :]
            A = np.einsum("pkm,mn,pn->pk", gain - loss, Gs, Yw[:, sh3])
            out[ci] += np.einsum("p,pk,pa,pb->kab", w, A, Rv[:, :, l2], Rw[:, :, l3], optimize=True)
    for ci, ch in enumerate(chans):
        out[ci] *= 8.0 * np.pi**2 / S[cidx[ch]]
    return out
