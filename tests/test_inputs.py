"""The seeded input generators: the exact projection of a drifting Maxwellian onto the basis
(the two-Maxwellian cells of the benchmark workloads) against a direct 3D evaluation.

c_a = integral of rho M_{U,T}(v) phi_a(v) dv, phi_a = R_kl(|v|) Y_lm(v/|v|) a polynomial of
degree 2k + l, so a Gauss-Hermite product rule centred at U with scale sqrt(T) and enough
points per axis is exact; the generator instead projects along the drift axis (zonal
Gauss-Hermite x Gauss-Laguerre rule) and rotates by the addition theorem."""
import math

import numpy as np
import pytest

import wef_inputs as wi
from oracle import basis


def _direct(kmax, lmax, rho, U, T):
    K, NQ = kmax + 1, (lmax + 1) ** 2
    lq = np.array([basis.lm_of_q(q)[0] for q in range(NQ)])
    n = (2 * kmax + lmax) // 2 + 2
    x, w = np.polynomial.hermite_e.hermegauss(n)
    w = w / math.sqrt(2 * math.pi)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    Wt = np.einsum("i,j,k->ijk", w, w, w).reshape(-1)
    v = np.asarray(U)[None, :] + math.sqrt(T) * X
    r = np.linalg.norm(v, axis=1)
    Y = basis.real_sh_all(lmax, v / np.maximum(r, 1e-300)[:, None])  # [P, NQ]
    Rr = basis.radial_all(K, lmax, r)[:, :, lq]  # [P, K, NQ]
    return rho * np.einsum("p,pkq->kq", Wt, Rr * Y[:, None, :])


@pytest.mark.parametrize("U,T", [((0.0, 0.0, 0.0), 1.0), ((0.0, 0.0, 0.4), 0.7), ((0.3, -0.2, 0.1), 1.6),
                                 ((-0.45, 0.1, -0.2), 0.5)])
def test_maxwellian_projection_matches_direct_3d(U, T):
    kmax, lmax, rho = 3, 4, 0.37
    c = wi.maxwellian_coefficients(kmax, lmax, np.array([rho]), np.array([U]), np.array([T]))[0]
    ref = _direct(kmax, lmax, rho, U, T)
    assert np.max(np.abs(c - ref)) < 1e-13


def test_maxwellian_projection_moments():
    """Mass, momentum and energy of the projection in closed form: c_000 = rho, the l = 1
    components carry rho U, and c_100 = rho N_10 (3/2 - (3T + |U|^2)/2)."""
    kmax, lmax, rho, U, T = 2, 2, 0.6, np.array([0.2, -0.3, 0.25]), 1.3
    c = wi.maxwellian_coefficients(kmax, lmax, np.array([rho]), U[None, :], np.array([T]))[0]
    assert c[0, 0] == pytest.approx(rho, abs=1e-14)
    # R_01 Y_1m = N_01 v Y_1m(v_hat) = N_01 sqrt(3 / 4 pi) v_(y,z,x) for m = -1, 0, 1
    n01 = basis.radial_norm(0, 1) * math.sqrt(3.0 / (4 * math.pi))
    assert np.allclose(c[0, 1:4], rho * n01 * U[[1, 2, 0]], rtol=0, atol=1e-14)
    n10 = basis.radial_norm(1, 0) / math.sqrt(4 * math.pi)
    assert c[1, 0] == pytest.approx(rho * n10 * (1.5 - (3 * T + U @ U) / 2), abs=1e-14)


def test_two_maxwellian_cells_are_seeded_mixtures():
    """Same seed, same cells; every cell has unit density (rho1 + rho2 = 1)."""
    a = wi.two_maxwellians(2, 3, 17, seed=5, pool=8)
    b = wi.two_maxwellians(2, 3, 17, seed=5, pool=8)
    assert np.array_equal(a, b)
    assert np.allclose(a[:, 0, 0], 1.0, rtol=0, atol=1e-14)
    assert not np.array_equal(a, wi.two_maxwellians(2, 3, 17, seed=6, pool=8))
