"""Pins of the oracle's dense contraction (§2.3, §4.1, §4.4, §4.5)."""
import numpy as np
import pytest

import wef_inputs as wi
from oracle import basis, dense, gaunt


def _literal_discrete_sum(kmax, lmax, R, f):
    """The full discrete factored sum of §4.5 written as loops over the COO rows z
    and the radial orders, in pure Python (tiny sizes only)."""
    K, NQ = kmax + 1, (lmax + 1) ** 2
    q1, q2, q3, c, g = gaunt.coo(lmax)
    Q = np.zeros((K, NQ))
    for z in range(len(g)):
        for k1 in range(K):
            acc = 0.0
            for k2 in range(K):
                for k3 in range(K):
                    acc += R[c[z], k1, k2, k3] * f[k2, q2[z]] * f[k3, q3[z]]
            Q[k1, q1[z]] += g[z] * acc
    return Q


def test_dense_equals_literal_sum():
    km, lm = 2, 2
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=5)
    f = wi.random_cells(km, lm, 2, seed=6)
    Qd = dense.DenseOperator(km, lm, R).evaluate(f.reshape(2, -1))
    for i in range(2):
        Ql = _literal_discrete_sum(km, lm, R, f[i])
        assert np.allclose(Qd[i], Ql.reshape(-1), rtol=0, atol=1e-13)


def test_absolute_terms_brute_force():
    """T_a1 = sum |C_a1a2a3| |f_a2| |f_a3|, the cancellation scale the GPU parity tests guard
    with: against the full tensor C = R * G assembled entry by entry from the oracle's Gaunt
    tensor and summed term by term in pure Python; T >= |Q| everywhere, with equality
    exactly where every term of a row has the same sign (here: |f| and |R| make every term
    of a row share the sign of its Gaunt weights, so T = |Q| on rows whose weights agree)."""
    km, lm = 1, 2
    K, NQ = km + 1, (lm + 1) ** 2
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=15)
    f = wi.random_cells(km, lm, 2, seed=16)
    op = dense.DenseOperator(km, lm, R)
    Q, T = op.evaluate_rows_with_terms(f.reshape(2, -1))
    G = gaunt.gaunt_dense(lm)
    cidx = gaunt.channel_index(lm)
    lq = [basis.lm_of_q(q)[0] for q in range(NQ)]
    for i in range(2):
        fi = f[i]
        for k1 in range(K):
            for q1 in range(NQ):
                t = 0.0
                for k2 in range(K):
                    for q2 in range(NQ):
                        for k3 in range(K):
                            for q3 in range(NQ):
                                g = G[q1, q2, q3]
                                if g == 0.0:
                                    continue
                                c = cidx[(lq[q1], lq[q2], lq[q3])]
                                t += abs(R[c, k1, k2, k3] * g * fi[k2, q2] * fi[k3, q3])
                assert abs(T[i, k1 * NQ + q1] - t) <= 1e-14 * max(t, 1e-300)
    assert np.all(T >= np.abs(Q) * (1 - 1e-14))
    # all terms of one sign: a core and cells made non-negative, rows whose Gaunt weights
    # are all positive (the l1 = 0 rows: g = delta / sqrt(4 pi) >= 0) give T = Q
    Qp, Tp = dense.DenseOperator(km, lm, np.abs(R)).evaluate_rows_with_terms(np.abs(f).reshape(2, -1), [0, NQ])
    assert np.allclose(Qp, Tp, rtol=1e-14, atol=0)


def _rotation(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 3))
    Qm, Rm = np.linalg.qr(A)
    Qm = Qm * np.sign(np.diag(Rm))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] *= -1
    return Qm


def _wigner_real(lmax, rot):
    """Block-diagonal real Wigner matrix D with Y(rot n) = D Y(n), by exact sphere quadrature."""
    xyz, w = gaunt.sphere_rule(2 * lmax)
    Y = basis.real_sh_all(lmax, xyz)
    Yr = basis.real_sh_all(lmax, xyz @ rot.T)
    return (Yr * w[:, None]).T @ Y


@pytest.mark.parametrize("seed", [1, 2])
def test_rotation_equivariance(seed):
    """Q(D f) = D Q(f) for every rotation D, whatever the core: the Gaunt structure alone
    carries the SO(3) covariance (§3.2).  Catches wrong signs/phases in the Gaunt table."""
    km, lm = 2, 3
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=seed)
    op = dense.DenseOperator(km, lm, R)
    f = wi.random_cells(km, lm, 1, seed=10 + seed)[0]
    D = _wigner_real(lm, _rotation(seed))
    assert np.allclose(D @ D.T, np.eye(D.shape[0]), atol=1e-13)
    Qf = op.evaluate(f.reshape(1, -1))[0].reshape(km + 1, -1)
    QDf = op.evaluate((f @ D.T).reshape(1, -1))[0].reshape(km + 1, -1)
    assert np.allclose(QDf, Qf @ D.T, atol=1e-12)


def test_parity_covariance():
    """Inversion v -> -v multiplies shell l by (-1)^l and commutes with Q (even channels only)."""
    km, lm = 2, 3
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=3)
    op = dense.DenseOperator(km, lm, R)
    f = wi.random_cells(km, lm, 1, seed=4)[0]
    sgn = np.array([(-1) ** basis.lm_of_q(q)[0] for q in range((lm + 1) ** 2)])
    Qf = op.evaluate(f.reshape(1, -1))[0].reshape(km + 1, -1)
    Qp = op.evaluate((f * sgn).reshape(1, -1))[0].reshape(km + 1, -1)
    assert np.allclose(Qp, Qf * sgn, atol=1e-13)


def test_conservation_zeroing_exact():
    """§4.4: after the null-space and detailed-balance zeroing, the mass, momentum and energy
    outputs are exactly 0 for any input, and Q(M, M) = 0 for the reference Maxwellian."""
    km, lm = 3, 3
    NQ = (lm + 1) ** 2
    R = dense.conservation_zeroing(wi.random_core(len(gaunt.channels(lm)), km, seed=8), lm)
    op = dense.DenseOperator(km, lm, R)
    f = wi.random_cells(km, lm, 3, seed=9).reshape(3, -1)
    Q = op.evaluate(f)
    for a in (0, 1, 2, 3, NQ):  # (k=0,l=0), (k=0,l=1,m=-1..1), (k=1,l=0)
        assert np.all(Q[:, a] == 0.0)
    e0 = np.zeros((1, op.N))
    e0[0, 0] = 1.0
    assert np.all(op.evaluate(e0) == 0.0)


def test_bilinear_symmetric_part_only():
    """Q(f,f) sees only the part of C symmetric in (a2, a3): transposing every R^(c)
    in (k2, k3) and swapping channels (l1,l2,l3) <-> (l1,l3,l2) leaves Q unchanged."""
    km, lm = 2, 3
    ch = gaunt.channels(lm)
    idx = gaunt.channel_index(lm)
    R = wi.random_core(len(ch), km, seed=11)
    Rs = np.stack([R[idx[(l1, l3, l2)]].transpose(0, 2, 1) for (l1, l2, l3) in ch])
    f = wi.random_cells(km, lm, 2, seed=12).reshape(2, -1)
    Q1 = dense.DenseOperator(km, lm, R).evaluate(f)
    Q2 = dense.DenseOperator(km, lm, Rs).evaluate(f)
    assert np.allclose(Q1, Q2, atol=1e-13)


@pytest.mark.parametrize("km,lm,ncells", [(0, 0, 3), (2, 3, 7), (3, 4, 5)])
def test_angular_first_equals_dense(km, lm, ncells):
    """The factorised angular-first evaluation (§4.5.4) and the dense form (§4.5.1) are the
    same bilinear form: equal to rounding on a random core and random cells."""
    from oracle import angular_first

    rng = np.random.default_rng(km * 10 + lm)
    R = rng.standard_normal((len(gaunt.channels(lm)), km + 1, km + 1, km + 1))
    f = rng.standard_normal((ncells, km + 1, (lm + 1) ** 2))
    Qa = angular_first.evaluate(km, lm, R, f)
    Qd = dense.evaluate(km, lm, R, f.reshape(ncells, -1)).reshape(f.shape)
    assert np.max(np.abs(Qa - Qd)) <= 1e-12 * max(np.max(np.abs(Qd)), 1.0)
