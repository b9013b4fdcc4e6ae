"""Pins of the oracle's angular geometry (§4.1, §4.2, §4.6) against the paper and textbook identities."""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import basis, gaunt


@pytest.fixture(scope="module")
def G4():
    return gaunt.gaunt_dense(4)


def test_table1_rows(G4):
    """Table 1: the printed COO rows (1-based), column-major order, weights to 4 decimals."""
    q1, q2, q3, c, g = gaunt.coo(4, G4)
    assert len(g) == 1158
    assert len(gaunt.channels(4)) == 42
    for z, a, b, d, ch, gv in golden("table1_coo_L4.txt"):
        i = int(z) - 1
        assert (q1[i] + 1, q2[i] + 1, q3[i] + 1, c[i] + 1) == (int(a), int(b), int(d), int(ch))
        assert round(g[i], 4) == pytest.approx(float(gv), abs=1e-12)


def test_table6_counts():
    """Table 6: DOFs, Gaunt nonzeros and the naive dense size at Kmax = 4."""
    for L, dofs, ng, gib in golden("table6_memory.txt"):
        L = int(L)
        N = 5 * (L + 1) ** 2
        assert N == int(dofs)
        # printed with coarse rounding (0.495 -> "0.50", 22.48 -> "22.50")
        assert N**3 * 8 / 2**30 == pytest.approx(float(gib), abs=0.03)
        if L <= 12:
            assert len(gaunt.coo(L)[4]) == int(ng)


@pytest.mark.slow
def test_table6_count_L16():
    assert len(gaunt.coo(16)[4]) == 601569


def test_channel_counts():
    """N_T from the selection rules (§4.6); 106/215/616 at Lmax = 6/8/12."""
    assert [len(gaunt.channels(L)) for L in (4, 6, 8, 12)] == [42, 106, 215, 616]
    ch = gaunt.channels(4)
    assert ch[6] == (1, 1, 0) and ch[14] == (2, 1, 1) and ch[41] == (4, 4, 4)


def test_selection_rules_bruteforce(G4):
    """Every nonzero real Gaunt entry obeys the triangle, parity and azimuthal rules of §4.1
    (for real harmonics the azimuthal rule reads |m1| = ||m2| +- |m3||), and every
    zero that the rules allow is a genuine zero only if the rules forbid it."""
    NQ = G4.shape[0]
    lm = [basis.lm_of_q(q) for q in range(NQ)]
    for a in range(NQ):
        for b in range(NQ):
            for d in range(NQ):
                (l1, m1), (l2, m2), (l3, m3) = lm[a], lm[b], lm[d]
                allowed = (
                    abs(l2 - l3) <= l1 <= l2 + l3
                    and (l1 + l2 + l3) % 2 == 0
                    and abs(m1) in (abs(m2) + abs(m3), abs(abs(m2) - abs(m3)))
                )
                if G4[a, b, d] != 0.0:
                    assert allowed, (lm[a], lm[b], lm[d])


def test_y00_special_case(G4):
    """Textbook: integral of Y_00 Y_q2 Y_q3 = delta_{q2 q3} / sqrt(4 pi)."""
    assert np.allclose(G4[0], np.eye(25) / math.sqrt(4 * math.pi), atol=1e-15)


def _threej000(l1, l2, l3):
    """Closed form of the 3-j symbol (l1 l2 l3; 0 0 0) (no sum)."""
    J = l1 + l2 + l3
    if J % 2:
        return 0.0
    g = J // 2
    f = math.factorial
    val = math.sqrt(f(J - 2 * l1) * f(J - 2 * l2) * f(J - 2 * l3) / f(J + 1)) * f(g) / (f(g - l1) * f(g - l2) * f(g - l3))
    return (-1) ** g * val


def test_zonal_closed_form():
    """Zonal entries: G[(l1,0),(l2,0),(l3,0)] = sqrt((2l1+1)(2l2+1)(2l3+1)/4pi) * 3j(l1 l2 l3; 000)^2."""
    L = 6
    G = gaunt.gaunt_dense(L)
    for l1 in range(L + 1):
        for l2 in range(L + 1):
            for l3 in range(L + 1):
                if not abs(l1 - l2) <= l3 <= l1 + l2:
                    continue
                ref = math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4 * math.pi)) * _threej000(l1, l2, l3) ** 2
                got = G[l1 * l1 + l1, l2 * l2 + l2, l3 * l3 + l3]
                assert got == pytest.approx(ref, abs=1e-14)


def test_clebsch_gordan_orthogonality(G4):
    """Orthogonality of the coupled basis: for a channel (l1,l2,l3),
    sum_{m1,m2} G[q1,q2,q3] G[q1,q2,q3'] = delta_{q3 q3'} S_c / (2 l3 + 1)."""
    S = gaunt.channel_norm(4, G4)
    for c, (l1, l2, l3) in enumerate(gaunt.channels(4)):
        blk = G4[l1 * l1:(l1 + 1) ** 2, l2 * l2:(l2 + 1) ** 2, l3 * l3:(l3 + 1) ** 2]
        M = np.einsum("abc,abd->cd", blk, blk)
        assert np.allclose(M, np.eye(2 * l3 + 1) * S[c] / (2 * l3 + 1), atol=1e-14)
