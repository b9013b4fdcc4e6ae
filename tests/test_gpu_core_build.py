"""The GPU core builder (same quadrature as the host builder, Sec. 4.3 / Appendix A-B)
against the host builder and the oracle's literal 5D quadrature."""
import math

import numpy as np
import pytest

from oracle import core as ocore
from oracle import gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("km,lm,gamma,pads", [(0, 0, 0.0, (20, 20)), (2, 3, 0.0, (20, 20)), (3, 4, 1.0, (5, 7)),
                                              (4, 2, 0.5, (20, 20)), (1, 6, 1.0, (0, 0))])
def test_device_core_equals_host_core(km, lm, gamma, pads):
    op = W.Operator(km, lm, gamma)
    Rh = op.build_core(*pads)
    Rd = op.build_core(*pads, device=True)
    # entries are O(1); at Kmax = Lmax = 0 the only entry is the mass balance, zero up to rounding
    assert np.max(np.abs(Rd - Rh)) <= 1e-12 * max(np.max(np.abs(Rh)), 1.0)


def test_device_core_equals_oracle_core():
    km, lm = 2, 2
    op = W.Operator(km, lm, 1.0)
    Rd = op.build_core(device=True)
    Ro = ocore.core(km, lm, 1.0)
    assert np.max(np.abs(Rd - Ro)) <= 1e-12 * np.max(np.abs(Ro))


def test_device_core_wcu_eigenvalues():
    """Maxwell molecules: the (l, 0, l) and (l, l, 0) channels give the closed-form WCU
    eigenvalues on the diagonal of the linearized blocks (Sec. 5.2.2)."""
    from scipy import special

    km, lm = 3, 4
    op = W.Operator(km, lm, 0.0)
    R = op.build_core(device=True)
    chans = gaunt.channels(lm)
    g0 = 1.0 / math.sqrt(4 * math.pi)
    x, w = np.polynomial.legendre.leggauss(60)
    cc, ss = np.sqrt((1 + x) / 2), np.sqrt((1 - x) / 2)
    for l in range(lm + 1):
        B = (R[chans.index((l, 0, l))][:, 0, :] + R[chans.index((l, l, 0))][:, :, 0]) * g0
        for k in range(km + 1):
            if (l == 0 and k < 2) or (l == 1 and k == 0):
                continue
            n = 2 * k + l
            lam = 0.5 * np.sum(w * (cc**n * special.eval_legendre(l, cc) + ss**n * special.eval_legendre(l, ss) - 1.0
                                    - (1.0 if k == l == 0 else 0.0)))
            assert B[k, k] == pytest.approx(lam, abs=1e-12)
