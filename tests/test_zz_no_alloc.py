"""wef_evaluate_noalloc: the FP64 evaluation for callers that cannot allocate device memory
when they evaluate (their device memory is owned by their own pool, or they run where
cudaMalloc's implicit synchronisation is not allowed).  It uses a fixed scratch array kept
by the library instead of a caller workspace.

Checked through the C ABI against wef_evaluate on two calls in a row (the scratch keeps the
previous call's contents), on a batch smaller than one 32-cell tile and at the size limit
(928 cells at Kmax = Lmax = 12 accepted, 929 rejected); after a first call, further calls
leave the device's free memory unchanged.  This file is collected last on purpose."""
import numpy as np
import pytest

import wef_inputs as wi
from oracle import gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not __import__("os").path.exists(W.LIB_PATH):
        from paper_2605_28475_gb300 import build

        build.build()


def _rel(a, b):
    return float((a - b).abs().max() / max(float(b.abs().max()), 1e-300))


@pytest.mark.parametrize("km,lm,ncells", [(4, 4, 77), (4, 4, 5), (12, 12, 600), (12, 12, 928)])
def test_noalloc_matches_evaluate_twice(km, lm, ncells):
    op = W.Operator(km, lm, 1.0)
    op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=21))
    stream = torch.cuda.current_stream()
    for call in range(2):
        f = torch.from_numpy(wi.random_cells(km, lm, ncells, seed=30 + call)).cuda()
        q_ref = op.evaluate(f, precision="fp64")
        q = torch.full_like(f, float("nan"))
        W.wef_evaluate_noalloc(op.h, f.data_ptr(), q.data_ptr(), ncells, stream.cuda_stream)
        torch.cuda.synchronize()
        assert not torch.isnan(q).any()
        assert _rel(q, q_ref) <= FP64_TOL
    op.close()


def test_noalloc_rejects_too_many_cells():
    km = lm = 12
    op = W.Operator(km, lm, 1.0)
    op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=22))
    for n in (929, 1000):
        f = torch.zeros(n, km + 1, (lm + 1) ** 2, dtype=torch.float64, device="cuda")
        q = torch.empty_like(f)
        with pytest.raises(W.WefError) as e:
            W.wef_evaluate_noalloc(op.h, f.data_ptr(), q.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
        assert e.value.status == W.WEF_EINVAL and "928" in str(e.value)
    op.close()


def test_noalloc_allocates_nothing_after_first_call():
    km = lm = 8
    op = W.Operator(km, lm, 1.0)
    op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=23))
    f = torch.from_numpy(wi.random_cells(km, lm, 300, seed=24)).cuda()
    q = torch.empty_like(f)
    st = torch.cuda.current_stream().cuda_stream
    W.wef_evaluate_noalloc(op.h, f.data_ptr(), q.data_ptr(), 300, st)  # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        W.wef_evaluate_noalloc(op.h, f.data_ptr(), q.data_ptr(), 300, st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    op.close()
