"""Evaluation from host memory (chunked, copies overlapping the evaluations) gives the same
Q as the device-resident evaluation, bit for bit, for every chunking."""
import numpy as np
import pytest

import wef_inputs as wi
from oracle import gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec", ["rf32", "fp64", "tf32"])
@pytest.mark.parametrize("chunk", [1, 37, 64, 1000])
def test_host_evaluation_equals_device(prec, chunk):
    km, lm, n = 3, 4, 150
    op = W.Operator(km, lm, 1.0)
    op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=21))
    f = torch.from_numpy(wi.random_cells(km, lm, n, seed=22))
    qd = op.evaluate(f.cuda(), precision=prec)
    fp = f.pin_memory()
    qh = op.evaluate_host(fp, precision=prec, chunk_cells=chunk)
    torch.cuda.synchronize()
    assert torch.equal(qh, qd.cpu())


def test_host_evaluation_pageable_and_errors():
    km, lm, n = 2, 2, 40
    op = W.Operator(km, lm, 0.0)
    op.upload_core(op.build_core())
    f = torch.from_numpy(wi.random_cells(km, lm, n, seed=3))  # pageable memory: still correct
    qh = op.evaluate_host(f, precision="fp64", chunk_cells=16)
    torch.cuda.synchronize()
    assert torch.equal(qh, op.evaluate(f.cuda()).cpu())
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(W.WefError):  # workspace too small
        W.wef_evaluate_host(op.h, f.data_ptr(), qh.data_ptr(), n, 16, 0, ws.data_ptr(), ws.numel(), st)
    with pytest.raises(W.WefError):  # chunk of zero cells
        W.wef_evaluate_host(op.h, f.data_ptr(), qh.data_ptr(), n, 0, 0, ws.data_ptr(), ws.numel(), st)
    W.wef_evaluate_host(op.h, 0, 0, 0, 16, 0, 0, 0, st)  # empty batch: nothing to do
    assert np.isfinite(qh.numpy()).all()


@pytest.mark.parametrize("prec", ["rf32", "fp64", "tf32"])
def test_evaluation_captured_in_a_cuda_graph(prec):
    """wef_evaluate launches only stream-ordered work (no allocation, no synchronisation), so
    a caller can capture it in a CUDA graph: replays give the direct call's Q bit for bit."""
    km, lm, n = 4, 5, 70
    op = W.Operator(km, lm, 1.0)
    op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=31))
    f = torch.from_numpy(wi.random_cells(km, lm, n, seed=32)).cuda()
    q_direct = op.evaluate(f, precision=prec).clone()
    q = torch.empty_like(f)
    p = W.PRECISIONS[prec]
    ws = torch.empty(W.wef_workspace_size(op.h, n, p), dtype=torch.uint8, device="cuda")
    W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), n, p, ws.data_ptr(), ws.numel(),
                   torch.cuda.current_stream().cuda_stream)  # first call outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), n, p, ws.data_ptr(), ws.numel(),
                       torch.cuda.current_stream().cuda_stream)
    q.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(q, q_direct)
