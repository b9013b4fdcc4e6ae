"""Continuous batching: every request's result, delivered to host memory, is the same alone
and in the mix (batches of one shape on the tensor-core paths, ragged batches mixing shapes
on the radial-first and FP64 paths); memory admission defers and rejects as it should."""
import numpy as np
import pytest

import wef_inputs as wi
from oracle import gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402
from paper_2605_28475_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not __import__("os").path.exists(W.LIB_PATH):
        from paper_2605_28475_gb300 import build

        build.build()


@pytest.mark.parametrize("prec", ["tf32", "fp64", "rf32"])
def test_alone_equals_in_mix(prec):
    shapes = [(4, 4), (6, 6), (8, 8)]
    ops = {}
    for i, (km, lm) in enumerate(shapes):
        op = W.Operator(km, lm, 1.0)
        op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=40 + i))
        ops[(km, lm)] = op
    reqs = serve.poisson_requests(400.0, 0.15, shapes, 200, seed=9,
                                  make_cells=lambda sh, n, s: wi.random_cells(sh[0], sh[1], n, seed=s))
    assert len(reqs) > 20
    # a burst at t = 0 is always batched (three requests of each shape wait together);
    # the Poisson stream then arrives while batches are on the GPU
    burst = [serve.Request(0.0, 1000 + i, shapes[i % 3], wi.random_cells(*shapes[i % 3], 20, seed=500 + i))
             for i in range(9)]
    reqs = sorted(burst + reqs)
    # a small arena forces some requests to wait for memory
    srv = serve.Server(ops, arena_bytes=16 << 20, nslots=3, precision=prec, keep_results=True, max_batch_cells=500)
    res = serve.run(srv, reqs)
    assert res["completed"] == len(reqs) and res["rejected"] == 0
    assert res["batches"] < len(reqs)  # requests were batched together
    if prec in ("rf32", "fp64"):  # one ragged batch mixes shapes
        assert srv.ragged
    for r in srv.completed:
        alone = ops[r.shape].evaluate(torch.from_numpy(r.f).cuda(), precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(r.q, alone.cpu()), r.rid


def test_rejects_what_never_fits():
    op = W.Operator(4, 4, 1.0)
    op.upload_core(wi.random_core(len(gaunt.channels(4)), 4, seed=1))
    srv = serve.Server({(4, 4): op}, arena_bytes=1 << 20, nslots=2, precision="fp64")
    big = serve.Request(0.0, 0, (4, 4), wi.random_cells(4, 4, 2000, seed=2))
    small = serve.Request(0.0, 1, (4, 4), wi.random_cells(4, 4, 10, seed=3))
    res = serve.run(srv, [big, small])
    assert res["rejected"] == 1 and res["completed"] == 1 and srv.completed[0].rid == 1


def test_pinned_requests_mixed_shapes():
    """Requests set up with pin_requests (pinned inputs and outputs, no page-locking while
    serving), four shapes mixed in every batch: results equal the requests evaluated alone."""
    shapes = [(4, 4), (6, 6), (8, 8), (12, 12)]
    ops = {}
    for i, (km, lm) in enumerate(shapes):
        op = W.Operator(km, lm, 1.0)
        op.upload_core(wi.random_core(len(gaunt.channels(lm)), km, seed=60 + i))
        ops[(km, lm)] = op
    # a burst: everything arrives together, so batches must mix shapes
    reqs = [serve.Request(0.0, i, shapes[i % 4], wi.random_cells(*shapes[i % 4], 1 + (37 * i) % 90, seed=700 + i))
            for i in range(24)]
    raw = [r.f.copy() for r in reqs]
    serve.pin_requests(reqs)
    srv = serve.Server(ops, arena_bytes=256 << 20, nslots=4, precision="rf32", max_batch_cells=400)
    res = serve.run(srv, reqs)
    assert res["completed"] == len(reqs) and res["batches"] < len(reqs)
    assert any(len({r.shape for r in b}) > 1 for b in srv.batch_log)  # a batch mixed shapes
    for r in srv.completed:
        alone = ops[r.shape].evaluate(torch.from_numpy(raw[r.rid]).cuda(), precision="rf32")
        torch.cuda.synchronize()
        assert torch.equal(r.out, alone.cpu()), r.rid
