"""Ragged batches through plans (wef_plan_*), checked against the per-shape evaluation
(same arithmetic, so bit-identical) and against the oracle on sampled cells."""
import numpy as np
import pytest

import wef_inputs as wi
from oracle import dense, gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not __import__("os").path.exists(W.LIB_PATH):
        from paper_2605_28475_gb300 import build

        build.build()


def _setup(shapes, counts, gamma=0.5, seed=0):
    ops, cores, fs = [], [], []
    for i, ((km, lm), n) in enumerate(zip(shapes, counts)):
        op = W.Operator(km, lm, gamma)
        R = wi.random_core(len(gaunt.channels(lm)), km, seed=seed + i)
        op.upload_core(R)
        ops.append(op)
        cores.append(R)
        fs.append(wi.random_cells(km, lm, n, seed=seed + 100 + i))
    return ops, cores, fs


def _flat(fs):
    return torch.from_numpy(np.concatenate([f.reshape(-1) for f in fs])).cuda()


def _segments(q, shapes, counts):
    out, o = [], 0
    for (km, lm), n in zip(shapes, counts):
        size = n * (km + 1) * (lm + 1) ** 2
        out.append(q[o:o + size].reshape(n, km + 1, (lm + 1) ** 2))
        o += size
    return out


@pytest.mark.parametrize("prec", ["tf32", "bf16", "rf32"])
def test_ragged_equals_per_shape(prec):
    """One plan over five shapes equals the per-shape evaluations bit for bit (tensor-core
    paths: one persistent launch; radial-first: one launch per shape on forked streams),
    also when replayed from its CUDA graph and after autotuning."""
    shapes = [(2, 3), (4, 4), (6, 6), (3, 5), (16, 2)] + ([(0, 3)] if prec == "rf32" else [])
    counts = [37, 64, 5, 100, 33] + ([9] if prec == "rf32" else [])
    ops, cores, fs = _setup(shapes, counts)
    f = _flat(fs)
    q = torch.full_like(f, float("nan"))
    plan = W.wef_plan_create([o.h for o in ops], counts, W.PRECISIONS[prec], 0)
    ws = torch.empty(max(W.wef_plan_workspace_size(plan), 256), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    W.wef_plan_execute(plan, f.data_ptr(), q.data_ptr(), ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    W.wef_plan_status(plan)
    for op, fi, qi in zip(ops, fs, _segments(q, shapes, counts)):
        ref = op.evaluate(torch.from_numpy(fi).cuda(), precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(qi, ref)
    # graph replay gives identical results
    q2 = torch.full_like(f, float("nan"))
    for _ in range(2):
        W.wef_plan_graph_launch(plan, f.data_ptr(), q2.data_ptr(), ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    assert torch.equal(q2, q)
    # the autotuner keeps results identical
    g = W.wef_plan_autotune(plan, f.data_ptr(), q2.data_ptr(), ws.data_ptr(), ws.numel(), st)
    assert g >= 1
    W.wef_plan_execute(plan, f.data_ptr(), q2.data_ptr(), ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    assert torch.equal(q2, q)
    W.wef_plan_destroy(plan)


def test_ragged_config4_shapes_vs_oracle():
    """Configuration-4 shape set: (Kmax, Lmax) drawn independently from {6,8,10,12,16}; VHS;
    TF32 radial stage.  Cells per shape drawn at random; oracle on one cell per small shape."""
    vals = [6, 8, 10, 12, 16]
    rng = np.random.default_rng(4)
    shapes = [(k, l) for k in vals for l in vals]
    counts = list(rng.integers(20, 90, len(shapes)))
    ops, cores, fs = _setup(shapes, counts, gamma=0.5, seed=50)
    f = _flat(fs)
    q = torch.empty_like(f)
    plan = W.wef_plan_create([o.h for o in ops], counts, W.WEF_MIXED_TF32, 0)
    ws = torch.empty(W.wef_plan_workspace_size(plan), dtype=torch.uint8, device="cuda")
    W.wef_plan_execute(plan, f.data_ptr(), q.data_ptr(), ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    W.wef_plan_status(plan)
    segs = _segments(q, shapes, counts)
    for (km, lm), R, fi, qi in zip(shapes, cores, fs, segs):
        if lm > 8 or km > 10:
            continue
        op = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
        idx = [0, len(fi) - 1]
        Qo = op.evaluate(fi[idx].reshape(2, -1)).reshape(2, km + 1, -1)
        err = float(np.max(np.abs(qi[idx].cpu().numpy() - Qo)) / np.max(np.abs(Qo)))
        assert err < 5e-3, ((km, lm), err)
    W.wef_plan_destroy(plan)


def test_plan_errors():
    op = W.Operator(2, 2, 0.0)
    with pytest.raises(W.WefError) as e:
        W.wef_plan_create([op.h], [10], W.WEF_MIXED_TF32, 0)
    assert e.value.status == W.WEF_ENOCORE
    op.upload_core(np.zeros((len(gaunt.channels(2)), 3, 3, 3)))
    with pytest.raises(W.WefError):
        W.wef_plan_create([op.h], [10], W.WEF_FP64, 0)
    plan = W.wef_plan_create([op.h], [10], W.WEF_MIXED_BF16, 2)
    with pytest.raises(W.WefError):
        W.wef_plan_execute(plan, 0, 0, 0, 0, 0)
    W.wef_plan_destroy(plan)
