"""Ragged batches through plans (wef_plan_*), checked against the per-shape evaluation
(same arithmetic, so bit-identical) and against the oracle on sampled cells."""
import numpy as np
import pytest

import wef_inputs as wi
from _parity import cell_errors, summary, tolerance
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
    if prec == "rf32":  # streams and L2 tile-group size, chosen together
        assert g % 16 in (1, 2, 4, 8) and g // 16 in (12, 24, 48)
    W.wef_plan_execute(plan, f.data_ptr(), q2.data_ptr(), ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    assert torch.equal(q2, q)
    W.wef_plan_destroy(plan)


@pytest.mark.parametrize("prec", ["tf32", "rf32"])
def test_ragged_config4_shapes_vs_oracle(prec):
    """Configuration-4 shape set: (Kmax, Lmax) drawn independently from {6,8,10,12,16}; VHS;
    the TF32 tensor-core plan and the radial-first plan.  Cells per shape drawn at random;
    every one of the 25 shapes checked against the oracle on its first and last cell, over
    24 output rows (the five invariant rows, the last row and 18 drawn at random)."""
    vals = [6, 8, 10, 12, 16]
    rng = np.random.default_rng(4)
    shapes = [(k, l) for k in vals for l in vals]
    counts = list(rng.integers(20, 90, len(shapes)))
    ops, cores, fs = _setup(shapes, counts, gamma=0.5, seed=50)
    f = _flat(fs)
    q = torch.empty_like(f)
    plan = W.wef_plan_create([o.h for o in ops], counts, W.PRECISIONS[prec], 0)
    ws = torch.empty(W.wef_plan_workspace_size(plan), dtype=torch.uint8, device="cuda")
    W.wef_plan_execute(plan, f.data_ptr(), q.data_ptr(), ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    W.wef_plan_status(plan)
    segs = _segments(q, shapes, counts)
    worst = 0.0
    for (km, lm), R, fi, qi in zip(shapes, cores, fs, segs):
        K, NQ = km + 1, (lm + 1) ** 2
        N = K * NQ
        rows = sorted(set([0, 1, 2, 3, NQ, N - 1]
                          + list(np.random.default_rng(km * 100 + lm).choice(np.arange(4, N - 1), 18, replace=False))))
        o = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
        idx = [0, len(fi) - 1]
        Qo, T = o.evaluate_rows_with_terms(fi[idx].reshape(2, -1), rows)
        Qg = qi[idx].cpu().numpy().reshape(2, -1)[:, rows]
        e = summary(cell_errors(Qg, Qo, T))["max"]
        worst = max(worst, e)
        assert e <= tolerance(prec), ((km, lm), e)
        inv = [rows.index(a) for a in (0, 1, 2, 3, NQ)]
        assert np.all(Qg[:, inv] == 0.0)  # the mass, momentum and energy rows
    print(f"PARITY {prec} ragged config-4 shapes: per-cell max {worst:.3e} (bound {tolerance(prec):.2e})")
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


def _ragged_layout(shapes, counts, fs, n_bad, seed):
    """Cells of every shape plus n_bad cells with out-of-range operator indices (-1 and
    nops, alternately), in a shuffled order at scattered offsets: gaps of 5 doubles between
    cells, NaN in the gaps.  Returns the cells as (shape or None, index), the device-side
    arrays as numpy, the flat f and the per-shape cell sizes."""
    rng = np.random.default_rng(seed)
    cells = [(s, i) for s, n in enumerate(counts) for i in range(n)] + [(None, b) for b in range(n_bad)]
    cells = [cells[i] for i in rng.permutation(len(cells))]
    sizes = [(km + 1) * (lm + 1) ** 2 for km, lm in shapes]
    sid, off, cur = [], [], 0
    for s, i in cells:
        sid.append(s if s is not None else (-1 if i % 2 == 0 else len(shapes)))
        off.append(cur)
        cur += (sizes[s] if s is not None else 3) + 5
    f = np.full(cur, np.nan)
    for (s, i), o in zip(cells, off):
        if s is not None:
            f[o:o + sizes[s]] = fs[s][i].reshape(-1)
    return cells, np.array(sid, np.int32), np.array(off, np.int64), f, sizes


@pytest.mark.parametrize("prec", ["rf32", "fp64"])
def test_evaluate_ragged_interleaved(prec):
    """wef_evaluate_ragged on cells of six operators interleaved in a shuffled order at
    scattered offsets, with cells whose operator index is out of range (skipped): every
    cell's Q is bitwise the Q wef_evaluate gives for it, nothing outside the cells' Q is
    written, repeated calls and a CUDA-graph replay agree, and the first and last cell of
    every operator match the oracle on sampled output rows."""
    shapes = [(2, 3), (4, 4), (12, 12), (3, 5), (16, 2), (0, 3)]
    counts = [37, 64, 45, 100, 33, 9]
    ops, cores, fs = _setup(shapes, counts, gamma=1.0, seed=70)
    cells, sid, off, fh, sizes = _ragged_layout(shapes, counts, fs, 6, 5)
    hs = [o.h for o in ops]
    f = torch.from_numpy(fh).cuda()
    q = torch.full_like(f, float("nan"))
    sid_d, off_d = torch.from_numpy(sid).cuda(), torch.from_numpy(off).cuda()
    P = W.PRECISIONS[prec]
    ws = torch.empty(W.wef_ragged_workspace_size(hs, len(cells), P), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    W.wef_evaluate_ragged(hs, sid_d.data_ptr(), off_d.data_ptr(), f.data_ptr(), q.data_ptr(), len(cells), P,
                          ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    qh = q.cpu().numpy()
    refs = []
    for op, fi in zip(ops, fs):
        refs.append(op.evaluate(torch.from_numpy(fi).cuda(), precision=prec).cpu().numpy())
    written = np.zeros(qh.size, bool)
    for (s, i), o in zip(cells, off):
        if s is not None:
            assert np.array_equal(qh[o:o + sizes[s]], refs[s][i].reshape(-1)), (shapes[s], i)
            written[o:o + sizes[s]] = True
    assert np.all(np.isnan(qh[~written]))  # gaps and skipped cells untouched
    # a second call and a CUDA-graph replay give the same bits
    q2 = torch.full_like(f, float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        W.wef_evaluate_ragged(hs, sid_d.data_ptr(), off_d.data_ptr(), f.data_ptr(), q2.data_ptr(), len(cells), P,
                              ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(q2, nan=7.0), torch.nan_to_num(q, nan=7.0))
    # oracle: first and last cell of every operator, sampled rows
    worst = 0.0
    for s, ((km, lm), R, fi) in enumerate(zip(shapes, cores, fs)):
        K, NQ = km + 1, (lm + 1) ** 2
        N = K * NQ
        rows = sorted(set([0, 1, 2, 3, N - 1] + ([NQ] if K > 1 else [])
                          + list(np.random.default_rng(s).choice(N, min(N, 16), replace=False))))
        o = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
        idx = [0, len(fi) - 1]
        Qo, T = o.evaluate_rows_with_terms(fi[idx].reshape(2, -1), rows)
        e = summary(cell_errors(refs[s][idx].reshape(2, -1)[:, rows], Qo, T))["max"]
        worst = max(worst, e)
        assert e <= tolerance(prec), ((km, lm), e)
    print(f"PARITY {prec} wef_evaluate_ragged 6 operators: per-cell max {worst:.3e} (bound {tolerance(prec):.2e})")


def test_evaluate_ragged_errors():
    op = W.Operator(2, 2, 0.0)
    op.upload_core(np.zeros((len(gaunt.channels(2)), 3, 3, 3)))
    d = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(W.WefError):  # tensor-core precisions go through plans
        W.wef_ragged_workspace_size([op.h], 4, W.WEF_MIXED_TF32)
    need = W.wef_ragged_workspace_size([op.h], 4, W.WEF_RADIAL_FP32)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(W.WefError):  # workspace too small
        W.wef_evaluate_ragged([op.h], d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 4, W.WEF_RADIAL_FP32,
                              ws.data_ptr(), need - 256, st)
    with pytest.raises(W.WefError):  # no operators
        W.wef_evaluate_ragged([], d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 4, W.WEF_RADIAL_FP32,
                              ws.data_ptr(), need, st)
    W.wef_evaluate_ragged([op.h], 0, 0, 0, 0, 0, W.WEF_RADIAL_FP32, 0, 0, st)  # no cells: no-op
    op2 = W.Operator(2, 2, 0.0)
    with pytest.raises(W.WefError) as e:
        W.wef_evaluate_ragged([op.h, op2.h], d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 4,
                              W.WEF_RADIAL_FP32, ws.data_ptr(), need, st)
    assert e.value.status == W.WEF_ENOCORE
