"""The unfactorised GPU baselines of Sec. 4.5 (naive COO loop, dense tensor via cuBLAS)
against the dense oracle: they evaluate the same FP64 bilinear form."""
import numpy as np
import pytest

import wef_inputs as wi
from _parity import FP64_TOL, cell_errors
from oracle import dense, gaunt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_28475_gb300 as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(km, lm, ncells, seed):
    R = wi.random_core(len(gaunt.channels(lm)), km, seed=seed)
    op = W.Operator(km, lm, 1.0)
    op.upload_core(R)
    f = wi.random_cells(km, lm, ncells, seed=seed + 1)
    o = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
    ref = o.evaluate_rows_with_terms(f.reshape(ncells, -1))
    return op, f, ref, R


def _err(a, ref):
    """Largest per-cell guarded error (tests/_parity.py) against the oracle's (Q, T)."""
    return float(np.max(cell_errors(a, *ref)))


@pytest.mark.parametrize("km,lm,ncells", [(0, 0, 2), (2, 3, 45), (4, 4, 33), (3, 6, 5)])
def test_naive_coo_matches_oracle(km, lm, ncells):
    op, f, ref, _ = _case(km, lm, ncells, 40 + km)
    fd = torch.from_numpy(f).cuda()
    q = torch.empty_like(fd)
    ws = torch.empty(max(W.wef_workspace_size(op.h, ncells, 0), 256), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    W.wef_naive_evaluate(op.h, fd.data_ptr(), q.data_ptr(), ncells, ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    err = _err(q.cpu().numpy(), ref)
    assert err < FP64_TOL, err
    # same result as the factorised FP64 path, to rounding
    q2 = op.evaluate(fd)
    torch.cuda.synchronize()
    assert _err(q2.cpu().numpy(), (q.cpu().numpy(), ref[1])) < FP64_TOL


@pytest.mark.parametrize("km,lm,ncells,chunk", [(0, 0, 2, 1), (2, 3, 45, 7), (4, 4, 33, 256)])
def test_dense_tensor_matches_oracle(km, lm, ncells, chunk):
    op, f, ref, R = _case(km, lm, ncells, 60 + km)
    N = op.N
    C = torch.empty(W.wef_dense_tensor_size(op.h) // 8, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    W.wef_dense_assemble(op.h, C.data_ptr(), C.numel() * 8, st)
    fd = torch.from_numpy(f).cuda()
    q = torch.empty_like(fd)
    ws = torch.empty(N * N * 8 * chunk, dtype=torch.uint8, device="cuda")  # `chunk` cells per GEMM
    W.wef_dense_evaluate(op.h, C.data_ptr(), fd.data_ptr(), q.data_ptr(), ncells, ws.data_ptr(), ws.numel(), st)
    torch.cuda.synchronize()
    qn = q.cpu().numpy()
    err = _err(qn, ref)
    assert err < FP64_TOL, err
    assert np.all(qn[:, 0, :4] == 0.0)
    if km >= 1:
        assert np.all(qn[:, 1, 0] == 0.0)
    # the assembled tensor has the symmetric part (in a2, a3) of the oracle's dense C
    o = dense.DenseOperator(km, lm, dense.conservation_zeroing(R, lm))
    Cn = C.cpu().numpy().reshape(N, N, N)
    for a1 in range(N):
        S = o.slice(a1)
        if (a1 // op.NQ == 0 and a1 % op.NQ < 4) or (km >= 1 and a1 == op.NQ):
            assert np.all(Cn[a1] == 0.0)
        else:
            assert np.allclose(Cn[a1] + Cn[a1].T, S + S.T, rtol=0, atol=1e-13)


def test_dense_rejects_short_buffers():
    op, f, _, _ = _case(1, 2, 3, 7)
    N = op.N
    st = torch.cuda.current_stream().cuda_stream
    C = torch.empty(W.wef_dense_tensor_size(op.h) // 8, dtype=torch.float64, device="cuda")
    with pytest.raises(W.WefError):
        W.wef_dense_assemble(op.h, C.data_ptr(), C.numel() * 8 - 8, st)
    fd = torch.from_numpy(f).cuda()
    with pytest.raises(W.WefError):
        W.wef_dense_evaluate(op.h, C.data_ptr(), fd.data_ptr(), fd.data_ptr(), 3, C.data_ptr(), N * N * 8 - 8, st)
