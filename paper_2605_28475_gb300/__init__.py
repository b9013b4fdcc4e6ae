"""Python binding of libwef (the C ABI in include/wef.h): argument marshalling only.

Every computation runs in the library: the evaluation in its sm_103a kernels,
table and core construction in its host code.  The functions below carry the
C names; ``Operator`` is a small convenience wrapper that takes torch tensors
(PyTorch is used only for device memory and streams).  If the shared library
is missing the import of any function fails loudly; there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwef.so")

WEF_OK, WEF_EINVAL, WEF_ENOMEM, WEF_ECUDA, WEF_ENOCORE, WEF_ESHAPE, WEF_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
WEF_FP64, WEF_MIXED_BF16, WEF_MIXED_TF32, WEF_RADIAL_FP32, WEF_RADIAL_TC = 0, 1, 2, 3, 4
WEF_CORE_APPLY_NULLSPACE = 1
PRECISIONS = {"fp64": WEF_FP64, "bf16": WEF_MIXED_BF16, "tf32": WEF_MIXED_TF32, "rf32": WEF_RADIAL_FP32,
              "rftc": WEF_RADIAL_TC}

_lib = None


class WefError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"wef status {status}: {msg}")
        self.status = status


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python {os.path.join(_HERE, 'build.py')}`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32p, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "wef_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(vp)], ctypes.c_int),
            "wef_sizes": ([vp, i64p, i64p, i64p, i64p], ctypes.c_int),
            "wef_gaunt_coo": ([vp, i32p, i32p, i32p, i32p, dp], ctypes.c_int),
            "wef_upload_core": ([vp, dp, i64, ctypes.c_uint], ctypes.c_int),
            "wef_workspace_size": ([vp, i64, ctypes.c_int, i64p], ctypes.c_int),
            "wef_evaluate": ([vp, vp, vp, i64, ctypes.c_int, vp, i64, vp], ctypes.c_int),
            "wef_core_build": ([vp, ctypes.c_int, ctypes.c_int, dp, i64], ctypes.c_int),
            "wef_core_build_device": ([vp, ctypes.c_int, ctypes.c_int, dp, i64], ctypes.c_int),
            "wef_flops": ([vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "wef_set_trace_events": ([vp, vp, vp], ctypes.c_int),
            "wef_device_status": ([vp, ctypes.c_int], ctypes.c_int),
            "wef_plan_create": ([ctypes.POINTER(vp), i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
            "wef_plan_workspace_size": ([vp, i64p], ctypes.c_int),
            "wef_plan_execute": ([vp, vp, vp, vp, i64, vp], ctypes.c_int),
            "wef_plan_graph_launch": ([vp, vp, vp, vp, i64, vp], ctypes.c_int),
            "wef_plan_autotune": ([vp, vp, vp, vp, i64, vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "wef_plan_status": ([vp, ctypes.c_int], ctypes.c_int),
            "wef_plan_destroy": ([vp], ctypes.c_int),
            "wef_evaluate_noalloc": ([vp, vp, vp, i64, vp], ctypes.c_int),
            "wef_ragged_workspace_size": ([ctypes.POINTER(vp), ctypes.c_int, i64, ctypes.c_int, i64p], ctypes.c_int),
            "wef_evaluate_ragged": ([ctypes.POINTER(vp), ctypes.c_int, vp, vp, vp, vp, i64, ctypes.c_int, vp, i64, vp],
                                    ctypes.c_int),
            "wef_integrate_workspace_size": ([vp, i64, ctypes.c_int, i64p], ctypes.c_int),
            "wef_integrate": ([vp, vp, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, i64, vp], ctypes.c_int),
            "wef_linearized_apply": ([vp, vp, vp, vp, i64, ctypes.c_int, vp, i64, vp], ctypes.c_int),
            "wef_host_workspace_size": ([vp, i64, ctypes.c_int, i64p], ctypes.c_int),
            "wef_evaluate_host": ([vp, vp, vp, i64, i64, ctypes.c_int, vp, i64, vp], ctypes.c_int),
            "wef_naive_evaluate": ([vp, vp, vp, i64, vp, i64, vp], ctypes.c_int),
            "wef_dense_tensor_size": ([vp, i64p], ctypes.c_int),
            "wef_dense_assemble": ([vp, vp, i64, vp], ctypes.c_int),
            "wef_dense_workspace_size": ([vp, i64, i64p], ctypes.c_int),
            "wef_dense_evaluate": ([vp, vp, vp, vp, i64, vp, i64, vp], ctypes.c_int),
            "wef_last_error": ([], ctypes.c_char_p),
            "wef_destroy": ([vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != WEF_OK:
        raise WefError(status, lib().wef_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def wef_create(kmax, lmax, gamma):
    h = ctypes.c_void_p()
    _check(lib().wef_create(int(kmax), int(lmax), float(gamma), ctypes.byref(h)))
    return h


def wef_sizes(op):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().wef_sizes(op, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def wef_gaunt_coo(op):
    n = wef_sizes(op)[2]
    q1, q2, q3, c = (np.empty(n, np.int32) for _ in range(4))
    g = np.empty(n, np.float64)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
    _check(lib().wef_gaunt_coo(op, ip(q1), ip(q2), ip(q3), ip(c), _dp(g)))
    return q1, q2, q3, c, g


def wef_upload_core(op, R, flags=WEF_CORE_APPLY_NULLSPACE):
    R = np.ascontiguousarray(R, dtype=np.float64)
    _check(lib().wef_upload_core(op, _dp(R), R.size, int(flags)))


def wef_workspace_size(op, ncells, prec=WEF_FP64):
    b = ctypes.c_int64()
    _check(lib().wef_workspace_size(op, int(ncells), int(prec), ctypes.byref(b)))
    return b.value


def wef_evaluate(op, f_ptr, q_ptr, ncells, prec, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_evaluate(op, f_ptr, q_ptr, int(ncells), int(prec), ws_ptr, int(ws_bytes), stream_ptr))


def wef_evaluate_noalloc(op, f_ptr, q_ptr, ncells, stream_ptr):
    _check(lib().wef_evaluate_noalloc(op, f_ptr, q_ptr, int(ncells), stream_ptr))


def _op_array(ops):
    return (ctypes.c_void_p * len(ops))(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops])


def wef_ragged_workspace_size(ops, ncells, prec=WEF_RADIAL_FP32):
    b = ctypes.c_int64()
    _check(lib().wef_ragged_workspace_size(_op_array(ops), len(ops), int(ncells), int(prec), ctypes.byref(b)))
    return b.value


def wef_evaluate_ragged(ops, shape_id_ptr, offset_ptr, f_ptr, q_ptr, ncells, prec, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_evaluate_ragged(_op_array(ops), len(ops), shape_id_ptr, offset_ptr, f_ptr, q_ptr, int(ncells),
                                     int(prec), ws_ptr, int(ws_bytes), stream_ptr))


def wef_core_build(op, pad_rad=20, pad_ang=20):
    n = wef_sizes(op)[3]
    R = np.empty(n, np.float64)
    _check(lib().wef_core_build(op, int(pad_rad), int(pad_ang), _dp(R), n))
    return R


def wef_core_build_device(op, pad_rad=20, pad_ang=20):
    n = wef_sizes(op)[3]
    R = np.empty(n, np.float64)
    _check(lib().wef_core_build_device(op, int(pad_rad), int(pad_ang), _dp(R), n))
    return R


def wef_flops(op, prec=WEF_FP64):
    a, t = ctypes.c_double(), ctypes.c_double()
    _check(lib().wef_flops(op, int(prec), ctypes.byref(a), ctypes.byref(t)))
    return a.value, t.value


def wef_set_trace_events(op, ev_start, ev_stop):
    _check(lib().wef_set_trace_events(op, ev_start, ev_stop))


def wef_device_status(op, reset=False):
    _check(lib().wef_device_status(op, 1 if reset else 0))


def wef_plan_create(ops, ncells, prec=WEF_MIXED_TF32, granularity=0):
    n = len(ops)
    arr = (ctypes.c_void_p * n)(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops])
    cnt = (ctypes.c_int64 * n)(*[int(c) for c in ncells])
    h = ctypes.c_void_p()
    _check(lib().wef_plan_create(arr, cnt, n, int(prec), int(granularity), ctypes.byref(h)))
    return h


def wef_plan_workspace_size(plan):
    b = ctypes.c_int64()
    _check(lib().wef_plan_workspace_size(plan, ctypes.byref(b)))
    return b.value


def wef_plan_execute(plan, f_ptr, q_ptr, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_plan_execute(plan, f_ptr, q_ptr, ws_ptr, int(ws_bytes), stream_ptr))


def wef_plan_graph_launch(plan, f_ptr, q_ptr, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_plan_graph_launch(plan, f_ptr, q_ptr, ws_ptr, int(ws_bytes), stream_ptr))


def wef_plan_autotune(plan, f_ptr, q_ptr, ws_ptr, ws_bytes, stream_ptr):
    g = ctypes.c_int()
    _check(lib().wef_plan_autotune(plan, f_ptr, q_ptr, ws_ptr, int(ws_bytes), stream_ptr, ctypes.byref(g)))
    return g.value


def wef_plan_status(plan, reset=False):
    _check(lib().wef_plan_status(plan, 1 if reset else 0))


def wef_plan_destroy(plan):
    _check(lib().wef_plan_destroy(plan))


def wef_integrate_workspace_size(op, ncells, prec=WEF_FP64):
    b = ctypes.c_int64()
    _check(lib().wef_integrate_workspace_size(op, int(ncells), int(prec), ctypes.byref(b)))
    return b.value


def wef_integrate(op, f_ptr, ncells, dt, nsteps, prec, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_integrate(op, f_ptr, int(ncells), float(dt), int(nsteps), int(prec), ws_ptr, int(ws_bytes), stream_ptr))


def wef_linearized_apply(op, c0_ptr, d_ptr, out_ptr, ncells, prec, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_linearized_apply(op, c0_ptr, d_ptr, out_ptr, int(ncells), int(prec), ws_ptr, int(ws_bytes), stream_ptr))


def wef_host_workspace_size(op, chunk_cells, prec=WEF_FP64):
    b = ctypes.c_int64()
    _check(lib().wef_host_workspace_size(op, int(chunk_cells), int(prec), ctypes.byref(b)))
    return b.value


def wef_evaluate_host(op, f_ptr, q_ptr, ncells, chunk_cells, prec, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_evaluate_host(op, f_ptr, q_ptr, int(ncells), int(chunk_cells), int(prec), ws_ptr, int(ws_bytes),
                                   stream_ptr))


def wef_naive_evaluate(op, f_ptr, q_ptr, ncells, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_naive_evaluate(op, f_ptr, q_ptr, int(ncells), ws_ptr, int(ws_bytes), stream_ptr))


def wef_dense_tensor_size(op):
    b = ctypes.c_int64()
    _check(lib().wef_dense_tensor_size(op, ctypes.byref(b)))
    return b.value


def wef_dense_assemble(op, c_ptr, nbytes, stream_ptr):
    _check(lib().wef_dense_assemble(op, c_ptr, int(nbytes), stream_ptr))


def wef_dense_workspace_size(op, ncells):
    b = ctypes.c_int64()
    _check(lib().wef_dense_workspace_size(op, int(ncells), ctypes.byref(b)))
    return b.value


def wef_dense_evaluate(op, c_ptr, f_ptr, q_ptr, ncells, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().wef_dense_evaluate(op, c_ptr, f_ptr, q_ptr, int(ncells), ws_ptr, int(ws_bytes), stream_ptr))


def wef_last_error():
    return lib().wef_last_error().decode()


def wef_destroy(op):
    _check(lib().wef_destroy(op))


def _cells_arg(t, n_per_cell, name, cuda=True, device=None):
    """Number of cells of a [ncells, K, NQ] (or [ncells, K * NQ]) float64 tensor, after
    checking what the library cannot: dtype, contiguity, placement and the per-cell size
    (a tensor shaped for another operator would be read or written past its end)."""
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 tensor")
    if t.is_cuda != cuda or (device is not None and t.device != device):
        raise ValueError(f"{name} must be on {device if device is not None else ('a CUDA device' if cuda else 'the host')}")
    if t.dim() < 1 or t.numel() != t.shape[0] * n_per_cell:
        raise ValueError(f"{name} must hold {n_per_cell} doubles per cell, got shape {tuple(t.shape)}")
    return t.shape[0]


class Operator:
    """Owns a wef_op; evaluates Q(f, f) on torch CUDA tensors [ncells, K, NQ] float64.

    The helper keeps one workspace per kind of call and reuses it: calls made through the
    same Operator on different streams must be ordered by the caller."""

    def __init__(self, kmax, lmax, gamma):
        self.kmax, self.lmax, self.gamma = kmax, lmax, gamma
        self.K, self.NQ = kmax + 1, (lmax + 1) ** 2
        self.h = wef_create(kmax, lmax, gamma)
        self.N, self.n_channels, self.n_gaunt, self.core_len = wef_sizes(self.h)
        self._ws = None

    def build_core(self, pad_rad=20, pad_ang=20, device=False):
        """The raw kinematic core [channel][k1][k2][k3]: host builder, or the GPU one (device=True)."""
        fn = wef_core_build_device if device else wef_core_build
        return fn(self.h, pad_rad, pad_ang).reshape(self.n_channels, self.K, self.K, self.K)

    def upload_core(self, R, flags=WEF_CORE_APPLY_NULLSPACE):
        wef_upload_core(self.h, R, flags)

    def workspace(self, ncells, prec, device):
        import torch

        need = wef_workspace_size(self.h, ncells, prec)
        if self._ws is None or self._ws.numel() < max(need, 256) or self._ws.device != device:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
        return self._ws

    def evaluate(self, f, q=None, precision="fp64", stream=None):
        import torch

        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        ncells = _cells_arg(f, self.N, "f")
        if q is None:
            q = torch.empty_like(f)
        elif _cells_arg(q, self.N, "q", device=f.device) != ncells:
            raise ValueError("q must have as many cells as f")
        ws = self.workspace(ncells, prec, f.device)
        st = stream if stream is not None else torch.cuda.current_stream(f.device)
        wef_evaluate(self.h, f.data_ptr(), q.data_ptr(), ncells, prec, ws.data_ptr(), ws.numel(), st.cuda_stream)
        return q

    def _dyn_workspace(self, ncells, prec, device):
        import torch

        need = wef_integrate_workspace_size(self.h, ncells, prec)
        ws = getattr(self, "_dws", None)
        if ws is None or ws.numel() < max(need, 256) or ws.device != device:
            self._dws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
        return self._dws

    def integrate(self, f, dt, nsteps, precision="fp64", stream=None):
        """Advance df/dt = Q(f, f) in place by `nsteps` RK4 steps of size `dt`."""
        import torch

        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _cells_arg(f, self.N, "f")
        ws = self._dyn_workspace(f.shape[0], prec, f.device)
        st = stream if stream is not None else torch.cuda.current_stream(f.device)
        wef_integrate(self.h, f.data_ptr(), f.shape[0], dt, nsteps, prec, ws.data_ptr(), ws.numel(), st.cuda_stream)
        return f

    def linearized_apply(self, c0, d, out=None, precision="fp64", stream=None):
        """out = L d, L the linearization of Q at the base states c0 (one per cell)."""
        import torch

        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        ncells = _cells_arg(d, self.N, "d")
        if _cells_arg(c0, self.N, "c0", device=d.device) != ncells:
            raise ValueError("c0 and d must have the same number of cells")
        if out is None:
            out = torch.empty_like(d)
        elif _cells_arg(out, self.N, "out", device=d.device) != ncells:
            raise ValueError("out must have as many cells as d")
        ws = self._dyn_workspace(d.shape[0], prec, d.device)
        st = stream if stream is not None else torch.cuda.current_stream(d.device)
        wef_linearized_apply(self.h, c0.data_ptr(), d.data_ptr(), out.data_ptr(), d.shape[0], prec, ws.data_ptr(),
                             ws.numel(), st.cuda_stream)
        return out

    def evaluate_host(self, f, q=None, precision="fp64", chunk_cells=4096, stream=None, device=None):
        """Q(f, f) for f in host memory (a CPU float64 tensor, ideally pinned); the copies of
        one chunk overlap the evaluation of the next.  Returns q (host) after the stream's
        work is queued; synchronize the stream before reading it."""
        import torch

        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        ncells = _cells_arg(f, self.N, "f", cuda=False)
        if q is None:
            q = torch.empty_like(f, pin_memory=f.is_pinned())
        elif _cells_arg(q, self.N, "q", cuda=False) != ncells:
            raise ValueError("q must have as many cells as f")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        need = wef_host_workspace_size(self.h, chunk_cells, prec)
        ws = getattr(self, "_hws", None)
        if ws is None or ws.numel() < need or ws.device != dev:
            self._hws = ws = torch.empty(need, dtype=torch.uint8, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        wef_evaluate_host(self.h, f.data_ptr(), q.data_ptr(), f.shape[0], chunk_cells, prec, ws.data_ptr(), ws.numel(),
                          st.cuda_stream)
        return q

    def close(self):
        if self.h is not None:
            wef_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
