"""Thin ctypes binding of libwlr.so (the C ABI in include/wlr.h).

Argument marshalling only: every step of the sWLR iteration runs in the library's
CUDA kernels.  Functions keep the C names (wlr_create, wlr_set_data, ...).  Matrix
arguments may be torch tensors (device or host) or NumPy arrays (host); they must be
column-major (Fortran order; a torch tensor ``t`` qualifies when ``t.T`` is
contiguous) or have column stride 1 with a leading dimension.

There is no fallback: if the shared library is missing or fails to load, importing
this module raises, so nothing silently runs elsewhere.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libwlr.so")

WLR_OK = 0
WLR_ERR_INVALID_ARG = 1
WLR_ERR_NONPOSITIVE_WEIGHT = 2
WLR_ERR_RANK_DEFICIENT = 3
WLR_ERR_NOT_SPD = 4
WLR_ERR_NO_CONVERGENCE = 5
WLR_ERR_DEVICE_TIMEOUT = 6
WLR_ERR_CUDA = 7
WLR_ERR_OOM = 8
WLR_ERR_NOT_READY = 9
WLR_ERR_UNSUPPORTED = 10

WLR_F32, WLR_F64 = 0, 1
WLR_MEM_DEVICE, WLR_MEM_HOST = 0, 1
WLR_PREC_FP64, WLR_PREC_FP32 = 0, 1
WLR_INIT_A1, WLR_INIT_RANDOM, WLR_INIT_USER = 0, 1, 2
WLR_STOP_PAPER, WLR_STOP_RELATIVE, WLR_STOP_NONE, WLR_STOP_OBJECTIVE = 0, 1, 2, 3


class wlr_options(ct.Structure):
    _fields_ = [
        ("precision", ct.c_int32),
        ("stop", ct.c_int32),
        ("eig_block", ct.c_int32),
        ("eig_iters", ct.c_int32),
        ("eig_iters_cold", ct.c_int32),
        ("use_graph", ct.c_int32),
        ("seed", ct.c_uint64),
        ("autotune", ct.c_int32),
    ]


class wlr_ws_shape(ct.Structure):
    _fields_ = [("h", ct.c_int32), ("w", ct.c_int32), ("c1", ct.c_int32), ("c2", ct.c_int32),
                ("hidden", ct.c_int32), ("r_max", ct.c_int32)]


class WlrError(RuntimeError):
    def __init__(self, status: int, message: str, index: int = -1):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status
        self.index = index   # failing handle of a batched call, -1 otherwise


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libwlr.so not built at {_LIB_PATH}; run __graft_entry__.build()")
    lib = ct.CDLL(_LIB_PATH)
    H = ct.c_void_p
    P = ct.c_void_p
    i64, i32, u64, dbl = ct.c_int64, ct.c_int32, ct.c_uint64, ct.c_double
    sig = {
        "wlr_default_options": (None, [ct.POINTER(wlr_options)]),
        "wlr_create": (i32, [ct.POINTER(H), i64, i64, i64, i64, ct.POINTER(wlr_options), P]),
        "wlr_set_data": (i32, [H, P, i64, P, i64, i32, i32]),
        "wlr_set_init": (i32, [H, i32, P, i64, i32, i32, u64]),
        "wlr_step": (i32, [H, ct.POINTER(dbl)]),
        "wlr_solve": (i32, [H, dbl, i32, ct.POINTER(i32), ct.POINTER(dbl)]),
        "wlr_objective": (i32, [H, ct.POINTER(dbl)]),
        "wlr_get_result": (i32, [H, P, i64, P, i64, i32, i32]),
        "wlr_get_factors": (i32, [H, P, P, P]),
        "wlr_get_history": (i32, [H, P, P, i32, ct.POINTER(i32)]),
        "wlr_get_iteration": (i32, [H, ct.POINTER(i32)]),
        "wlr_get_state": (i32, [H, P, i64, ct.POINTER(i64)]),
        "wlr_set_state": (i32, [H, P, i64]),
        "wlr_solve_batched": (i32, [ct.POINTER(H), i32, i32, ct.POINTER(i32)]),
        "wlr_refine": (i32, [H, P, i64, i32, ct.POINTER(dbl), ct.POINTER(dbl)]),
        "wlr_destroy": (i32, [H]),
        "wlr_status_string": (ct.c_char_p, [i32]),
        "wlr_last_error": (ct.c_char_p, [H]),
        "wlr_kernel_launches": (i64, [H]),
        "wlr_profile": (i32, [H, i32, ct.c_char_p, i32, P, P, i32, ct.POINTER(i32)]),
        "wlr_x1_update_noalloc": (i32, [P, i64, P, i64, P, i64, i64, i64, i64, P, P, P, P, P, P]),
        "wlr_ws_create": (i32, [ct.POINTER(H), ct.POINTER(wlr_ws_shape), i32, u64, P]),
        "wlr_ws_destroy": (i32, [H]),
        "wlr_ws_param_count": (i64, [H]),
        "wlr_ws_get_params": (i32, [H, P, i32]),
        "wlr_ws_get_grads": (i32, [H, P, i32]),
        "wlr_ws_set_params": (i32, [H, P, i32]),
        "wlr_ws_prepare": (i32, [H, P, i64, P, i64, i32, i32, i32, i32, P]),
        "wlr_ws_forward": (i32, [H, P, i32, P, i32, P]),
        "wlr_ws_loss": (i32, [H, P, i64, i32, i32, i32, P, i32, P, i64, P, P]),
        "wlr_ws_backward": (i32, [H, P]),
        "wlr_ws_adam": (i32, [H, ct.c_float, ct.c_float, ct.c_float, ct.c_float, ct.c_float]),
        "wlr_ws_launches": (i64, [H]),
        "wlr_get_basis": (i32, [H, P, i64]),
        "wlr_set_data_cols": (i32, [H, P, i64, P, i64, i32, i32, P]),
        "wlr_selftest_bounded_wait": (i32, [i64, P]),
        "wlr_get_x": (i32, [H, P, i64, i32, i32]),
        "wlr_set_init_learned": (i32, [H, H, i32, i32, i32, ct.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTED = (
    "wlr_default_options", "wlr_create", "wlr_set_data", "wlr_set_init", "wlr_step",
    "wlr_solve", "wlr_objective", "wlr_get_result", "wlr_get_factors", "wlr_get_history",
    "wlr_get_iteration", "wlr_get_state", "wlr_set_state", "wlr_solve_batched", "wlr_refine",
    "wlr_destroy",
    "wlr_status_string",
    "wlr_last_error",
    "wlr_kernel_launches", "wlr_profile", "wlr_x1_update_noalloc",
    "wlr_ws_create", "wlr_ws_destroy", "wlr_ws_param_count", "wlr_ws_get_params",
    "wlr_ws_get_grads", "wlr_ws_set_params", "wlr_ws_prepare", "wlr_ws_forward", "wlr_ws_loss",
    "wlr_ws_backward", "wlr_ws_adam", "wlr_ws_launches", "wlr_get_basis", "wlr_set_init_learned",
    "wlr_set_data_cols", "wlr_get_x", "wlr_selftest_bounded_wait",
)


def library_path() -> str:
    return _LIB_PATH


def status_string(st: int) -> str:
    return _lib.wlr_status_string(int(st)).decode()


def _check(st: int, h=None, ok=(WLR_OK,)):
    if st not in ok:
        msg = _lib.wlr_last_error(h).decode() if h is not None else _lib.wlr_last_error(None).decode()
        raise WlrError(st, msg)
    return st


# ------------------------------------------------------------------ marshalling
def _matrix(x):
    """(pointer, leading dimension, dtype code, memory code, keepalive) of a column-major
    matrix given as a torch tensor or a NumPy array."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype == torch.float32:
            dt = WLR_F32
        elif x.dtype == torch.float64:
            dt = WLR_F64
        else:
            raise TypeError("float32 or float64 tensors only")
        if x.dim() != 2 or x.stride(0) != 1:
            raise ValueError("need a 2-D column-major tensor (stride(0) == 1)")
        ld = max(x.stride(1), x.shape[0]) if x.shape[1] > 1 else x.shape[0]
        mem = WLR_MEM_DEVICE if x.is_cuda else WLR_MEM_HOST
        return x.data_ptr(), ld, dt, mem, x
    a = np.asarray(x)
    if a.dtype == np.float32:
        dt = WLR_F32
    elif a.dtype == np.float64:
        dt = WLR_F64
    else:
        raise TypeError("float32 or float64 arrays only")
    if a.ndim != 2:
        raise ValueError("need a 2-D array")
    if not a.flags.f_contiguous:
        a = np.asfortranarray(a)
    return a.ctypes.data, a.shape[0], dt, WLR_MEM_HOST, a


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------------ C names
def wlr_default_options() -> wlr_options:
    o = wlr_options()
    _lib.wlr_default_options(ct.byref(o))
    return o


def wlr_create(m, n, k, r, options: wlr_options | None = None, stream=None):
    h = ct.c_void_p()
    st = _lib.wlr_create(ct.byref(h), int(m), int(n), int(k), int(r),
                         ct.byref(options) if options is not None else None, _stream_ptr(stream))
    if st != WLR_OK:
        raise WlrError(st, _lib.wlr_last_error(None).decode())
    return h


def wlr_set_data(h, A, W1):
    pa, lda, dta, mema, ka = _matrix(A)
    pw, ldw, dtw, memw, kw = _matrix(W1)
    if dta != dtw or mema != memw:
        raise ValueError("A and W1 must share dtype and memory kind")
    return _check(_lib.wlr_set_data(h, pa, lda, pw, ldw, dta, mema), h)


def wlr_set_data_cols(h, A, W1, cols):
    """wlr_set_data with the weighted frames at the columns `cols` of A (W1's column order)."""
    pa, lda, dta, mema, ka = _matrix(A)
    pw, ldw, dtw, memw, kw = _matrix(W1)
    if dta != dtw or mema != memw:
        raise ValueError("A and W1 must share dtype and memory kind")
    c = np.ascontiguousarray(cols, dtype=np.int32)
    if c.ndim != 1 or c.size != W1.shape[1]:
        raise ValueError("cols must list one column of A per column of W1")
    return _check(_lib.wlr_set_data_cols(h, pa, lda, pw, ldw, dta, mema, c.ctypes.data), h)


def wlr_get_x(h, X):
    """X = (X1, X2) in the caller's column order (m x n, column-major)."""
    if isinstance(X, np.ndarray) and not X.flags.f_contiguous:
        raise ValueError("NumPy outputs must be Fortran-ordered")
    p, ld, dt, mem, _keep = _matrix(X)
    _check(_lib.wlr_get_x(h, p, ld, dt, mem), h)


def wlr_selftest_bounded_wait(limit_ns=10_000_000, stream=None):
    """Status of the bounded-wait self-test (WLR_ERR_DEVICE_TIMEOUT is the expected one)."""
    return int(_lib.wlr_selftest_bounded_wait(int(limit_ns), _stream_ptr(stream)))


def wlr_set_init(h, kind=WLR_INIT_A1, X1_0=None, seed=0):
    if X1_0 is None:
        return _check(_lib.wlr_set_init(h, kind, None, 0, WLR_F64, WLR_MEM_HOST, int(seed)), h)
    p, ld, dt, mem, keep = _matrix(X1_0)
    return _check(_lib.wlr_set_init(h, kind, p, ld, dt, mem, int(seed)), h)


def wlr_step(h, want_objective=True):
    F = ct.c_double(np.nan)
    _check(_lib.wlr_step(h, ct.byref(F) if want_objective else None), h)
    return F.value if want_objective else None


def wlr_solve(h, tol=1e-7, max_iter=100):
    it = ct.c_int32(0)
    F = ct.c_double(np.nan)
    st = _check(_lib.wlr_solve(h, float(tol), int(max_iter), ct.byref(it), ct.byref(F)), h,
                ok=(WLR_OK, WLR_ERR_NO_CONVERGENCE))
    return it.value, F.value, st == WLR_OK


def wlr_objective(h):
    F = ct.c_double(np.nan)
    _check(_lib.wlr_objective(h, ct.byref(F)), h)
    return F.value


def wlr_get_result(h, X1=None, X2=None):
    """Copy X1 (and X2 = X1 C + D) into caller buffers (torch tensors or NumPy arrays,
    column-major, float32/float64, same dtype and memory kind)."""
    p1 = ld1 = 0
    p2 = ld2 = 0
    dt = mem = None
    keep = []
    if X1 is not None:
        p1, ld1, dt, mem, k1 = _matrix(X1)
        keep.append(k1)
    if X2 is not None:
        p2, ld2, dt2, mem2, k2 = _matrix(X2)
        keep.append(k2)
        if dt is not None and (dt2 != dt or mem2 != mem):
            raise ValueError("X1 and X2 must share dtype and memory kind")
        dt, mem = dt2, mem2
    if dt is None:
        return
    if isinstance(X1, np.ndarray) and not X1.flags.f_contiguous:
        raise ValueError("NumPy outputs must be Fortran-ordered")
    if isinstance(X2, np.ndarray) and not X2.flags.f_contiguous:
        raise ValueError("NumPy outputs must be Fortran-ordered")
    _check(_lib.wlr_get_result(h, p1 or None, ld1, p2 or None, ld2, dt, mem), h)


def wlr_get_factors(h, k, n2, s):
    C = np.zeros((k, n2), order="F")
    Vs = np.zeros((n2, s), order="F")
    sig2 = np.zeros(max(s, 0))
    _check(_lib.wlr_get_factors(h, C.ctypes.data if C.size else None,
                                Vs.ctypes.data if Vs.size else None,
                                sig2.ctypes.data if sig2.size else None), h)
    return C, Vs, sig2


def wlr_get_history(h, cap=65536):
    n = ct.c_int32(0)
    _check(_lib.wlr_get_history(h, None, None, 0, ct.byref(n)), h)
    F = np.zeros(max(n.value, 1))
    E = np.zeros(max(n.value, 1))
    _check(_lib.wlr_get_history(h, F.ctypes.data, E.ctypes.data, n.value, ct.byref(n)), h)
    return F[:n.value], E[:n.value]


def wlr_get_iteration(h):
    p = ct.c_int32(0)
    _check(_lib.wlr_get_iteration(h, ct.byref(p)), h)
    return p.value


def wlr_get_state(h):
    """Checkpoint of the iteration as bytes (host copy of the library's state)."""
    n = ct.c_int64(0)
    _check(_lib.wlr_get_state(h, None, 0, ct.byref(n)), h)
    buf = ct.create_string_buffer(max(n.value, 1))
    _check(_lib.wlr_get_state(h, buf, n.value, ct.byref(n)), h)
    return buf.raw[:n.value]


def wlr_set_state(h, state):
    """Restore a checkpoint made by wlr_get_state (same sizes, options and data)."""
    b = bytes(state)
    buf = ct.create_string_buffer(b, max(len(b), 1))
    _check(_lib.wlr_set_state(h, buf, len(b)), h)


def wlr_solve_batched(handles, iters):
    """`iters` iterations on every handle of the list, joined into one graph launch per
    three iterations once each handle is warmed up (see include/wlr.h)."""
    hs = list(handles)
    arr = (ct.c_void_p * max(len(hs), 1))(*hs)
    failed = ct.c_int32(-1)
    st = _lib.wlr_solve_batched(arr, len(hs), int(iters), ct.byref(failed))
    if st != WLR_OK:
        h = hs[failed.value] if 0 <= failed.value < len(hs) else (hs[0] if hs and hs[0] else None)
        msg = _lib.wlr_last_error(h).decode()
        if not msg and h is not None:
            msg = _lib.wlr_last_error(None).decode()
        raise WlrError(st, msg, failed.value)
    return st


def wlr_refine(h, X1_out=None):
    """FP64 refinement sweep from the current X1_p (see include/wlr.h).  X1_out: float64
    column-major m x k torch tensor or NumPy array, or None.  Returns (F_p, F_{p+1})."""
    F0, F1 = ct.c_double(0), ct.c_double(0)
    if X1_out is None:
        _check(_lib.wlr_refine(h, None, 0, WLR_MEM_DEVICE, ct.byref(F0), ct.byref(F1)), h)
    else:
        if isinstance(X1_out, np.ndarray) and not X1_out.flags.f_contiguous:
            raise ValueError("X1_out must be column-major (Fortran order)")
        ptr, ld, dt, mem, _keep = _matrix(X1_out)
        if dt != WLR_F64:
            raise TypeError("X1_out must be float64")
        _check(_lib.wlr_refine(h, ptr, ld, mem, ct.byref(F0), ct.byref(F1)), h)
    return F0.value, F1.value


def solve_batched(solvers, iters):
    """wlr_solve_batched over Solver objects."""
    return wlr_solve_batched([s.h for s in solvers], iters)


def wlr_destroy(h):
    if h:
        _lib.wlr_destroy(h)


def wlr_status_string(st):
    return status_string(st)


def wlr_last_error(h=None):
    return _lib.wlr_last_error(h).decode()


def wlr_kernel_launches(h):
    return int(_lib.wlr_kernel_launches(h))


def wlr_profile(h, reps=20, max_kernels=64):
    """{kernel name: (total ms, launches)} over reps further iterations."""
    buf = ct.create_string_buffer(8192)
    ms = np.zeros(max_kernels)
    ln = np.zeros(max_kernels, dtype=np.int32)
    n = ct.c_int32(0)
    _check(_lib.wlr_profile(h, int(reps), buf, 8192, ms.ctypes.data, ln.ctypes.data, max_kernels,
                            ct.byref(n)), h)
    names = buf.value.decode().split("\n")[:n.value]
    return {nm: (float(ms[q]), int(ln[q])) for q, nm in enumerate(names)}


def wlr_x1_update_noalloc(A, W1, X1, k, r, C, Vs, X1_next, wterm=None, status=None, stream=None):
    """X1 update into X1_next without any device allocation (see include/wlr.h).
    A, W1, X1, C, Vs, X1_next: float32 CUDA tensors, column-major; X1 and X1_next with
    leading dimension m; wterm: a 1-element float64 CUDA tensor or None; status: a
    1-element int32 CUDA tensor or None.  Asynchronous on `stream`."""
    pa, lda, dta, mema, _ = _matrix(A)
    pw, ldw, dtw, memw, _ = _matrix(W1)
    px, ldx, dtx, memx, _ = _matrix(X1)
    pn, ldn, dtn, memn, _ = _matrix(X1_next)
    m, n = A.shape
    k, r = int(k), int(r)
    n2, s = n - k, r - k
    if {dta, dtw, dtx, dtn} != {WLR_F32} or {mema, memw, memx, memn} != {WLR_MEM_DEVICE}:
        raise ValueError("float32 device tensors only")
    if tuple(X1.shape) != (m, k) or tuple(X1_next.shape) != (m, k) or tuple(W1.shape) != (m, k):
        raise ValueError("W1, X1 and X1_next must be m x k")
    if ldx != m or ldn != m:
        raise ValueError("X1 and X1_next need leading dimension m")

    def factor(t, rows, cols, name):
        # column-major float32 device matrix rows x cols with leading dimension rows
        if rows * cols == 0:
            return None
        if t is None:
            raise ValueError(f"{name} is required")
        p, ld, dt, mem, _ = _matrix(t)
        if dt != WLR_F32 or mem != WLR_MEM_DEVICE:
            raise ValueError(f"{name} must be a float32 device tensor")
        if tuple(t.shape) != (rows, cols) or ld != rows:
            raise ValueError(f"{name} must be {rows} x {cols}, column-major with leading dimension {rows}")
        return p

    pc = factor(C, k, n2, "C")
    pv = factor(Vs, n2, s, "Vs")
    st = _lib.wlr_x1_update_noalloc(pa, lda, pw, ldw, px, m, n, k, r, pc, pv, pn,
                                    wterm.data_ptr() if wterm is not None else None,
                                    status.data_ptr() if status is not None else None,
                                    _stream_ptr(stream))
    if st != WLR_OK:
        raise WlrError(st, "wlr_x1_update_noalloc: " + _lib.wlr_last_error(None).decode())
    return st


# ------------------------------------------------------------------ learned warm start
def _dev_f32(t, name):
    """data_ptr of a contiguous float32 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
        raise ValueError(f"{name} must be a float32 CUDA tensor")
    if not t.is_contiguous() and not (t.dim() == 2 and t.stride(0) == 1):
        raise ValueError(f"{name} must be contiguous (row-major) or column-major")
    return t.data_ptr()


def _net_check(st, net):
    if st != WLR_OK:
        raise WlrError(st, _lib.wlr_last_error(None).decode())
    return st


def wlr_ws_create(h, w, c1, c2, hidden, r_max, max_frames, seed=0, stream=None):
    sh = wlr_ws_shape(h, w, c1, c2, hidden, r_max)
    net = ct.c_void_p()
    _net_check(_lib.wlr_ws_create(ct.byref(net), ct.byref(sh), int(max_frames), int(seed),
                                  _stream_ptr(stream)), None)
    return net


def wlr_ws_destroy(net):
    if net:
        _lib.wlr_ws_destroy(net)


def wlr_ws_param_count(net):
    return int(_lib.wlr_ws_param_count(net))


def wlr_ws_get_params(net):
    out = np.empty(wlr_ws_param_count(net), dtype=np.float32)
    _net_check(_lib.wlr_ws_get_params(net, out.ctypes.data, WLR_MEM_HOST), net)
    return out


def wlr_ws_get_grads(net):
    out = np.empty(wlr_ws_param_count(net), dtype=np.float32)
    _net_check(_lib.wlr_ws_get_grads(net, out.ctypes.data, WLR_MEM_HOST), net)
    return out


def wlr_ws_set_params(net, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != wlr_ws_param_count(net):
        raise ValueError("wrong parameter count")
    _net_check(_lib.wlr_ws_set_params(net, a.ctypes.data, WLR_MEM_HOST), net)


def wlr_ws_prepare(net, A, W1, H, W, k, X):
    """Network input X (n, 2, h, w) of the clip A (m x n, column-major float32 CUDA tensor)."""
    pa, lda, dta, mema, _ = _matrix(A)
    pw, ldw, dtw, memw, _ = _matrix(W1)
    if {dta, dtw} != {WLR_F32} or {mema, memw} != {WLR_MEM_DEVICE}:
        raise ValueError("A and W1 must be float32 CUDA tensors")
    _net_check(_lib.wlr_ws_prepare(net, pa, lda, pw, ldw, int(H), int(W), int(A.shape[1]), int(k),
                                   _dev_f32(X, "X")), net)


def wlr_ws_forward(net, X, clip_start, Omega):
    cs = np.ascontiguousarray(clip_start, dtype=np.int32)
    frames = int(cs[-1])
    _net_check(_lib.wlr_ws_forward(net, _dev_f32(X, "X"), frames, cs.ctypes.data, len(cs) - 1,
                                   _dev_f32(Omega, "Omega")), net)


def wlr_ws_loss(net, A, k, Omega_c, r, V, loss, dOmega_c):
    """Adds the clip's loss to loss (1-element float64 CUDA tensor); writes dOmega_c."""
    pa, lda, dta, mema, _ = _matrix(A)
    pv, ldv, dtv, memv, _ = _matrix(V)
    if {dta, dtv} != {WLR_F32} or {mema, memv} != {WLR_MEM_DEVICE}:
        raise ValueError("A and V must be float32 CUDA tensors")
    m, n = A.shape
    _net_check(_lib.wlr_ws_loss(net, pa, lda, int(m), int(n), int(k), _dev_f32(Omega_c, "Omega_c"), int(r),
                                pv, ldv, loss.data_ptr(), _dev_f32(dOmega_c, "dOmega_c")), net)


def wlr_ws_backward(net, dOmega):
    _net_check(_lib.wlr_ws_backward(net, _dev_f32(dOmega, "dOmega")), net)


def wlr_ws_adam(net, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0):
    _net_check(_lib.wlr_ws_adam(net, float(lr), float(beta1), float(beta2), float(eps),
                                float(grad_scale)), net)


def wlr_ws_launches(net):
    return int(_lib.wlr_ws_launches(net))


def wlr_get_basis(h, V):
    """Orthonormal basis (m x r float32 CUDA tensor, column-major) of span(X1, X1 C + D)."""
    p, ld, dt, mem, _ = _matrix(V)
    if dt != WLR_F32 or mem != WLR_MEM_DEVICE:
        raise ValueError("V must be a float32 CUDA tensor")
    _check(_lib.wlr_get_basis(h, p, ld), h)


def wlr_set_init_learned(h, net, H, W, fallback=False):
    """X1_0 from the network; with fallback, the start with the lower FP64 objective among
    it and A1.  Returns True when the network's start is used."""
    used = ct.c_int32(0)
    _check(_lib.wlr_set_init_learned(h, net, int(H), int(W), 1 if fallback else 0, ct.byref(used)), h)
    return bool(used.value)


class WarmStartNet:
    """Owner of one warm-start network (destroyed with the object)."""

    def __init__(self, h=30, w=40, c1=16, c2=32, hidden=384, r_max=64, max_frames=4096, seed=0,
                 stream=None):
        # by default the network works on torch's current stream, so its kernels are
        # ordered with the torch operations that make its inputs and read its outputs
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        self.shape = (h, w, c1, c2, hidden, r_max)
        self.h, self.w, self.r_max = h, w, r_max
        self.net = wlr_ws_create(h, w, c1, c2, hidden, r_max, max_frames, seed, stream)

    def params(self):
        return wlr_ws_get_params(self.net)

    def grads(self):
        return wlr_ws_get_grads(self.net)

    def set_params(self, p):
        wlr_ws_set_params(self.net, p)

    def prepare(self, A, W1, H, W, k, X):
        wlr_ws_prepare(self.net, A, W1, H, W, k, X)

    def forward(self, X, clip_start, Omega):
        wlr_ws_forward(self.net, X, clip_start, Omega)

    def loss(self, A, k, Omega_c, r, V, loss, dOmega_c):
        wlr_ws_loss(self.net, A, k, Omega_c, r, V, loss, dOmega_c)

    def backward(self, dOmega):
        wlr_ws_backward(self.net, dOmega)

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0):
        wlr_ws_adam(self.net, lr, beta1, beta2, eps, grad_scale)

    def launches(self):
        return wlr_ws_launches(self.net)

    def close(self):
        if getattr(self, "net", None):
            wlr_ws_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Convenience owner of one handle (destroyed with the object)."""

    def __init__(self, m, n, k, r, precision=WLR_PREC_FP32, stop=WLR_STOP_RELATIVE,
                 eig_block=0, eig_iters=0, eig_iters_cold=0, use_graph=1, seed=None, stream=None,
                 autotune=0):
        o = wlr_default_options()
        o.precision, o.stop = precision, stop
        o.autotune = autotune
        o.eig_block, o.eig_iters, o.eig_iters_cold, o.use_graph = eig_block, eig_iters, eig_iters_cold, use_graph
        if seed is not None:
            o.seed = seed
        self.m, self.n, self.k, self.r = int(m), int(n), int(k), int(r)
        self.h = wlr_create(m, n, k, r, o, stream)

    def set_data(self, A, W1):
        self._data = (A, W1)  # borrowed device buffers must outlive the handle's use
        return wlr_set_data(self.h, A, W1)

    def set_init(self, kind=WLR_INIT_A1, X1_0=None, seed=0):
        return wlr_set_init(self.h, kind, X1_0, seed)

    def set_data_cols(self, A, W1, cols):
        self._data = (A, W1)
        return wlr_set_data_cols(self.h, A, W1, cols)

    def x(self, X):
        return wlr_get_x(self.h, X)

    def step(self, want_objective=True):
        return wlr_step(self.h, want_objective)

    def solve(self, tol=1e-7, max_iter=100):
        return wlr_solve(self.h, tol, max_iter)

    def objective(self):
        return wlr_objective(self.h)

    def result(self, X1=None, X2=None):
        return wlr_get_result(self.h, X1, X2)

    def refine(self, X1_out=None):
        return wlr_refine(self.h, X1_out)

    def basis(self, V):
        return wlr_get_basis(self.h, V)

    def set_init_learned(self, net, H, W, fallback=False):
        return wlr_set_init_learned(self.h, net.net if isinstance(net, WarmStartNet) else net, H, W, fallback)

    def factors(self):
        return wlr_get_factors(self.h, self.k, self.n - self.k, self.r - self.k)

    def history(self):
        return wlr_get_history(self.h)

    def iteration(self):
        return wlr_get_iteration(self.h)

    def get_state(self):
        return wlr_get_state(self.h)

    def set_state(self, state):
        return wlr_set_state(self.h, state)

    def launches(self):
        return wlr_kernel_launches(self.h)

    def profile(self, reps=20):
        return wlr_profile(self.h, reps)

    def close(self):
        if getattr(self, "h", None):
            wlr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
