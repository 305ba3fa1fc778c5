"""Thin ctypes binding of libmhe.so (include/mhe.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch supplies device memory and the current CUDA stream.  The functions
keep the C names (mhe_create, mhe_factor, mhe_solve, mhe_factor_solve,
mhe_destroy, mhe_assemble, mhe_workspace_bytes); `Solver` wraps them.
If libmhe.so cannot be loaded the call raises: there is no other path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhe.so")
# MHE_BOUNDS_CHECK=1: the bounds-checked debug build (build.build(bounds_check=True))
if os.environ.get("MHE_BOUNDS_CHECK") == "1":
    LIB_PATH = os.path.join(HERE, "libmhe_bounds.so")

MHE_FP64 = 0
MHE_FP32_IR = 1
MHE_TF32_IR = 2
MHE_BF16_IR = 3
MHE_IP_PREDICTOR_CORRECTOR = 0
MHE_IP_PATH_FOLLOWING = 1

STATUS = {0: "MHE_OK", 1: "MHE_PENDING", -1: "MHE_E_ARG", -2: "MHE_E_NOMEM", -3: "MHE_E_NOT_PD",
          -4: "MHE_E_NONFINITE", -5: "MHE_E_NOT_FACTORED", -6: "MHE_E_NO_CONVERGE",
          -7: "MHE_E_TIMEOUT", -8: "MHE_E_CUDA", -9: "MHE_E_ADMISSION", -10: "MHE_E_BOUNDS"}

c_int, c_double, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong


class mhe_dims(ctypes.Structure):
    _fields_ = [("nx", c_int), ("nw", c_int), ("batch", c_int), ("N", ctypes.POINTER(c_int)),
                ("prec", c_int), ("leaf_len", c_int), ("branching", c_int), ("top_len", c_int),
                ("refine_tol", c_double), ("max_refine", c_int), ("fp64_masters", c_int), ("down_pass", c_int),
                ("team", c_int)]


class mhe_matrices(ctypes.Structure):
    _fields_ = [("A", c_void_p), ("B", c_void_p), ("Q", c_void_p), ("P0inv", c_void_p)]


class mhe_rhs(ctypes.Structure):
    _fields_ = [("l", c_void_p), ("a", c_void_p), ("x0", c_void_p)]


class mhe_problem(ctypes.Structure):
    _fields_ = [("ny", c_int), ("A", c_void_p), ("B", c_void_p), ("C", c_void_p), ("R", c_void_p),
                ("a", c_void_p), ("yt", c_void_p), ("wt", c_void_p), ("x0", c_void_p), ("P0inv", c_void_p)]


class mhe_ip_opts(ctypes.Structure):
    _fields_ = [("w_lo", c_void_p), ("w_hi", c_void_p), ("mu0", c_double), ("mu_final", c_double),
                ("max_newton", c_int), ("method", c_int)]


class mhe_info(ctypes.Structure):
    _fields_ = [("status", c_int), ("level", c_int), ("chunk", c_int), ("stage", c_int),
                ("refine_iters", c_int), ("pad", c_int), ("relres", c_double), ("est_relerr", c_double)]


INFO_DTYPE = np.dtype([("status", np.int32), ("level", np.int32), ("chunk", np.int32),
                       ("stage", np.int32), ("refine_iters", np.int32), ("pad", np.int32),
                       ("relres", np.float64), ("est_relerr", np.float64)])

_lib = None
_lock = threading.Lock()


def _declare(L):
    P = ctypes.POINTER
    L.mhe_create.argtypes = [P(mhe_dims), c_void_p, P(c_void_p)]
    L.mhe_create.restype = c_int
    L.mhe_workspace_bytes.argtypes = [P(mhe_dims)]
    L.mhe_workspace_bytes.restype = ctypes.c_size_t
    L.mhe_factor.argtypes = [c_void_p, P(mhe_matrices)]
    L.mhe_factor.restype = c_int
    L.mhe_solve.argtypes = [c_void_p, P(mhe_rhs), c_void_p, c_void_p, c_void_p, c_void_p]
    L.mhe_solve.restype = c_int
    L.mhe_factor_solve.argtypes = [c_void_p, P(mhe_matrices), P(mhe_rhs), c_void_p, c_void_p,
                                   c_void_p, c_void_p]
    L.mhe_factor_solve.restype = c_int
    L.mhe_estimate.argtypes = [c_void_p, P(mhe_problem), c_void_p, c_void_p, c_void_p, c_void_p]
    L.mhe_estimate.restype = c_int
    L.mhe_estimate_host.argtypes = [c_void_p, P(mhe_problem), c_void_p, c_void_p, c_void_p, c_void_p, c_int]
    L.mhe_estimate_host.restype = c_int
    L.mhe_destroy.argtypes = [c_void_p]
    L.mhe_destroy.restype = c_int
    L.mhe_assemble.argtypes = [c_int, c_int, c_int, c_ll, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p]
    L.mhe_assemble.restype = c_int
    L.mhe_shapes.argtypes = [P(c_int), P(c_int), c_int]
    L.mhe_shapes.restype = c_int
    L.mhe_shape_teams.argtypes = [c_int, c_int, P(c_int), c_int]
    L.mhe_shape_teams.restype = c_int
    L.mhe_timing_enable.argtypes = [c_void_p, c_int]
    L.mhe_timing_enable.restype = c_int
    L.mhe_timing_read.argtypes = [c_void_p, ctypes.POINTER(c_double), c_int]
    L.mhe_timing_read.restype = c_int
    L.mhe_plan_info.argtypes = [c_void_p, ctypes.POINTER(c_ll), c_int]
    L.mhe_plan_info.restype = c_int
    L.mhe_launch_count.argtypes = [c_void_p]
    L.mhe_launch_count.restype = c_ll
    L.mhe_assemble_count.argtypes = []
    L.mhe_assemble_count.restype = c_ll
    L.mhe_estimate_host_async.argtypes = L.mhe_estimate_host.argtypes
    L.mhe_estimate_host_async.restype = c_int
    L.mhe_estimate_host_wait.argtypes = [c_void_p]
    L.mhe_estimate_host_wait.restype = c_int
    L.mhe_pipe_timeline.argtypes = [c_void_p, P(c_double), c_int]
    L.mhe_pipe_timeline.restype = c_int
    L.mhe_set_host_in_place.argtypes = [c_void_p, c_int]
    L.mhe_set_host_in_place.restype = c_int
    L.mhe_set_graph.argtypes = [c_void_p, c_int]
    L.mhe_set_graph.restype = c_int
    L.mhe_ip_solve.argtypes = [c_void_p, P(mhe_matrices), P(mhe_rhs), P(mhe_ip_opts), c_void_p, c_void_p, c_void_p,
                               c_void_p, P(c_int)]
    L.mhe_ip_solve.restype = c_int
    L.mhe_rts_workspace_bytes.argtypes = [c_int, c_int, c_int, c_int, P(c_int)]
    L.mhe_rts_workspace_bytes.restype = ctypes.c_size_t
    L.mhe_rts_smooth.argtypes = [c_int, c_int, c_int, c_int, P(c_int)] + [c_void_p] * 12 + [ctypes.c_size_t,
                                                                                            c_void_p, c_void_p]
    L.mhe_rts_smooth.restype = c_int
    L.mhe_set_double_float_residual.argtypes = [c_void_p, c_int]
    L.mhe_set_double_float_residual.restype = c_int
    L.mhe_debug_set_tc_wait_limit.argtypes = [c_int]
    L.mhe_debug_set_tc_wait_limit.restype = c_int
    L.mhe_solve_serial_noalloc.argtypes = [c_int, c_int, c_int] + [c_void_p] * 12
    L.mhe_solve_serial_noalloc.restype = c_int
    L.mhe_autotune.argtypes = [P(mhe_dims), P(mhe_matrices), P(mhe_rhs), c_void_p, c_int, P(mhe_dims),
                               P(c_double)]
    L.mhe_autotune.restype = c_int
    L.mhe_server_create.argtypes = [ctypes.c_size_t, c_int, c_double, c_int, P(c_void_p)]
    L.mhe_server_create.restype = c_int
    L.mhe_estimator_open.argtypes = [c_void_p, c_int, c_int, c_int, c_int] + [c_void_p] * 9 + [P(c_int)]
    L.mhe_estimator_open.restype = c_int
    L.mhe_submit.argtypes = [c_void_p, c_int, c_void_p, P(ctypes.c_ulonglong)]
    L.mhe_submit.restype = c_int
    L.mhe_poll.argtypes = [c_void_p, ctypes.c_ulonglong, c_void_p, P(mhe_info), P(c_double)]
    L.mhe_poll.restype = c_int
    L.mhe_server_set_plan.argtypes = [c_void_p, c_int, c_int, c_int]
    L.mhe_server_set_plan.restype = c_int
    L.mhe_server_used_bytes.argtypes = [c_void_p]
    L.mhe_server_used_bytes.restype = ctypes.c_size_t
    L.mhe_server_set_reuse.argtypes = [c_void_p, c_int]
    L.mhe_server_set_reuse.restype = c_int
    L.mhe_server_stats.argtypes = [c_void_p, ctypes.POINTER(c_ll), c_int]
    L.mhe_server_stats.restype = c_int
    L.mhe_server_destroy.argtypes = [c_void_p]
    L.mhe_server_destroy.restype = c_int
    L.mhe_last_error.argtypes = []
    L.mhe_last_error.restype = ctypes.c_char_p
    return L


def lib():
    """Load libmhe.so (raises if it is missing: build it with build.py)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_1510_03110_gb300/build.py")
            _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


class MheError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().mhe_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, where):
    if rc != 0:
        raise MheError(rc, where)
    return rc


def _ptr(t):
    if t is None:
        return None
    import torch
    # checked always (not by assert): a host pointer handed to the kernels would fault the GPU
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def shapes():
    L = lib()
    nx = (c_int * 64)()
    nw = (c_int * 64)()
    k = L.mhe_shapes(nx, nw, 64)
    return [(nx[i], nw[i]) for i in range(k)]


def shape_teams(nx, nw):
    """Team widths compiled for (nx, nw), the default first (mhe_shape_teams)."""
    t = (c_int * 16)()
    k = lib().mhe_shape_teams(int(nx), int(nw), t, 16)
    return [t[i] for i in range(min(k, 16))]


def make_dims(nx, nw, N, prec=MHE_FP64, leaf_len=0, branching=0, top_len=0, refine_tol=0.0,
              max_refine=-1, fp64_masters=False, down_pass=0, team=0):
    N = np.ascontiguousarray(np.asarray(N, dtype=np.int32).reshape(-1))
    d = mhe_dims(int(nx), int(nw), int(N.size), N.ctypes.data_as(ctypes.POINTER(c_int)), int(prec),
                 int(leaf_len), int(branching), int(top_len), float(refine_tol), int(max_refine),
                 int(bool(fp64_masters)), int(down_pass), int(team))
    return d, N


def mhe_create(dims, stream=None):
    ctx = c_void_p()
    _check(lib().mhe_create(ctypes.byref(dims), _stream(stream), ctypes.byref(ctx)), "mhe_create")
    return ctx


def mhe_workspace_bytes(dims):
    return int(lib().mhe_workspace_bytes(ctypes.byref(dims)))


def mhe_factor(ctx, A, B, Q, P0inv):
    m = mhe_matrices(_ptr(A), _ptr(B), _ptr(Q), _ptr(P0inv))
    return _check(lib().mhe_factor(ctx, ctypes.byref(m)), "mhe_factor")


def mhe_solve(ctx, l, a, x0, x, w, lam, info=None):
    r = mhe_rhs(_ptr(l), _ptr(a), _ptr(x0))
    ip = ctypes.c_void_p(info.data_ptr()) if info is not None else None
    return _check(lib().mhe_solve(ctx, ctypes.byref(r), _ptr(x), _ptr(w), _ptr(lam), ip), "mhe_solve")


def mhe_factor_solve(ctx, A, B, Q, P0inv, l, a, x0, x, w, lam, info=None):
    m = mhe_matrices(_ptr(A), _ptr(B), _ptr(Q), _ptr(P0inv))
    r = mhe_rhs(_ptr(l), _ptr(a), _ptr(x0))
    ip = ctypes.c_void_p(info.data_ptr()) if info is not None else None
    return _check(lib().mhe_factor_solve(ctx, ctypes.byref(m), ctypes.byref(r), _ptr(x), _ptr(w),
                                         _ptr(lam), ip), "mhe_factor_solve")


def mhe_estimate(ctx, ny, A, B, C, R, a, yt, wt, x0, P0inv, x, w, lam, info=None):
    p = mhe_problem(int(ny), _ptr(A), _ptr(B), _ptr(C), _ptr(R), _ptr(a), _ptr(yt), _ptr(wt), _ptr(x0),
                    _ptr(P0inv))
    ip = ctypes.c_void_p(info.data_ptr()) if info is not None else None
    return _check(lib().mhe_estimate(ctx, ctypes.byref(p), _ptr(x), _ptr(w), _ptr(lam), ip), "mhe_estimate")


def _hptr(t):
    """Host array (contiguous float64 numpy array or CPU torch tensor) -> pointer."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not (t.dtype == np.float64 and t.flags["C_CONTIGUOUS"]):
            raise TypeError("expected a contiguous float64 array")
        return ctypes.c_void_p(t.ctypes.data)
    import torch
    if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CPU tensor or numpy array")
    return ctypes.c_void_p(t.data_ptr())


def _host_args(ny, A, B, C, R, a, yt, wt, x0, P0inv, info):
    p = mhe_problem(int(ny), _hptr(A), _hptr(B), _hptr(C), _hptr(R), _hptr(a), _hptr(yt), _hptr(wt), _hptr(x0),
                    _hptr(P0inv))
    if info is None:
        ip = None
    elif isinstance(info, np.ndarray):
        ip = ctypes.c_void_p(info.ctypes.data)
    else:
        ip = ctypes.c_void_p(info.data_ptr())
    return p, ip


def mhe_estimate_host(ctx, ny, A, B, C, R, a, yt, wt, x0, P0inv, x, w, lam, info=None, pieces=8):
    """mhe_estimate_host: problem and outputs in host memory (pinned for overlap)."""
    p, ip = _host_args(ny, A, B, C, R, a, yt, wt, x0, P0inv, info)
    return _check(lib().mhe_estimate_host(ctx, ctypes.byref(p), _hptr(x), _hptr(w), _hptr(lam), ip, int(pieces)),
                  "mhe_estimate_host")


def mhe_estimate_host_async(ctx, ny, A, B, C, R, a, yt, wt, x0, P0inv, x, w, lam, info=None, pieces=8):
    """mhe_estimate_host_async: issue the host pipeline and return; mhe_estimate_host_wait completes it."""
    p, ip = _host_args(ny, A, B, C, R, a, yt, wt, x0, P0inv, info)
    return _check(lib().mhe_estimate_host_async(ctx, ctypes.byref(p), _hptr(x), _hptr(w), _hptr(lam), ip,
                                                int(pieces)), "mhe_estimate_host_async")


def mhe_estimate_host_wait(ctx):
    return _check(lib().mhe_estimate_host_wait(ctx), "mhe_estimate_host_wait")


def mhe_destroy(ctx):
    return _check(lib().mhe_destroy(ctx), "mhe_destroy")


PHASES = {0: "reduce", 1: "rhs", 2: "down", 3: "resid", 4: "prep"}


def mhe_timing_enable(ctx, enable=True):
    return _check(lib().mhe_timing_enable(ctx, int(bool(enable))), "mhe_timing_enable")


def mhe_timing_read(ctx):
    """[(phase name, level, passes, total ms, longest pass ms)] since the last read (synchronises)."""
    buf = (c_double * 5120)()
    k = lib().mhe_timing_read(ctx, buf, 1024)
    if k < 0:
        raise MheError(k, "mhe_timing_read")
    return [(PHASES[int(buf[5 * i])], int(buf[5 * i + 1]), int(buf[5 * i + 2]), float(buf[5 * i + 3]),
             float(buf[5 * i + 4])) for i in range(min(k, 1024))]


def _iptr(t):
    """A device int32 buffer of at least one element (a status word) -> pointer;
    None passes as NULL.  Checked always: the kernel writes through it, so a host
    pointer or a tensor of another type would fault the GPU."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()
            and t.numel() >= 1):
        raise TypeError("status must be None or a contiguous int32 CUDA tensor of at least one element")
    return ctypes.c_void_p(t.data_ptr())


def mhe_solve_serial_noalloc(nx, nw, N, A, B, Q, P0inv, l, a, x0, x, w, lam, status=None,
                             stream=None):
    """One instance, serial plan, FP64, no device allocation (fixed library scratch).

    Every array is checked against the layout of include/mhe.h for batch = 1
    (S = N - 1 caller stages) before the call: the library takes raw pointers
    and cannot check their extents."""
    nx, nw, N = int(nx), int(nw), int(N)
    S, nq = max(N - 1, 0), nx + nw
    for t, count, name in ((A, S * nx * nx, "A"), (B, S * nx * nw, "B"), (Q, S * nq * nq, "Q"),
                           (l, S * nq, "l"), (a, S * nx, "a"), (P0inv, nx * nx, "P0inv"), (x0, nx, "x0"),
                           (x, (N + 1) * nx, "x"), (w, nx + S * nw, "w"), (lam, (N + 1) * nx, "lam")):
        _need(t, count, name)
    sp = _iptr(status)
    return _check(lib().mhe_solve_serial_noalloc(nx, nw, N, _ptr(A), _ptr(B), _ptr(Q),
                                                 _ptr(P0inv), _ptr(l), _ptr(a), _ptr(x0), _ptr(x), _ptr(w),
                                                 _ptr(lam), sp, _stream(stream)),
                  "mhe_solve_serial_noalloc")


def mhe_autotune(dims, A, B, Q, P0inv, l, a, x0, reps=2, stream=None):
    """Fastest plan (leaf_len, branching, top_len) for this problem and its time in ms."""
    m = mhe_matrices(_ptr(A), _ptr(B), _ptr(Q), _ptr(P0inv))
    r = mhe_rhs(_ptr(l), _ptr(a), _ptr(x0))
    best = mhe_dims()
    ms = c_double()
    _check(lib().mhe_autotune(ctypes.byref(dims), ctypes.byref(m), ctypes.byref(r), _stream(stream), int(reps),
                              ctypes.byref(best), ctypes.byref(ms)), "mhe_autotune")
    return dict(leaf_len=best.leaf_len, branching=best.branching, top_len=best.top_len, down_pass=best.down_pass,
                team=best.team, ms=ms.value)


def mhe_pipe_timeline(ctx, cap=256):
    """mhe_pipe_timeline: per piece (engine, b0, b1, host issue ms, inputs issued, inputs arrived, solved,
    outputs back) of the last mhe_estimate_host call made with timing enabled."""
    out = (c_double * (8 * cap))()
    k = lib().mhe_pipe_timeline(ctx, out, cap)
    if k < 0:
        raise MheError(k, "mhe_pipe_timeline")
    return [tuple(out[8 * i:8 * i + 8]) for i in range(min(k, cap))]


def mhe_launch_count(ctx):
    return int(lib().mhe_launch_count(ctx))


def mhe_assemble_count():
    return int(lib().mhe_assemble_count())


def mhe_rts_smooth(nx, nw, ny, N, A, B, C, R, a, yt, wt, x0, P0inv, x, w, work=None, status=None, stream=None):
    """Kalman filter + RTS smoother on the GPU (S = 0 models): the x, w of the MHE Newton step.
    Every array is checked against the batch layout; work (uint8 CUDA tensor) is allocated when None."""
    import torch
    N = np.ascontiguousarray(np.asarray(N, dtype=np.int32).reshape(-1))
    batch = int(N.size)
    S = int(np.sum(N - 1))
    X = int(np.sum(N + 1))
    W = int(np.sum(nx + (N - 1) * nw))
    for t, count, name in ((A, S * nx * nx, "A"), (B, S * nx * nw, "B"), (C, S * ny * nx, "C"),
                           (R, S * (nw + ny) ** 2, "R"), (a, S * nx, "a"), (yt, S * ny, "yt"), (wt, S * nw, "wt"),
                           (x0, batch * nx, "x0"), (P0inv, batch * nx * nx, "P0inv"), (x, X * nx, "x"), (w, W, "w")):
        _need(t, count, name)
    nbytes = int(lib().mhe_rts_workspace_bytes(int(nx), int(nw), int(ny), batch,
                                               N.ctypes.data_as(ctypes.POINTER(c_int))))
    if nbytes == 0:
        raise SizeError("no RTS smoother for this shape, or a horizon below 2")
    if work is None:
        work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    if not (isinstance(work, torch.Tensor) and work.is_cuda and work.numel() * work.element_size() >= nbytes):
        raise TypeError(f"work must be a CUDA tensor of at least {nbytes} bytes")
    sp = _iptr(status) if status is not None else None
    if status is not None:
        _need(status, batch, "status")
    return _check(lib().mhe_rts_smooth(int(nx), int(nw), int(ny), batch, N.ctypes.data_as(ctypes.POINTER(c_int)),
                                       _ptr(A), _ptr(B), _ptr(C), _ptr(R), _ptr(a), _ptr(yt), _ptr(wt), _ptr(x0),
                                       _ptr(P0inv), _ptr(x), _ptr(w), ctypes.c_void_p(work.data_ptr()),
                                       ctypes.c_size_t(nbytes), sp, _stream(stream)), "mhe_rts_smooth")


def mhe_set_double_float_residual(ctx, on=True):
    """The mixed-precision MHE-form residual in double-float (True, default) or FP64 arithmetic."""
    return _check(lib().mhe_set_double_float_residual(ctx, int(bool(on))), "mhe_set_double_float_residual")


def mhe_debug_set_tc_wait_limit(tries):
    """Tries of the tensor-core product waits (< 0: the default); a test of the timeout path."""
    return _check(lib().mhe_debug_set_tc_wait_limit(int(tries)), "mhe_debug_set_tc_wait_limit")


def mhe_plan_info(ctx):
    """[(level, chunks, stages)] of the planned tree."""
    buf = (c_ll * (3 * 256))()     # 3 long longs per level, up to 256 levels
    k = lib().mhe_plan_info(ctx, buf, 256)
    return [(int(buf[3 * i]), int(buf[3 * i + 1]), int(buf[3 * i + 2])) for i in range(min(k, 256))]


def mhe_assemble(nx, nw, ny, C, R, yt, wt, Q, l, c=None, stream=None):
    """Step a0 for S stages; C is (S, ny * nx) (one column-major block per row),
    which fixes S."""
    if C is not None and (C.dim() != 2 or C.shape[1] != ny * nx):
        raise SizeError(f"C must be (S, ny * nx) = (S, {ny * nx}), got {tuple(C.shape)}")
    S = C.shape[0] if C is not None else 0
    nq = nx + nw
    for t, count, name in ((R, S * (nw + ny) ** 2, "R"), (yt, S * ny, "yt"), (wt, S * nw, "wt"),
                           (Q, S * nq * nq, "Q"), (l, S * nq, "l"), (c, S if c is not None else 0, "c")):
        _need(t, count, name)
    return _check(lib().mhe_assemble(int(nx), int(nw), int(ny), int(S), _ptr(C), _ptr(R), _ptr(yt),
                                     _ptr(wt), _ptr(Q), _ptr(l), _ptr(c), _stream(stream)),
                  "mhe_assemble")


def info_array(t):
    """Device/host byte tensor of mhe_info records -> numpy structured array."""
    return t.cpu().numpy().view(INFO_DTYPE)


class SizeError(MheError, ValueError):
    """An argument array shorter than the problem's layout needs (MHE_E_ARG,
    raised by the binding before the call)."""

    def __init__(self, msg):
        RuntimeError.__init__(self, f"MHE_E_ARG: {msg}")
        self.code = -1


def _need(t, count, name):
    """Raise SizeError unless tensor/array t holds at least `count` elements (the
    library takes raw pointers and cannot check: a short buffer would be read or
    written past its end on the GPU).  None is left to the library, which reports
    a NULL pointer as MHE_E_ARG."""
    if t is None:
        return
    have = int(t.numel()) if hasattr(t, "numel") else int(np.asarray(t).size)
    if have < count:
        raise SizeError(f"{name} holds {have} elements; this problem needs {count}")


def check_sizes(nx, nw, S, batch, X, W, ny=None, **arrays):
    """Element counts of the batch's arrays against the layout of include/mhe.h:
    S caller stages, batch instances, X states (sum of N_b + 1), W inputs
    (sum of nx + (N_b - 1) nw); ny for the MHE-form arrays C, R, yt, wt."""
    nq = nx + nw
    need = dict(A=S * nx * nx, B=S * nx * nw, Q=S * nq * nq, P0inv=batch * nx * nx, l=S * nq, a=S * nx,
                x0=batch * nx, x=X * nx, w=W, lam=X * nx)
    if ny is not None:
        need.update(C=S * ny * nx, R=S * (nw + ny) ** 2, yt=S * ny, wt=S * nw)
    for name, t in arrays.items():
        _need(t, need[name], name)


class Solver:
    """One context: dims fixed at construction, tensors passed per call.

    Output sizes: x and lam (sum_b (N_b + 1), nx); w sum_b (nx + (N_b - 1) nw).
    """

    def __init__(self, nx, nw, N, prec=MHE_FP64, leaf_len=0, branching=0, top_len=0,
                 refine_tol=0.0, max_refine=-1, stream=None, fp64_masters=False, down_pass=0, team=0):
        import torch
        self.nx, self.nw = int(nx), int(nw)
        self.N = np.asarray(N, dtype=np.int64).reshape(-1)
        self.batch = int(self.N.size)
        self.dims, self._N32 = make_dims(nx, nw, self.N, prec, leaf_len, branching, top_len,
                                         refine_tol, max_refine, fp64_masters, down_pass, team)
        self.stream = stream
        self.ctx = mhe_create(self.dims, stream)
        self.X = int(np.sum(self.N + 1))
        self.W = int(np.sum(self.nx + (self.N - 1) * self.nw))
        self.S = int(np.sum(self.N - 1))
        self.info = torch.zeros(self.batch * INFO_DTYPE.itemsize, dtype=torch.uint8, device="cuda")

    def outputs(self):
        import torch
        x = torch.empty(self.X, self.nx, dtype=torch.float64, device="cuda")
        w = torch.empty(max(1, self.W), dtype=torch.float64, device="cuda")
        lam = torch.empty(self.X, self.nx, dtype=torch.float64, device="cuda")
        return x, w, lam

    def _sizes(self, ny=None, **arrays):
        check_sizes(self.nx, self.nw, self.S, self.batch, self.X, self.W, ny, **arrays)

    def factor(self, A, B, Q, P0inv):
        self._sizes(A=A, B=B, Q=Q, P0inv=P0inv)
        mhe_factor(self.ctx, A, B, Q, P0inv)

    def solve(self, l, a, x0, out=None):
        x, w, lam = out if out is not None else self.outputs()
        self._sizes(l=l, a=a, x0=x0, x=x, w=w, lam=lam)
        mhe_solve(self.ctx, l, a, x0, x, w, lam, self.info)
        return x, w, lam

    def factor_solve(self, A, B, Q, P0inv, l, a, x0, out=None):
        x, w, lam = out if out is not None else self.outputs()
        self._sizes(A=A, B=B, Q=Q, P0inv=P0inv, l=l, a=a, x0=x0, x=x, w=w, lam=lam)
        mhe_factor_solve(self.ctx, A, B, Q, P0inv, l, a, x0, x, w, lam, self.info)
        return x, w, lam

    def estimate(self, ny, A, B, C, R, a, yt, wt, x0, P0inv, out=None):
        """Steps a0..a7 from MHE data (mhe_estimate)."""
        x, w, lam = out if out is not None else self.outputs()
        self._sizes(ny, A=A, B=B, C=C, R=R, a=a, yt=yt, wt=wt, x0=x0, P0inv=P0inv, x=x, w=w, lam=lam)
        mhe_estimate(self.ctx, ny, A, B, C, R, a, yt, wt, x0, P0inv, x, w, lam, self.info)
        return x, w, lam

    def set_host_in_place(self, on=True):
        """mhe_set_host_in_place: mhe_estimate_host reads pinned host inputs in place (no copies)."""
        _check(lib().mhe_set_host_in_place(self.ctx, int(bool(on))), "mhe_set_host_in_place")

    def set_graph(self, on=True):
        """mhe_set_graph: replay each entry point's launch sequence as a CUDA graph."""
        _check(lib().mhe_set_graph(self.ctx, int(bool(on))), "mhe_set_graph")

    def ip_solve(self, A, B, Q, P0inv, l, a, x0, w_lo, w_hi, mu0=0.0, mu_final=0.0, max_newton=0, out=None,
                 method=0):
        """mhe_ip_solve: bounds w_lo <= w_t <= w_hi ([batch][nw] each) by a primal-dual interior-point loop whose
        Newton steps are this context's factor + solve (method MHE_IP_PREDICTOR_CORRECTOR or
        MHE_IP_PATH_FOLLOWING).  Returns (x, w, lam, iterations)."""
        x, w, lam = out if out is not None else self.outputs()
        self._sizes(A=A, B=B, Q=Q, P0inv=P0inv, l=l, a=a, x0=x0, x=x, w=w, lam=lam)
        _need(w_lo, self.batch * self.nw, "w_lo")
        _need(w_hi, self.batch * self.nw, "w_hi")
        m = mhe_matrices(_ptr(A), _ptr(B), _ptr(Q), _ptr(P0inv))
        r = mhe_rhs(_ptr(l), _ptr(a), _ptr(x0))
        o = mhe_ip_opts(_ptr(w_lo), _ptr(w_hi), float(mu0), float(mu_final), int(max_newton), int(method))
        steps = c_int()
        _check(lib().mhe_ip_solve(self.ctx, ctypes.byref(m), ctypes.byref(r), ctypes.byref(o), _ptr(x), _ptr(w),
                                  _ptr(lam), ctypes.c_void_p(self.info.data_ptr()), ctypes.byref(steps)),
               "mhe_ip_solve")
        return x, w, lam, steps.value

    def infos(self):
        return info_array(self.info)

    def close(self):
        if self.ctx is not None:
            mhe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving -------------------------------------------------------------------

def pack_stage(A, B, C, R, a, yt, wt):
    """One MHE stage (math orientation) -> the packed host layout of mhe_submit."""
    cm = lambda M: np.ascontiguousarray(np.asarray(M, np.float64).T).reshape(-1)  # noqa: E731
    return np.concatenate([cm(A), cm(B), cm(C), cm(R), np.asarray(a, np.float64).reshape(-1),
                           np.asarray(yt, np.float64).reshape(-1), np.asarray(wt, np.float64).reshape(-1)])


class Server:
    """Continuous-batching server of receding-horizon MHE estimators (C-ABI mhe_server_*)."""

    def __init__(self, device_bytes, prec=MHE_FP32_IR, refine_tol=0.0, max_refine=-1):
        self.s = c_void_p()
        _check(lib().mhe_server_create(int(device_bytes), int(prec), float(refine_tol), int(max_refine),
                                       ctypes.byref(self.s)), "mhe_server_create")
        self.nx = {}
        self.stage_len = {}   # doubles of one packed stage, per estimator

    def open(self, p):
        """Admit an estimator whose initial window is the N-1 stages of p (mhe_instance format)."""
        cm = lambda X: np.ascontiguousarray(np.swapaxes(np.asarray(X, np.float64), -1, -2))  # noqa: E731
        arrs = [cm(p["A"]), cm(p["B"]), cm(p["C"]), cm(p["R"]), np.ascontiguousarray(p["a"], np.float64),
                np.ascontiguousarray(p["yt"], np.float64), np.ascontiguousarray(p["wt"], np.float64),
                np.ascontiguousarray(p["x0"], np.float64), cm(p["P0inv"])]
        n, m, q, S = int(p["n"]), int(p["m"]), int(p["q"]), int(p["N"]) - 1
        for arr, name, count in zip(arrs, ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv"),
                                    (S * n * n, S * n * m, S * q * n, S * (m + q) ** 2, S * n, S * q, S * m,
                                     n, n * n)):
            _need(arr, count, name)
        ptrs = [a.ctypes.data_as(c_void_p) for a in arrs]
        eid = c_int()
        _check(lib().mhe_estimator_open(self.s, n, m, q, int(p["N"]), *ptrs,
                                        ctypes.byref(eid)), "mhe_estimator_open")
        self.nx[eid.value] = n
        self.stage_len[eid.value] = n * n + n * m + q * n + (m + q) ** 2 + n + q + m
        return eid.value

    def submit(self, est, packed):
        if int(est) in self.stage_len:
            packed = np.ascontiguousarray(packed, dtype=np.float64)
            _need(packed, self.stage_len[int(est)], "packed stage")
        t = ctypes.c_ulonglong()
        _check(lib().mhe_submit(self.s, int(est), packed.ctypes.data_as(c_void_p), ctypes.byref(t)), "mhe_submit")
        return t.value

    def poll(self, ticket, nx):
        x = np.zeros(nx)
        info = mhe_info()
        lat = c_double()
        rc = lib().mhe_poll(self.s, ctypes.c_ulonglong(ticket), x.ctypes.data_as(c_void_p), ctypes.byref(info),
                            ctypes.byref(lat))
        if rc == 1:
            return None
        if rc not in (0, -6):
            raise MheError(rc, "mhe_poll")
        return dict(x=x, status=rc, relres=info.relres, iters=info.refine_iters, latency=lat.value)

    def wait(self, ticket, nx, timeout=60.0):
        import time
        t0 = time.time()
        while True:
            r = self.poll(ticket, nx)
            if r is not None:
                return r
            if time.time() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} not served within {timeout} s")
            time.sleep(0.0002)

    def set_plan(self, leaf_len=0, branching=0, top_len=0):
        _check(lib().mhe_server_set_plan(self.s, int(leaf_len), int(branching), int(top_len)), "mhe_server_set_plan")

    def used_bytes(self):
        return int(lib().mhe_server_used_bytes(self.s))

    def set_reuse(self, on=True):
        _check(lib().mhe_server_set_reuse(self.s, int(bool(on))), "mhe_server_set_reuse")

    def stats(self):
        """{rounds, requests, stages_reduced, stages_solved} since the server was created."""
        buf = (c_ll * 4)()
        k = lib().mhe_server_stats(self.s, buf, 4)
        if k < 0:
            raise MheError(k, "mhe_server_stats")
        return dict(rounds=int(buf[0]), requests=int(buf[1]), stages_reduced=int(buf[2]),
                    stages_solved=int(buf[3]))

    def close(self):
        if self.s:
            lib().mhe_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
