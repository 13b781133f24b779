"""Python binding of libgbfit's C ABI (argument marshalling only).

Every step of a fit runs in the CUDA library; this module converts Python
arguments to the C call and the outputs back.  It never falls back to a CPU
path: if libgbfit.so is missing or no GPU is present the call raises.

Data arrays may be torch tensors (CUDA or CPU) or NumPy arrays; CUDA tensors
are read in place, host arrays are copied to the device inside the call.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from .build import LIB

# ---- constants mirrored from include/gbfit.h
OK = 0
E_INVALID_ARG, E_INFEASIBLE_X0, E_OOM, E_BUDGET, E_CUDA, E_TIMEOUT, E_UNSUPPORTED, E_CANCELLED = -1, -2, -3, -4, -5, -6, -7, -8
MODEL_GAUSS1D, MODEL_DEXP, MODEL_GAUSS2D, MODEL_POLY2 = 0, 1, 2, 3
X_VEC, X_SOA2, X_GRID = 0, 1, 2
F32, F64 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
FIT_INVALID_DATA, FIT_NUMERICAL, FIT_MAX_NFEV, FIT_GTOL, FIT_FTOL, FIT_XTOL, FIT_FTOL_XTOL = -2, -1, 0, 1, 2, 3, 4
N_PARAMS = {0: 4, 1: 5, 2: 7, 3: 3}     # user-defined models are added by register_model
USER_MODEL_BASE = 100

EXPORTS = ["gbfit_version", "gbfit_last_error", "gbfit_default_options", "gbfit_model_info",
           "gbfit_curve_fit", "gbfit_curve_fit_batch", "gbfit_evaluate", "gbfit_tr_subproblem",
           "gbfit_stats_reset", "gbfit_stats_get", "gbfit_set_profiling", "gbfit_evaluate_noalloc",
           "gbfit_server_create", "gbfit_server_submit", "gbfit_server_step", "gbfit_server_poll",
           "gbfit_server_destroy", "gbfit_tune_get", "gbfit_tune_set", "gbfit_tune_shape", "gbfit_autotune",
           "gbfit_model_register", "gbfit_model_log", "gbfit_curve_fit_cov", "gbfit_evaluate_cov",
           "gbfit_check_rcp64", "gbfit_server_cancel", "gbfit_server_snapshot", "gbfit_server_submit_resume"]


class GbfitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gbfit error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("ftol", ctypes.c_double), ("xtol", ctypes.c_double), ("gtol", ctypes.c_double),
                ("max_nfev", ctypes.c_int), ("x_scale_jac", ctypes.c_int),
                ("x_scale", ctypes.POINTER(ctypes.c_double)), ("absolute_sigma", ctypes.c_int),
                ("precision", ctypes.c_int), ("tile_points", ctypes.c_int), ("group_tiles", ctypes.c_int),
                ("loss", ctypes.c_int), ("reserved", ctypes.c_int * 1), ("f_scale", ctypes.c_double),
                ("guard_cond", ctypes.c_double), ("guard_floor", ctypes.c_double), ("wait_limit_s", ctypes.c_double)]

LOSSES = {"linear": 0, "soft_l1": 1, "huber": 2, "cauchy": 3, "arctan": 4}

TUNE_BUCKETS = 32


class TuneTable(ctypes.Structure):
    _fields_ = [("tile_points", ctypes.c_int32 * TUNE_BUCKETS * 2 * 4),
                ("group_tiles", ctypes.c_int32 * TUNE_BUCKETS * 2 * 4)]


class Stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("fits", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("graph_rounds", ctypes.c_int64), ("passes", ctypes.c_int64), ("point_passes", ctypes.c_double),
                ("eval_ms", ctypes.c_double), ("eval_launches", ctypes.c_int64),
                ("phase_cycles", ctypes.c_double * 32), ("host_ms", ctypes.c_double),
                ("loop_busy_ms", ctypes.c_double), ("loop_wait_ms", ctypes.c_double), ("loop_ctas", ctypes.c_int64)]

PHASES = ["tile", "combine", "logic", "eigen", "comb_fence", "step", "prep", "finish", "comb_group", "comb_final",
          "eig_warm", "eig_j32", "eig_ns", "eig_rr", "j32_sweeps", "refine_passes", "gn_path", "n_gn", "n_eig",
          "n_alg2_iters", "n_bounded_nonfull", "pre_tile", "tile_loop", "ring_wait",
          "round_ns", "owner_wait_ns", "barrier_ns", "start_ns", "n_eval64", "n_guard_escalated",
          "n_guard_finished", "n_wide"]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("rounds_per_step", ctypes.c_int), ("reserved", ctypes.c_int * 4),
                ("guard_cond", ctypes.c_double), ("guard_floor", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("model_id", ctypes.c_int), ("x_layout", ctypes.c_int), ("dtype", ctypes.c_int),
                ("has_bounds", ctypes.c_int), ("m", ctypes.c_int64), ("grid_w", ctypes.c_int64),
                ("grid_h", ctypes.c_int64), ("xdata", ctypes.c_void_p), ("ydata", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("p0", ctypes.c_double * 8), ("lb", ctypes.c_double * 8),
                ("ub", ctypes.c_double * 8), ("ftol", ctypes.c_double), ("xtol", ctypes.c_double),
                ("gtol", ctypes.c_double), ("max_nfev", ctypes.c_int), ("tag", ctypes.c_uint64),
                ("loss", ctypes.c_int), ("f_scale", ctypes.c_double)]


SNAPSHOT_STATE_BYTES = 2048


class Snapshot(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("state_bytes", ctypes.c_uint32), ("model_id", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("m", ctypes.c_int64), ("reserved", ctypes.c_int64),
                ("state", ctypes.c_ubyte * SNAPSHOT_STATE_BYTES)]


class ResultRec(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("fit_status", ctypes.c_int), ("nfev", ctypes.c_int), ("n_params", ctypes.c_int),
                ("cost", ctypes.c_double), ("popt", ctypes.c_double * 8), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_LIB = None
_DEFAULT_OPT = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libgbfit.so (built by paper_2208_12187_gb300.build.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libgbfit.so not found at {path}; run paper_2208_12187_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    DP = ctypes.POINTER(ctypes.c_double)
    IP = ctypes.POINTER(ctypes.c_int)
    lib.gbfit_version.restype = I
    lib.gbfit_last_error.restype = ctypes.c_char_p
    lib.gbfit_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.gbfit_model_info.argtypes = [I, IP, IP]
    # the single-fit call takes raw addresses (lowest per-call marshalling cost)
    lib.gbfit_curve_fit.argtypes = [I, P, I64, I, P, P, P, I, P, P, P, P, P, P, P, P, P, P]
    lib.gbfit_curve_fit_batch.argtypes = [I, I, ctypes.POINTER(ctypes.c_int64), P, I, P, P, I, DP, DP, DP,
                                          ctypes.POINTER(Options), DP, DP, DP, IP, IP, P]
    lib.gbfit_evaluate.argtypes = [I, P, I64, I, ctypes.POINTER(ctypes.c_int64), P, P, I, DP, I, I, DP, P]
    lib.gbfit_tr_subproblem.argtypes = [I, DP, DP, D, D, DP, DP, DP, P]
    lib.gbfit_evaluate_noalloc.argtypes = [I, P, I64, I, ctypes.POINTER(ctypes.c_int64), P, P, I, DP, I, I, DP, P]
    lib.gbfit_stats_get.argtypes = [ctypes.POINTER(Stats)]
    lib.gbfit_check_rcp64.argtypes = [P, P, I64, P]
    lib.gbfit_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.gbfit_server_snapshot.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Snapshot)]
    lib.gbfit_server_submit_resume.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(Snapshot),
                                               ctypes.POINTER(ctypes.c_uint64)]
    lib.gbfit_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]
    lib.gbfit_server_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.gbfit_server_step.argtypes = [ctypes.c_void_p, IP, IP]
    lib.gbfit_server_poll.argtypes = [ctypes.c_void_p, ctypes.POINTER(ResultRec), I, IP]
    lib.gbfit_server_destroy.argtypes = [ctypes.c_void_p]
    lib.gbfit_tune_get.argtypes = [ctypes.POINTER(TuneTable)]
    lib.gbfit_tune_set.argtypes = [ctypes.POINTER(TuneTable)]
    lib.gbfit_tune_shape.argtypes = [I, I, I64, IP, IP]
    lib.gbfit_autotune.argtypes = [I, I, I64, I64, ctypes.POINTER(TuneTable), P]
    lib.gbfit_set_profiling.argtypes = [I]
    lib.gbfit_model_register.argtypes = [ctypes.c_char_p, ctypes.c_char_p, I, I, IP]
    lib.gbfit_curve_fit_cov.argtypes = [I, P, I64, I, P, P, P, I, P, P, P, P, P, P, P, P, P, P]
    lib.gbfit_evaluate_cov.argtypes = [I, P, I64, I, P, P, P, I, P, I, P, P]
    lib.gbfit_model_log.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    for name in EXPORTS:
        getattr(lib, name)
    _LIB = lib
    global _DEFAULT_OPT
    o = Options()
    lib.gbfit_default_options(ctypes.byref(o))
    _DEFAULT_OPT = bytes(o)
    return lib


def _check(rc: int):
    if rc != OK:
        raise GbfitError(rc, load().gbfit_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


_NP_CODE = {np.dtype(np.float32): F32, np.dtype(np.float64): F64}
_TORCH = None      # (torch.Tensor, {dtype: code}) once torch is importable


def _torch_types():
    global _TORCH
    if _TORCH is None:
        try:
            import torch
            _TORCH = (torch.Tensor, {torch.float32: F32, torch.float64: F64})
        except ImportError:
            _TORCH = (None, {})
    return _TORCH


def _array_info(a):
    """(address, dtype code, keepalive) for a torch tensor or NumPy array."""
    if a is None:
        return None, None, None
    tt, tcodes = _TORCH or _torch_types()
    if tt is not None and isinstance(a, tt):
        if not a.is_contiguous():
            a = a.contiguous()
        code = tcodes.get(a.dtype)
        if code is None:
            raise TypeError("data tensors must be float32 or float64")
        return a.data_ptr(), code, a
    a = np.ascontiguousarray(a)
    code = _NP_CODE.get(a.dtype)
    if code is None:
        raise TypeError("data arrays must be float32 or float64")
    return a.ctypes.data, code, a


def _cov_info(sigma, m):
    """(address, keepalive) of a 2D sigma (an [m, m] covariance matrix, FP64), else None."""
    shape = getattr(sigma, "shape", None)
    if sigma is None or shape is None or len(shape) != 2:
        return None
    if tuple(shape) != (m, m):
        raise ValueError("a 2D sigma must be the [m, m] covariance matrix")
    tt, _ = _TORCH or _torch_types()
    if tt is not None and isinstance(sigma, tt):
        import torch
        c = sigma.to(torch.float64).contiguous()
        return c.data_ptr(), c
    c = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    return c.ctypes.data, c


_RAW_STREAM = None     # (current_device, current raw stream) functions of torch, once looked up


def _current_stream_int() -> int:
    """torch's current CUDA stream on the current device, as an integer (0 without torch or CUDA)."""
    global _RAW_STREAM
    if _RAW_STREAM is None:
        try:
            import torch
            if not torch.cuda.is_available():
                _RAW_STREAM = False
            elif hasattr(torch._C, "_cuda_getCurrentRawStream"):
                _RAW_STREAM = (torch._C._cuda_getDevice, torch._C._cuda_getCurrentRawStream)
            else:
                _RAW_STREAM = (None, lambda _d: torch.cuda.current_stream().cuda_stream)
        except ImportError:
            _RAW_STREAM = False
    if not _RAW_STREAM:
        return 0
    dev_fn, raw_fn = _RAW_STREAM
    return raw_fn(dev_fn() if dev_fn else 0)


def _stream_int(stream) -> int:
    if stream is None:
        return _current_stream_int()
    v = getattr(stream, "cuda_stream", stream)
    return int(v or 0)


def _stream_ptr(stream):
    return ctypes.c_void_p(_stream_int(stream))


def _options(n, ftol, xtol, gtol, max_nfev, x_scale, absolute_sigma, precision, tile_points, group_tiles=0,
             loss="linear", f_scale=1.0, guard_cond=0.0, guard_floor=0.0, wait_limit_s=0.0):
    load()
    o = Options.from_buffer_copy(_DEFAULT_OPT)
    o.ftol, o.xtol, o.gtol = ftol, xtol, gtol
    o.max_nfev = int(max_nfev or 0)
    keep = None
    if isinstance(x_scale, (int, float)) and x_scale == 1.0:
        pass
    elif isinstance(x_scale, str):
        if x_scale != "jac":
            raise ValueError("x_scale must be 'jac' or positive numbers")
        o.x_scale_jac = 1
    elif x_scale is not None and not (np.isscalar(x_scale) and float(x_scale) == 1.0):
        keep = np.ascontiguousarray(np.broadcast_to(np.asarray(x_scale, dtype=np.float64), (n,)))
        o.x_scale = _dptr(keep)
    o.absolute_sigma = int(bool(absolute_sigma))
    o.precision = _PREC.get(precision, precision) if isinstance(precision, str) else int(precision)
    if isinstance(o.precision, str):
        raise KeyError(precision)
    o.tile_points = int(tile_points)
    o.group_tiles = int(group_tiles)
    o.loss = LOSSES[loss] if isinstance(loss, str) else int(loss)
    o.f_scale = float(f_scale)
    o.guard_cond = float(guard_cond)        # 0: library default; inf: off
    o.guard_floor = float(guard_floor)
    o.wait_limit_s = float(wait_limit_s)    # 0: library default (10 s)
    return o, keep


_PREC = {"fp64": PREC_FP64, "mixed": PREC_MIXED}


_TLS = threading.local()
_OPT_CACHE = {}        # option tuple -> Options (immutable once built)


class _Scratch:
    """Per-thread host buffer for one single-fit call's small arrays: p0, lb,
    ub, grid (W, H), and the outputs popt | pcov | cost | nfev, status.  One
    address lookup per thread instead of one per array per call."""
    P0, LB, UB, GRID, OUT = 0, 8, 16, 24, 32            # offsets in doubles
    INTS = 112                                           # nfev, status (two int32 in one double slot)

    def __init__(self):
        self.buf = (ctypes.c_double * 128)()
        self.base = ctypes.addressof(self.buf)
        self.v = np.frombuffer(self.buf, dtype=np.float64)
        self.i64 = self.v.view(np.int64)
        self.i32 = self.v.view(np.int32)


def _scratch() -> _Scratch:
    sc = getattr(_TLS, "sc", None)
    if sc is None:
        sc = _TLS.sc = _Scratch()
    return sc


def _cached_options(n, ftol, xtol, gtol, max_nfev, x_scale, absolute_sigma, precision, tile_points, group_tiles,
                    loss, f_scale, guard_cond=0.0, guard_floor=0.0, wait_limit_s=0.0):
    """(address of an Options, keepalive); options without an x_scale vector are cached."""
    if isinstance(x_scale, (int, float)) and x_scale == 1.0:
        key = (ftol, xtol, gtol, max_nfev, absolute_sigma, precision, tile_points, group_tiles, loss, f_scale,
               guard_cond, guard_floor, wait_limit_s)
        o = _OPT_CACHE.get(key)
        if o is None:
            o, _ = _options(n, ftol, xtol, gtol, max_nfev, x_scale, absolute_sigma, precision, tile_points,
                            group_tiles, loss, f_scale, guard_cond, guard_floor, wait_limit_s)
            if len(_OPT_CACHE) < 256:
                _OPT_CACHE[key] = o
        return ctypes.addressof(o), o
    o, keep = _options(n, ftol, xtol, gtol, max_nfev, x_scale, absolute_sigma, precision, tile_points, group_tiles,
                       loss, f_scale, guard_cond, guard_floor, wait_limit_s)
    return ctypes.addressof(o), (o, keep)


def _vec(v, n):
    a = np.asarray(v, dtype=np.float64)
    if a.shape != (n,):
        a = np.broadcast_to(a, (n,))
    return np.ascontiguousarray(a)


def _bounds(n, lb, ub):
    lbv = None if lb is None else np.ascontiguousarray(np.broadcast_to(np.asarray(lb, np.float64), (n,)))
    ubv = None if ub is None else np.ascontiguousarray(np.broadcast_to(np.asarray(ub, np.float64), (n,)))
    return lbv, ubv


def register_model(source: str, n_params: int, x_dims: int = 1, func_name: str = "model") -> int:
    """Compile a user-defined model h(x; p) and return its model id (gbfit_model_register).

    source defines ``template <class T, class S> __device__ T <func_name>(const T* p, S x, S x2)``
    in CUDA C++ over the library's dual-number type T (see include/gbfit.h).  Compiling takes
    some seconds (NVRTC); the id works with curve_fit, curve_fit_batch and evaluate."""
    lib = load()
    mid = ctypes.c_int(-1)
    rc = lib.gbfit_model_register(source.encode(), func_name.encode(), int(n_params), int(x_dims), ctypes.byref(mid))
    _check(rc)
    N_PARAMS[mid.value] = int(n_params)
    return mid.value


def model_log() -> str:
    """Compiler log of the last register_model call."""
    lib = load()
    n = ctypes.c_size_t(0)
    lib.gbfit_model_log(None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value + 1)
    lib.gbfit_model_log(buf, n.value + 1, ctypes.byref(n))
    return buf.value.decode(errors="replace")


def curve_fit(model: int, xdata, ydata, p0: Sequence[float], sigma=None, lb=None, ub=None,
              grid_wh=None, ftol=1e-8, xtol=1e-8, gtol=1e-8, max_nfev=None, x_scale=1.0,
              absolute_sigma=False, precision="mixed", tile_points=0, group_tiles=0, loss="linear",
              f_scale=1.0, stream=None, guard_cond=0.0, guard_floor=0.0, wait_limit_s=0.0) -> dict:
    """Fit `model` by the GPU trust-region-reflective method (gbfit_curve_fit).

    xdata: [m] (1D models), [2, m] (2D explicit coordinates) or None with
    grid_wh=(W, H) for the implicit pixel grid.  Returns dict(popt, pcov, cost,
    nfev, status).  guard_cond / guard_floor: the mixed path's precision guard
    (0: library defaults, inf: off; see gbfit_options).
    """
    lib = _LIB or load()
    n = N_PARAMS[model]
    yp, dt, ykeep = _array_info(ydata)
    xp, xdt, xkeep = _array_info(xdata)
    m = int(ykeep.shape[0])
    cov = _cov_info(sigma, m) if sigma is not None else None   # 2D sigma: full covariance (gbfit_curve_fit_cov)
    sp, sdt, skeep = _array_info(None if cov else sigma)
    if xp is not None and xdt != dt or sp is not None and sdt != dt:
        raise TypeError("xdata, ydata and sigma must share one dtype")
    sc = _scratch()
    v, base = sc.v, sc.base
    gwp = None
    if grid_wh is not None:
        layout = X_GRID
        sc.i64[_Scratch.GRID] = int(grid_wh[0])
        sc.i64[_Scratch.GRID + 1] = int(grid_wh[1])
        gwp = base + 8 * _Scratch.GRID
        xp = None
    else:
        layout = X_SOA2 if (xkeep is not None and len(xkeep.shape) == 2) else X_VEC
    v[_Scratch.P0:_Scratch.P0 + n] = p0
    lbp = ubp = None
    if lb is not None:
        v[_Scratch.LB:_Scratch.LB + n] = lb
        lbp = base + 8 * _Scratch.LB
    if ub is not None:
        v[_Scratch.UB:_Scratch.UB + n] = ub
        ubp = base + 8 * _Scratch.UB
    optp, okeep = _cached_options(n, ftol, xtol, gtol, max_nfev, x_scale, absolute_sigma, precision, tile_points,
                                  group_tiles, loss, f_scale, guard_cond, guard_floor, wait_limit_s)
    a = base + 8 * _Scratch.OUT                    # popt | pcov | cost
    ip = base + 8 * _Scratch.INTS                  # nfev | status
    call = lib.gbfit_curve_fit
    if cov:
        call, sp = lib.gbfit_curve_fit_cov, cov[0]
    rc = call(model, xp, m, layout, gwp, yp, sp, dt, base + 8 * _Scratch.P0, lbp, ubp, optp, a, a + 8 * n,
              a + 8 * (n + n * n), ip, ip + 4, _stream_int(stream))
    if rc != OK:
        _check(rc)
    o = v[_Scratch.OUT:_Scratch.OUT + n + n * n + 1].copy()
    ints = sc.i32[2 * _Scratch.INTS:2 * _Scratch.INTS + 2]
    return dict(popt=o[:n], pcov=o[n:n + n * n].reshape(n, n), cost=float(o[-1]), nfev=int(ints[0]),
                status=int(ints[1]))


def curve_fit_batch(model: int, offsets, xdata, ydata, p0, sigma=None, lb=None, ub=None,
                    ftol=1e-8, xtol=1e-8, gtol=1e-8, max_nfev=None, x_scale=1.0,
                    absolute_sigma=False, precision="mixed", tile_points=0, group_tiles=0, loss="linear",
                    f_scale=1.0, stream=None, guard_cond=0.0, guard_floor=0.0, wait_limit_s=0.0) -> dict:
    """Many independent fits over concatenated data (gbfit_curve_fit_batch).
    tile_points / group_tiles 0: each fit's shape from the tile table."""
    lib = load()
    n = N_PARAMS[model]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nf = off.shape[0] - 1
    yp, dt, ykeep = _array_info(ydata)
    xp, xdt, xkeep = _array_info(xdata)
    sp, sdt, skeep = _array_info(sigma)
    layout = X_SOA2 if len(xkeep.shape) == 2 else X_VEC
    p0a = np.ascontiguousarray(np.asarray(p0, dtype=np.float64).reshape(nf, n))
    lba = None if lb is None else np.ascontiguousarray(np.broadcast_to(np.asarray(lb, np.float64), (nf, n)))
    uba = None if ub is None else np.ascontiguousarray(np.broadcast_to(np.asarray(ub, np.float64), (nf, n)))
    opt, okeep = _options(n, ftol, xtol, gtol, max_nfev, x_scale, absolute_sigma, precision, tile_points, group_tiles,
                          loss, f_scale, guard_cond, guard_floor, wait_limit_s)
    popt = np.zeros((nf, n))
    pcov = np.zeros((nf, n, n))
    cost = np.zeros(nf)
    nfev = np.zeros(nf, dtype=np.int32)
    status = np.zeros(nf, dtype=np.int32)
    IP = ctypes.POINTER(ctypes.c_int)
    rc = lib.gbfit_curve_fit_batch(model, nf, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), xp, layout,
                                   yp, sp, dt, _dptr(p0a), None if lba is None else _dptr(lba),
                                   None if uba is None else _dptr(uba), ctypes.byref(opt), _dptr(popt),
                                   _dptr(pcov), _dptr(cost), nfev.ctypes.data_as(IP),
                                   status.ctypes.data_as(IP), _stream_ptr(stream))
    _check(rc)
    return dict(popt=popt, pcov=pcov, cost=cost, nfev=nfev, status=status)


def evaluate(model: int, xdata, ydata, p, sigma=None, grid_wh=None, precision="fp64", tile_points=0,
             stream=None):
    """One fused reduction at p: (B packed upper, g, cost) as FP64 arrays (gbfit_evaluate)."""
    lib = load()
    n = N_PARAMS[model]
    yp, dt, ykeep = _array_info(ydata)
    xp, _, xkeep = _array_info(xdata)
    m = int(ykeep.shape[0])
    cov = _cov_info(sigma, m)
    sp, _, skeep = _array_info(None if cov else sigma)
    if grid_wh is not None:
        layout, gw, xp = X_GRID, (ctypes.c_int64 * 2)(int(grid_wh[0]), int(grid_wh[1])), None
    else:
        layout, gw = (X_SOA2 if len(xkeep.shape) == 2 else X_VEC), None
    pa = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    nt = n * (n + 1) // 2
    out = np.zeros(nt + n + 1)
    prec = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision] if isinstance(precision, str) else int(precision)
    if cov:
        rc = lib.gbfit_evaluate_cov(model, xp, m, layout, None if gw is None else ctypes.addressof(gw), yp, cov[0],
                                    dt, pa.ctypes.data, prec, out.ctypes.data, _stream_ptr(stream))
    else:
        rc = lib.gbfit_evaluate(model, xp, m, layout, gw, yp, sp, dt, _dptr(pa), prec, int(tile_points),
                                _dptr(out), _stream_ptr(stream))
    _check(rc)
    return out[:nt], out[nt:nt + n], float(out[nt + n])


def tr_subproblem(B, g, Delta: float, alpha0: float = 0.0, stream=None):
    """Device solve of one scaled trust-region subproblem: (p, alpha, eigenvalues)."""
    lib = load()
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64))
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
    n = g.shape[0]
    p = np.zeros(n)
    lam = np.zeros(n)
    alpha = ctypes.c_double()
    rc = lib.gbfit_tr_subproblem(n, _dptr(B), _dptr(g), float(Delta), float(alpha0), _dptr(p),
                                 ctypes.byref(alpha), _dptr(lam), _stream_ptr(stream))
    _check(rc)
    return p, alpha.value, lam


def unpack_upper(packed, n):
    """Symmetric n x n matrix from its packed row-major upper triangle."""
    B = np.zeros((n, n))
    k = 0
    for i in range(n):
        for j in range(i, n):
            B[i, j] = B[j, i] = packed[k]
            k += 1
    return B


def check_rcp64(x, stream=None):
    """1/x by the device step's FP64 reciprocal (gbfit_check_rcp64); x: a CUDA
    float64 tensor.  Returns a new tensor."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError("x must be a CUDA float64 tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(load().gbfit_check_rcp64(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    ctypes.c_int64(x.numel()), _stream_ptr(stream)))
    return y


def stats_reset():
    _check(load().gbfit_stats_reset())


def stats() -> dict:
    """Process-wide counters (calls, fits, kernel launches, passes, profiled eval time)."""
    st = Stats()
    _check(load().gbfit_stats_get(ctypes.byref(st)))
    out = {name: getattr(st, name) for name, _ in Stats._fields_ if name != "phase_cycles"}
    out["phase_cycles"] = dict(zip(PHASES, list(st.phase_cycles)))
    return out


def set_profiling(on: bool):
    """CUDA-event timing of every loop-kernel launch (stats()["eval_ms"], ["eval_launches"])."""
    _check(load().gbfit_set_profiling(1 if on else 0))


def evaluate_noalloc(model: int, xdata, ydata, p, sigma=None, grid_wh=None, precision="fp64", tile_points=0,
                     stream=None):
    """Same as evaluate(), through gbfit_evaluate_noalloc: no device or pinned
    allocation at call time (data must already be on the device)."""
    lib = load()
    n = N_PARAMS[model]
    yp, dt, ykeep = _array_info(ydata)
    xp, _, xkeep = _array_info(xdata)
    sp, _, skeep = _array_info(sigma)
    m = int(ykeep.shape[0])
    if grid_wh is not None:
        layout, gw, xp = X_GRID, (ctypes.c_int64 * 2)(int(grid_wh[0]), int(grid_wh[1])), None
    else:
        layout, gw = (X_SOA2 if len(xkeep.shape) == 2 else X_VEC), None
    pa = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    nt = n * (n + 1) // 2
    out = np.zeros(nt + n + 1)
    prec = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision] if isinstance(precision, str) else int(precision)
    rc = lib.gbfit_evaluate_noalloc(model, xp, m, layout, gw, yp, sp, dt, _dptr(pa), prec, int(tile_points),
                                    _dptr(out), _stream_ptr(stream))
    _check(rc)
    return out[:nt], out[nt:nt + n], float(out[nt + n])


def _prec_code(precision):
    return {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision] if isinstance(precision, str) else int(precision)


def tune_get() -> dict:
    """The installed tile table: {"tile_points": int32[4, 2, 32], "group_tiles": ...}
    indexed [model][precision][floor(log2 m)]."""
    t = TuneTable()
    _check(load().gbfit_tune_get(ctypes.byref(t)))
    return {"tile_points": np.ctypeslib.as_array(t.tile_points).copy(),
            "group_tiles": np.ctypeslib.as_array(t.group_tiles).copy()}


def tune_set(table: dict):
    t = TuneTable()
    np.ctypeslib.as_array(t.tile_points)[...] = np.asarray(table["tile_points"], dtype=np.int32)
    np.ctypeslib.as_array(t.group_tiles)[...] = np.asarray(table["group_tiles"], dtype=np.int32)
    _check(load().gbfit_tune_set(ctypes.byref(t)))


def tune_shape(model: int, precision, m: int):
    """(tile_points, group_tiles) a batched or served fit of m points gets."""
    tp, gt = ctypes.c_int(), ctypes.c_int()
    _check(load().gbfit_tune_shape(model, _prec_code(precision), int(m), ctypes.byref(tp), ctypes.byref(gt)))
    return tp.value, gt.value


def autotune(model: int, precision="mixed", m_max: int = 1 << 22, points_per_run: int = 0, stream=None) -> dict:
    """Time candidate tile shapes per size bucket and install the fastest (gbfit_autotune)."""
    t = TuneTable()
    _check(load().gbfit_autotune(model, _prec_code(precision), int(m_max), int(points_per_run), ctypes.byref(t),
                                 _stream_ptr(stream)))
    return {"tile_points": np.ctypeslib.as_array(t.tile_points).copy(),
            "group_tiles": np.ctypeslib.as_array(t.group_tiles).copy()}


class Server:
    """Continuous-batching fit server (gbfit_server_*): submit requests at any
    time, call step() to retire finished fits, admit queued ones and run
    shared iterations, poll() for results."""

    def __init__(self, hbm_budget_bytes=1 << 30, max_slots=4096, precision="mixed", rounds_per_step=4,
                 guard_cond=0.0, guard_floor=0.0):
        lib = load()
        cfg = ServerConfig()
        cfg.guard_cond, cfg.guard_floor = float(guard_cond), float(guard_floor)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_slots = int(max_slots)
        cfg.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision] if isinstance(precision, str) else int(precision)
        cfg.rounds_per_step = int(rounds_per_step)
        h = ctypes.c_void_p()
        _check(lib.gbfit_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, model, xdata, ydata, p0, sigma=None, lb=None, ub=None, grid_wh=None, ftol=1e-8, xtol=1e-8,
               gtol=1e-8, max_nfev=0, tag=0, loss="linear", f_scale=1.0, resume=None) -> int:
        """Queue a request; resume: a Snapshot (from snapshot()) to continue from."""
        n = N_PARAMS[model]
        r = Request()
        yp, dt, yk = _array_info(ydata)
        xp, _, xk = _array_info(xdata)
        sp, _, sk = _array_info(sigma)
        r.model_id, r.dtype, r.m = model, dt, int(yk.shape[0])
        if grid_wh is not None:
            r.x_layout, r.grid_w, r.grid_h, r.xdata = X_GRID, int(grid_wh[0]), int(grid_wh[1]), None
        else:
            r.x_layout = X_SOA2 if len(xk.shape) == 2 else X_VEC
            r.xdata = xp
        r.ydata, r.sigma = yp, sp
        for i in range(n):
            r.p0[i] = float(p0[i])
        if lb is not None or ub is not None:
            r.has_bounds = 1
            lbv, ubv = _bounds(n, -np.inf if lb is None else lb, np.inf if ub is None else ub)
            for i in range(n):
                r.lb[i], r.ub[i] = lbv[i], ubv[i]
        r.ftol, r.xtol, r.gtol, r.max_nfev, r.tag = ftol, xtol, gtol, int(max_nfev), int(tag)
        r.loss = LOSSES[loss] if isinstance(loss, str) else int(loss)
        r.f_scale = float(f_scale)
        t = ctypes.c_uint64()
        if resume is None:
            _check(load().gbfit_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        else:
            _check(load().gbfit_server_submit_resume(self._h, ctypes.byref(r), ctypes.byref(resume), ctypes.byref(t)))
        self._keep[t.value] = (xk, yk, sk)
        return t.value

    def cancel(self, ticket: int):
        """Cancel a queued or resident request (its record is polled with status E_CANCELLED)."""
        _check(load().gbfit_server_cancel(self._h, int(ticket)))

    def snapshot(self, ticket: int) -> "Snapshot":
        """The device state of a resident request (checkpoint), for submit(..., resume=)."""
        snap = Snapshot()
        _check(load().gbfit_server_snapshot(self._h, int(ticket), ctypes.byref(snap)))
        return snap

    def step(self):
        a, q = ctypes.c_int(), ctypes.c_int()
        _check(load().gbfit_server_step(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, max_results=4096):
        buf = (ResultRec * max_results)()
        c = ctypes.c_int()
        _check(load().gbfit_server_poll(self._h, buf, max_results, ctypes.byref(c)))
        out = []
        for k in range(c.value):
            rr = buf[k]
            self._keep.pop(rr.ticket, None)
            out.append(dict(ticket=rr.ticket, tag=rr.tag, status=rr.status, fit_status=rr.fit_status,
                            nfev=rr.nfev, cost=rr.cost, popt=np.array(rr.popt[:rr.n_params]),
                            t_submit=rr.t_submit, t_admit=rr.t_admit, t_done=rr.t_done))
        return out

    def close(self):
        if self._h:
            load().gbfit_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
