"""Thin ctypes binding of the C ABI in ``include/qtm.h`` (same function names).

Argument marshalling only: every step of the trajectory method runs in the CUDA
library ``_build/libqtm.so``.  There is no fallback -- if the library cannot be
built or loaded, every call raises.  PyTorch is used for device memory (the
library allocates through the PyTorch caching allocator once
``use_torch_allocator()`` is called) and for the CUDA stream.
"""

from __future__ import annotations

import ctypes as ct
import threading
from typing import Optional

import numpy as np
import scipy.sparse as sp

from . import build as _build

QTM_OK = 0
QTM_ERR_ARG = 1
QTM_ERR_CUDA = 2
QTM_ERR_NOMEM = 3
QTM_ERR_MAXSTEPS = 4
QTM_ERR_STEPSIZE = 5
QTM_ERR_NONFINITE = 6
QTM_ERR_NO_CHANNEL = 7
QTM_ERR_TIMEOUT = 8
QTM_ERR_STATE = 9
QTM_ERR_UNSUPPORTED = 10

QTM_FORMAT_DENSE = 0
QTM_FORMAT_CSR = 1
QTM_PREC_C128 = 0
QTM_PREC_C64 = 1
QTM_PREC_DF64 = 3
QTM_PREC_BF16X6 = 4
QTM_FLAG_RECORD_JUMPS = 1
QTM_METHOD_DOPRI5 = 0
QTM_METHOD_EXPONENTIAL = 1

# every entry point declared in include/qtm.h
EXPORTS = ["qtm_set_allocator", "qtm_create", "qtm_run", "qtm_run_range", "qtm_expect", "qtm_sums",
           "qtm_moments", "qtm_moments_device", "qtm_scale_exponents", "qtm_moments_of_values",
           "qtm_combine_moments", "qtm_arith_peak_launch",
           "qtm_traj_expect", "qtm_jumps", "qtm_stats", "qtm_last_error", "qtm_status_string",
           "qtm_destroy", "qtm_version", "qtm_ensemble_reduce_static", "qtm_run_batch", "qtm_autotune",
           "qtm_set_layout", "qtm_proposal_collect", "qtm_proposal_pairs", "qtm_proposal_train",
           "qtm_proposal_set", "qtm_proposal_get", "qtm_proposal_enable", "qtm_mlp_loss_grad",
           "qtm_rhs_batch", "qtm_set_drive", "qtm_set_wait_limit", "qtm_set_method", "qtm_expo_ladder",
           "qtm_propagator"]

QTM_PROPOSAL_FLOATS = 4685
QTM_MOMENT_WORDS = 9
QTM_PEAK_FP64 = 0
QTM_PEAK_FP32 = 1
QTM_PEAK_DF64 = 2
MLP_PARAMS = 4673


class QtmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class QtmOp(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("format", ct.c_int32), ("row_ptr", ct.POINTER(ct.c_int32)),
                ("col_ind", ct.POINTER(ct.c_int32)), ("values", ct.POINTER(ct.c_double)),
                ("nnz", ct.c_int64)]


class QtmProblem(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("H", QtmOp), ("n_c", ct.c_int32), ("C", ct.POINTER(QtmOp)),
                ("n_obs", ct.c_int32), ("A", ct.POINTER(QtmOp)), ("psi0", ct.POINTER(ct.c_double)),
                ("n_t", ct.c_int32), ("t", ct.POINTER(ct.c_double)), ("rtol", ct.c_double),
                ("atol", ct.c_double), ("precision", ct.c_int32), ("max_steps", ct.c_int64),
                ("flags", ct.c_int32), ("max_jumps_recorded", ct.c_int32)]


class QtmStats(ct.Structure):
    _fields_ = [("trajectories", ct.c_int64), ("accepted", ct.c_int64), ("rejected", ct.c_int64),
                ("rhs_evals", ct.c_int64), ("jumps", ct.c_int64), ("root_iters", ct.c_int64),
                ("failed", ct.c_int64), ("first_error", ct.c_int32), ("kernel_group", ct.c_int32),
                ("kernel_rows", ct.c_int32), ("grid", ct.c_int32), ("block", ct.c_int32),
                ("reserved", ct.c_int32), ("kernel_ms", ct.c_double), ("reduce_ms", ct.c_double),
                ("proposal_misses", ct.c_int64), ("product_ms", ct.c_double)]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)

_lib = None
_lock = threading.Lock()
_keep_alive = []


def lib():
    """Builds (if sources changed) and loads libqtm.so; raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ct.CDLL(path)
            L.qtm_create.argtypes = [ct.POINTER(QtmProblem), ct.c_void_p, ct.POINTER(ct.c_void_p)]
            L.qtm_run.argtypes = [ct.c_void_p, ct.c_int64, ct.c_uint64]
            L.qtm_run_range.argtypes = [ct.c_void_p, ct.c_int64, ct.c_int64, ct.c_uint64]
            L.qtm_expect.argtypes = [ct.c_void_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
            L.qtm_sums.argtypes = [ct.c_void_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                   ct.POINTER(ct.c_int64)]
            i64p = ct.POINTER(ct.c_int64)
            i32p = ct.POINTER(ct.c_int32)
            L.qtm_moments.argtypes = [ct.c_void_p, i64p, i64p, i32p]
            L.qtm_arith_peak_launch.argtypes = [ct.c_int32, ct.c_int64, ct.c_void_p, ct.c_void_p,
                                                ct.POINTER(ct.c_double)]
            L.qtm_moments_device.argtypes = [ct.c_void_p, ct.c_void_p]
            L.qtm_scale_exponents.argtypes = [ct.POINTER(QtmProblem), i32p]
            L.qtm_moments_of_values.argtypes = [ct.POINTER(ct.c_double), ct.c_int64, ct.c_int32, ct.c_int32, i32p,
                                                i64p]
            L.qtm_combine_moments.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, i32p, i64p, i64p,
                                              ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                              ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
            L.qtm_traj_expect.argtypes = [ct.c_void_p, ct.POINTER(ct.c_double)]
            L.qtm_jumps.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_double),
                                    ct.POINTER(ct.c_int32)]
            L.qtm_stats.argtypes = [ct.c_void_p, ct.POINTER(QtmStats)]
            L.qtm_last_error.argtypes = [ct.c_void_p]
            L.qtm_last_error.restype = ct.c_char_p
            L.qtm_status_string.argtypes = [ct.c_int]
            L.qtm_status_string.restype = ct.c_char_p
            L.qtm_destroy.argtypes = [ct.c_void_p]
            L.qtm_destroy.restype = None
            L.qtm_version.restype = ct.c_char_p
            L.qtm_set_allocator.argtypes = [ALLOC_FN, FREE_FN, ct.c_void_p]
            L.qtm_ensemble_reduce_static.argtypes = [ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_void_p,
                                                     ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
            L.qtm_ensemble_reduce_static.restype = ct.c_int
            L.qtm_run_batch.argtypes = [ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                        ct.c_int32, ct.c_uint64]
            L.qtm_run_batch.restype = ct.c_int
            L.qtm_autotune.argtypes = [ct.c_void_p, ct.c_int64, ct.c_uint64, ct.POINTER(ct.c_int32),
                                       ct.POINTER(ct.c_int32)]
            L.qtm_autotune.restype = ct.c_int
            L.qtm_set_layout.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32]
            L.qtm_set_layout.restype = ct.c_int
            fp = ct.POINTER(ct.c_float)
            L.qtm_proposal_collect.argtypes = [ct.c_void_p, ct.c_int64, ct.c_uint64, ct.c_int32, ct.c_int32,
                                               ct.POINTER(ct.c_int64)]
            L.qtm_proposal_pairs.argtypes = [ct.c_void_p, fp, fp, ct.c_int64]
            L.qtm_proposal_train.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_float, ct.c_uint64, fp, fp]
            L.qtm_proposal_set.argtypes = [ct.c_void_p, fp]
            L.qtm_proposal_get.argtypes = [ct.c_void_p, fp]
            L.qtm_proposal_enable.argtypes = [ct.c_void_p, ct.c_int32, ct.c_float]
            L.qtm_mlp_loss_grad.argtypes = [fp, fp, fp, ct.c_int64, fp, fp]
            dp = ct.POINTER(ct.c_double)
            L.qtm_rhs_batch.argtypes = [ct.c_void_p, ct.c_int64, dp, dp]
            L.qtm_rhs_batch.restype = ct.c_int
            L.qtm_set_drive.argtypes = [ct.c_void_p, ct.c_int32, ct.POINTER(QtmOp), dp]
            L.qtm_set_drive.restype = ct.c_int
            L.qtm_set_wait_limit.argtypes = [ct.c_void_p, ct.c_uint64]
            L.qtm_set_wait_limit.restype = ct.c_int
            L.qtm_set_method.argtypes = [ct.c_void_p, ct.c_int32]
            L.qtm_set_method.restype = ct.c_int
            L.qtm_expo_ladder.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int32), dp]
            L.qtm_expo_ladder.restype = ct.c_int
            L.qtm_propagator.argtypes = [ct.POINTER(QtmProblem), ct.c_double, dp]
            L.qtm_propagator.restype = ct.c_int
            for name in ("qtm_proposal_collect", "qtm_proposal_pairs", "qtm_proposal_train", "qtm_proposal_set",
                         "qtm_proposal_get", "qtm_proposal_enable", "qtm_mlp_loss_grad"):
                getattr(L, name).restype = ct.c_int
            for name in ("qtm_create", "qtm_run", "qtm_run_range", "qtm_expect", "qtm_sums", "qtm_moments",
                         "qtm_moments_device", "qtm_scale_exponents", "qtm_moments_of_values",
                         "qtm_combine_moments", "qtm_arith_peak_launch",
                         "qtm_traj_expect", "qtm_jumps", "qtm_stats", "qtm_set_allocator"):
                getattr(L, name).restype = ct.c_int
            _lib = L
        return _lib


def _status_name(status: int) -> str:
    try:
        return lib().qtm_status_string(int(status)).decode()
    except Exception:  # pragma: no cover - only when the library itself is unusable
        return f"status {status}"


def qtm_version() -> str:
    return lib().qtm_version().decode()


def qtm_status_string(status: int) -> str:
    return _status_name(status)


def qtm_last_error(ctx: Optional["Ctx"] = None) -> str:
    return lib().qtm_last_error(ctx.handle if ctx is not None else None).decode()


def _check(status: int, ctx=None):
    if status != QTM_OK:
        raise QtmError(status, qtm_last_error(ctx))


def use_torch_allocator():
    """Routes the library's device allocations through the PyTorch caching allocator."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    cb = (ALLOC_FN(_alloc), FREE_FN(_free))
    _keep_alive.append(cb)
    _check(lib().qtm_set_allocator(cb[0], cb[1], None))


def use_default_allocator():
    _check(lib().qtm_set_allocator(ALLOC_FN(), FREE_FN(), None))


def current_stream():
    """The current PyTorch CUDA stream as a raw cudaStream_t (int)."""
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class Ctx:
    """A library context plus the shapes needed to size host output arrays."""

    def __init__(self, handle, n_t, n_obs, max_jumps):
        self.handle = handle
        self.n_t = n_t
        self.n_obs = n_obs
        self.max_jumps = max_jumps
        self.last_ntraj = None

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                qtm_destroy(self)
            except Exception:
                pass


def _op(m, dense: bool, keep: list) -> QtmOp:
    op = QtmOp()
    n = int(m.shape[0])
    op.n = n
    if dense:
        d = np.ascontiguousarray(m.toarray() if hasattr(m, "toarray") else m, dtype=np.complex128)
        v = d.view(np.float64).ravel()
        keep.append(v)
        op.format = QTM_FORMAT_DENSE
        op.values = v.ctypes.data_as(ct.POINTER(ct.c_double))
        op.nnz = 0
        return op
    m = m.tocsr()
    rp = np.ascontiguousarray(m.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(m.indices, dtype=np.int32)
    v = np.ascontiguousarray(m.data, dtype=np.complex128).view(np.float64)
    keep += [rp, ci, v]
    op.format = QTM_FORMAT_CSR
    op.row_ptr = rp.ctypes.data_as(ct.POINTER(ct.c_int32))
    op.col_ind = ci.ctypes.data_as(ct.POINTER(ct.c_int32))
    op.values = v.ctypes.data_as(ct.POINTER(ct.c_double))
    op.nnz = int(m.nnz)
    return op


def make_problem(prob, precision: int = QTM_PREC_C128, record_jumps: int = 0):
    """Marshals a problem object (H, C, A, psi0, t, rtol, atol, max_steps, dense)."""
    keep = []
    dense = bool(getattr(prob, "dense", False))
    p = QtmProblem()
    p.dim = int(prob.H.shape[0])
    p.H = _op(prob.H, dense, keep)
    cs = [_op(c, dense, keep) for c in prob.C]
    as_ = [_op(a, dense, keep) for a in prob.A]
    carr = (QtmOp * max(1, len(cs)))(*cs)
    aarr = (QtmOp * max(1, len(as_)))(*as_)
    keep += [carr, aarr]
    p.n_c = len(cs)
    p.C = ct.cast(carr, ct.POINTER(QtmOp))
    p.n_obs = len(as_)
    p.A = ct.cast(aarr, ct.POINTER(QtmOp))
    psi = np.ascontiguousarray(np.asarray(prob.psi0, dtype=np.complex128)).view(np.float64)
    t = np.ascontiguousarray(np.asarray(prob.t, dtype=np.float64))
    keep += [psi, t]
    p.psi0 = psi.ctypes.data_as(ct.POINTER(ct.c_double))
    p.n_t = len(t)
    p.t = t.ctypes.data_as(ct.POINTER(ct.c_double))
    p.rtol = float(prob.rtol)
    p.atol = float(prob.atol)
    p.precision = int(precision)
    p.max_steps = int(getattr(prob, "max_steps", 1_000_000))
    p.flags = QTM_FLAG_RECORD_JUMPS if record_jumps else 0
    p.max_jumps_recorded = int(record_jumps)
    return p, keep


def qtm_create(prob, stream=None, precision: int = QTM_PREC_C128, record_jumps: int = 0) -> Ctx:
    p, keep = make_problem(prob, precision, record_jumps)
    h = ct.c_void_p()
    _check(lib().qtm_create(ct.byref(p), ct.c_void_p(stream or 0), ct.byref(h)))
    ctx = Ctx(h.value, len(prob.t), len(prob.A), int(record_jumps))
    drive = list(getattr(prob, "drive", []) or [])
    if drive:
        try:
            qtm_set_drive(ctx, drive)
        except QtmError:
            qtm_destroy(ctx)
            raise
    return ctx


def qtm_run(ctx: Ctx, ntraj: int, seed: int):
    _check(lib().qtm_run(ctx.handle, int(ntraj), int(seed)), ctx)
    ctx.last_ntraj = int(ntraj)


def qtm_run_range(ctx: Ctx, first: int, ntraj: int, seed: int):
    _check(lib().qtm_run_range(ctx.handle, int(first), int(ntraj), int(seed)), ctx)
    ctx.last_ntraj = int(ntraj)


def qtm_run_batch(ctxs, ntrajs, seed: int, firsts=None):
    """Runs several contexts' ensembles in one CUDA graph (see qtm.h)."""
    arr = (ct.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    nt = (ct.c_int64 * len(ctxs))(*[int(x) for x in ntrajs])
    fs = (ct.c_int64 * len(ctxs))(*[int(x) for x in firsts]) if firsts is not None else None
    _check(lib().qtm_run_batch(arr, fs, nt, len(ctxs), int(seed)), ctxs[0])
    for c, n in zip(ctxs, ntrajs):
        c.last_ntraj = int(n)


def qtm_autotune(ctx: Ctx, sample: int, seed: int = 1):
    """Times the available lane layouts on `sample` trajectories and keeps the fastest;
    returns (threads per trajectory, rows per thread)."""
    g = ct.c_int32()
    r = ct.c_int32()
    _check(lib().qtm_autotune(ctx.handle, int(sample), int(seed), ct.byref(g), ct.byref(r)), ctx)
    return g.value, r.value


def qtm_set_layout(ctx: Ctx, group: int, rows: int):
    _check(lib().qtm_set_layout(ctx.handle, int(group), int(rows)), ctx)


def _fp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_float))


def qtm_proposal_collect(ctx: Ctx, ntraj: int, seed: int, stride: int = 16, max_per_traj: int = 64) -> int:
    n = ct.c_int64()
    _check(lib().qtm_proposal_collect(ctx.handle, int(ntraj), int(seed), int(stride), int(max_per_traj),
                                      ct.byref(n)), ctx)
    ctx.last_ntraj = int(ntraj)
    return n.value


def qtm_proposal_pairs(ctx: Ctx, capacity: int):
    f = np.zeros((capacity, 6), np.float32)
    dt = np.zeros(capacity, np.float32)
    _check(lib().qtm_proposal_pairs(ctx.handle, _fp(f), _fp(dt), int(capacity)), ctx)
    return f, dt


def qtm_proposal_train(ctx: Ctx, steps: int = 2000, batch: int = 4096, lr: float = 2e-3, seed: int = 11):
    """Trains the proposal network on the collected pairs; returns (loss, loss of the
    constant-rate estimate alone)."""
    loss = ct.c_float()
    base = ct.c_float()
    _check(lib().qtm_proposal_train(ctx.handle, int(steps), int(batch), float(lr), int(seed), ct.byref(loss),
                                    ct.byref(base)), ctx)
    return loss.value, base.value


def qtm_proposal_set(ctx: Ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == QTM_PROPOSAL_FLOATS
    _check(lib().qtm_proposal_set(ctx.handle, _fp(p)), ctx)


def qtm_proposal_get(ctx: Ctx):
    p = np.zeros(QTM_PROPOSAL_FLOATS, np.float32)
    _check(lib().qtm_proposal_get(ctx.handle, _fp(p)), ctx)
    return p


def qtm_proposal_enable(ctx: Ctx, on: bool = True, margin: float = 0.05):
    _check(lib().qtm_proposal_enable(ctx.handle, int(bool(on)), float(margin)), ctx)


def qtm_mlp_loss_grad(params, x, t):
    """(loss, gradient) of the training kernels for standardised inputs x[n][6], targets t[n]."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, np.float32)
    loss = np.zeros(1, np.float32)
    _check(lib().qtm_mlp_loss_grad(_fp(p), _fp(x), _fp(t), len(t), _fp(loss), _fp(g)))
    return float(loss[0]), g


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def qtm_expect(ctx: Ctx, check: bool = True):
    """(mean, stderr), each of shape (n_t, n_obs)."""
    mean = np.zeros((ctx.n_t, ctx.n_obs))
    se = np.zeros((ctx.n_t, ctx.n_obs))
    st = lib().qtm_expect(ctx.handle, _dp(mean), _dp(se))
    if check:
        _check(st, ctx)
    return mean, se


def qtm_sums(ctx: Ctx):
    s = np.zeros((ctx.n_t, ctx.n_obs))
    s2 = np.zeros((ctx.n_t, ctx.n_obs))
    n = ct.c_int64()
    _check(lib().qtm_sums(ctx.handle, _dp(s), _dp(s2), ct.byref(n)), ctx)
    return s, s2, n.value


def _i64p(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_int32))


def qtm_moments(ctx: Ctx):
    """(words [n_t * n_obs, QTM_MOMENT_WORDS] int64, trajectory count, scale exponents [n_obs])."""
    w = np.zeros((ctx.n_t * ctx.n_obs, QTM_MOMENT_WORDS), np.int64)
    n = ct.c_int64()
    e = np.zeros(max(1, ctx.n_obs), np.int32)
    _check(lib().qtm_moments(ctx.handle, _i64p(w), ct.byref(n), _i32p(e)), ctx)
    return w, n.value, e[:ctx.n_obs]


def qtm_arith_peak_launch(kind: int, iters: int, scratch_dev_ptr: int, stream: int = 0) -> float:
    """Launches one arithmetic-peak probe kernel on `stream`; returns its flop count."""
    f = ct.c_double()
    _check(lib().qtm_arith_peak_launch(int(kind), int(iters), ct.c_void_p(scratch_dev_ptr), ct.c_void_p(stream or 0),
                                       ct.byref(f)))
    return f.value


def qtm_moments_device(ctx: Ctx, words_dev_ptr: int):
    """Asynchronous copy of the run's moment words into a caller-owned device buffer."""
    _check(lib().qtm_moments_device(ctx.handle, ct.c_void_p(words_dev_ptr)), ctx)


def qtm_scale_exponents(prob) -> np.ndarray:
    """Scale exponents of the problem's observables (host only, no GPU)."""
    p, keep = make_problem(prob)
    e = np.zeros(max(1, len(prob.A)), np.int32)
    _check(lib().qtm_scale_exponents(ct.byref(p), _i32p(e)))
    return e[:len(prob.A)]


def qtm_moments_of_values(values, n_obs: int, scale_exp) -> np.ndarray:
    """Moment words of host values [ntraj, n_t, n_obs] (or [ntraj, n_t * n_obs]); no GPU."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    ntraj = v.shape[0]
    P = int(np.prod(v.shape[1:])) if v.ndim > 1 else 0
    e = np.ascontiguousarray(scale_exp, dtype=np.int32)
    w = np.zeros((P, QTM_MOMENT_WORDS), np.int64)
    _check(lib().qtm_moments_of_values(_dp(v), int(ntraj), int(P), int(n_obs), _i32p(e), _i64p(w)))
    return w


def qtm_combine_moments(words, counts, n_obs: int, scale_exp):
    """(mean, stderr, sum, sumsq), each [n_values], of shards' moment words
    [n_shards, n_values, QTM_MOMENT_WORDS] with counts [n_shards]; no GPU."""
    w = np.ascontiguousarray(words, dtype=np.int64)
    if w.ndim == 2:
        w = w[None]
    c = np.ascontiguousarray(np.atleast_1d(counts), dtype=np.int64)
    e = np.ascontiguousarray(scale_exp, dtype=np.int32)
    P = w.shape[1]
    out = [np.zeros(P) for _ in range(4)]
    _check(lib().qtm_combine_moments(int(w.shape[0]), int(P), int(n_obs), _i32p(e), _i64p(w), _i64p(c),
                                     *[_dp(o) for o in out]))
    return tuple(out)


def qtm_traj_expect(ctx: Ctx, check: bool = True):
    out = np.zeros((ctx.last_ntraj or 0, ctx.n_t, ctx.n_obs))
    st = lib().qtm_traj_expect(ctx.handle, _dp(out))
    if check:
        _check(st, ctx)
    return out


def qtm_jumps(ctx: Ctx):
    nt = ctx.last_ntraj or 0
    nj = np.zeros(nt, np.int32)
    jt = np.zeros((nt, max(1, ctx.max_jumps)))
    jc = np.zeros((nt, max(1, ctx.max_jumps)), np.int32)
    _check(lib().qtm_jumps(ctx.handle, nj.ctypes.data_as(ct.POINTER(ct.c_int32)), _dp(jt),
                           jc.ctypes.data_as(ct.POINTER(ct.c_int32))), ctx)
    return nj, jt, jc


def qtm_stats(ctx: Ctx) -> dict:
    s = QtmStats()
    _check(lib().qtm_stats(ctx.handle, ct.byref(s)), ctx)
    return {name: getattr(s, name) for name, _ in QtmStats._fields_}


def qtm_ensemble_reduce_static(values_dev: int, ntraj: int, n_values: int, sum_dev: int, sumsq_dev: int,
                               mean_dev: int, stderr_dev: int, stream: int = 0):
    """Mean / standard error of device-resident per-trajectory values with no device
    allocation (scratch is a fixed 4 MiB array inside the library; see qtm.h).
    All pointers are raw device addresses; the call is asynchronous on ``stream``."""
    _check(lib().qtm_ensemble_reduce_static(ct.c_void_p(values_dev), int(ntraj), int(n_values),
                                            ct.c_void_p(sum_dev), ct.c_void_p(sumsq_dev),
                                            ct.c_void_p(mean_dev), ct.c_void_p(stderr_dev),
                                            ct.c_void_p(stream or 0)))


def qtm_set_drive(ctx: Ctx, terms):
    """Time-dependent terms [(H_k, a_k, omega_k, phi_k), ...]: H(t) = H + sum a_k cos(omega_k t + phi_k) H_k."""
    keep = []
    ops = []
    for Hk, _, _, _ in terms:
        m = sp.csr_matrix(Hk)
        rp = np.ascontiguousarray(m.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(m.indices, dtype=np.int32)
        v = np.ascontiguousarray(m.data, dtype=np.complex128).view(np.float64)
        keep += [rp, ci, v]
        ops.append(QtmOp(int(m.shape[0]), QTM_FORMAT_CSR, rp.ctypes.data_as(ct.POINTER(ct.c_int32)),
                         ci.ctypes.data_as(ct.POINTER(ct.c_int32)), v.ctypes.data_as(ct.POINTER(ct.c_double)),
                         int(m.nnz)))
    arr = (QtmOp * max(1, len(ops)))(*ops)
    coef = np.ascontiguousarray([[float(a), float(w), float(ph)] for _, a, w, ph in terms] or [[0.0, 0.0, 0.0]],
                                dtype=np.float64)
    _check(lib().qtm_set_drive(ctx.handle, len(ops), arr, coef.ctypes.data_as(ct.POINTER(ct.c_double))), ctx)


def qtm_set_wait_limit(ctx: Ctx, limit_ns: int):
    """Bound of one device wait of the tensor-core engine (0: the default 2 s)."""
    _check(lib().qtm_set_wait_limit(ctx.handle, int(limit_ns)), ctx)


def qtm_rhs_batch(ctx: Ctx, y) -> np.ndarray:
    """M y for a batch of vectors y [n_vec][dim] (complex) through the tensor-core product."""
    y = np.ascontiguousarray(np.atleast_2d(y), dtype=np.complex128)
    out = np.empty_like(y)
    dp = ct.POINTER(ct.c_double)
    _check(lib().qtm_rhs_batch(ctx.handle, y.shape[0], y.ctypes.data_as(dp), out.ctypes.data_as(dp)), ctx)
    return out


def qtm_set_method(ctx: Ctx, method: int):
    """QTM_METHOD_DOPRI5 (default) or QTM_METHOD_EXPONENTIAL (exact propagation between jumps)."""
    _check(lib().qtm_set_method(ctx.handle, int(method)), ctx)


def qtm_expo_ladder(ctx: Ctx):
    """(levels, delta) of the exponential method's propagator ladder."""
    lv = ct.c_int32()
    d = ct.c_double()
    _check(lib().qtm_expo_ladder(ctx.handle, ct.byref(lv), ct.byref(d)), ctx)
    return lv.value, d.value


def qtm_propagator(prob, dt: float) -> np.ndarray:
    """exp(M dt) of the problem's effective operator, computed on the host (no GPU)."""
    p, keep = make_problem(prob)
    n = p.dim
    out = np.zeros((n, n), np.complex128)
    _check(lib().qtm_propagator(ct.byref(p), float(dt), out.view(np.float64).ctypes.data_as(ct.POINTER(ct.c_double))))
    return out


def qtm_destroy(ctx: Ctx):
    if ctx.handle:
        lib().qtm_destroy(ctx.handle)
        ctx.handle = None
