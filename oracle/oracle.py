"""ctypes front end of the plain-C FP64 oracle (``qtm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing in the library imports this
module, and this module imports nothing from the library; problems are passed in
as objects with the attributes ``H, C, A`` (scipy CSR matrices), ``psi0``, ``t``,
``rtol``, ``atol`` and ``max_steps`` (the seeded input generators produce them).

Every numerical step happens in C; this file only marshals arrays and computes
the ensemble mean / standard error with numpy (Sec. 3: the final trajectory is
the average of the trajectories).
"""

from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libqtm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C11, no target-specific flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcOp(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("row_ptr", ct.POINTER(ct.c_int32)),
                ("col", ct.POINTER(ct.c_int32)), ("val", ct.POINTER(ct.c_double))]


class OrcProblem(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("H", OrcOp), ("n_c", ct.c_int32), ("C", ct.POINTER(OrcOp)),
                ("n_obs", ct.c_int32), ("A", ct.POINTER(OrcOp)), ("psi0", ct.POINTER(ct.c_double)),
                ("n_t", ct.c_int32), ("t", ct.POINTER(ct.c_double)), ("rtol", ct.c_double),
                ("atol", ct.c_double), ("max_steps", ct.c_int64), ("n_drive", ct.c_int32),
                ("drive", ct.POINTER(OrcOp)), ("drive_coef", ct.POINTER(ct.c_double))]


class OrcResult(ct.Structure):
    _fields_ = [("obs_re", ct.POINTER(ct.c_double)), ("obs_im", ct.POINTER(ct.c_double)),
                ("max_jumps", ct.c_int32), ("n_jumps", ct.POINTER(ct.c_int32)),
                ("jump_t", ct.POINTER(ct.c_double)), ("jump_ch", ct.POINTER(ct.c_int32)),
                ("jump_norm", ct.POINTER(ct.c_double)), ("status", ct.POINTER(ct.c_int32)),
                ("counts", ct.POINTER(ct.c_int64))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ct.CDLL(build())
            _lib.orc_mcwf.restype = ct.c_int
            _lib.orc_mcwf.argtypes = [ct.POINTER(OrcProblem), ct.c_uint64, ct.c_int64, ct.c_int64,
                                      ct.c_int, ct.POINTER(OrcResult)]
            _lib.orc_lindblad.restype = ct.c_int
            _lib.orc_lindblad.argtypes = [ct.POINTER(OrcProblem), ct.c_double, ct.c_double,
                                          ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
            _lib.orc_effective_matrix.restype = ct.c_int
            _lib.orc_effective_matrix.argtypes = [ct.POINTER(OrcProblem), ct.POINTER(ct.c_double)]
            _lib.orc_philox4x64_10.restype = None
            _lib.orc_philox4x64_10.argtypes = [ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_uint64),
                                               ct.POINTER(ct.c_uint64)]
            _lib.orc_uniforms.restype = None
            _lib.orc_uniforms.argtypes = [ct.c_uint64, ct.c_int64, ct.c_int64,
                                          ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
            _lib.orc_dopri5_fixed.restype = ct.c_int
            _lib.orc_dopri5_fixed.argtypes = [ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                              ct.c_double, ct.c_int, ct.c_double,
                                              ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                              ct.POINTER(ct.c_double)]
            _lib.orc_step_trace.restype = ct.c_int
            _lib.orc_step_trace.argtypes = [ct.POINTER(OrcProblem), ct.c_uint64, ct.c_int64, ct.c_int64,
                                            ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]
            _lib.orc_dense_weights.restype = None
            _lib.orc_dense_weights.argtypes = [ct.c_double, ct.POINTER(ct.c_double)]
        return _lib


def _dptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _iptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_int32))


class _Marshalled:
    """Keeps the numpy buffers behind an OrcProblem alive."""

    def __init__(self, prob):
        self.keep = []
        self.p = OrcProblem()
        n = int(prob.H.shape[0])
        self.p.dim = n
        self.p.H = self._op(prob.H)
        ops_c = [self._op(c) for c in prob.C]
        ops_a = [self._op(a) for a in prob.A]
        self.carr = (OrcOp * max(1, len(ops_c)))(*ops_c)
        self.aarr = (OrcOp * max(1, len(ops_a)))(*ops_a)
        self.p.n_c = len(ops_c)
        self.p.C = ct.cast(self.carr, ct.POINTER(OrcOp))
        self.p.n_obs = len(ops_a)
        self.p.A = ct.cast(self.aarr, ct.POINTER(OrcOp))
        psi = np.ascontiguousarray(np.asarray(prob.psi0, dtype=np.complex128)).view(np.float64)
        t = np.ascontiguousarray(np.asarray(prob.t, dtype=np.float64))
        self.keep += [psi, t]
        self.p.psi0 = _dptr(psi)
        self.p.n_t = len(t)
        self.p.t = _dptr(t)
        self.p.rtol = float(prob.rtol)
        self.p.atol = float(prob.atol)
        self.p.max_steps = int(getattr(prob, "max_steps", 1_000_000))
        drive = list(getattr(prob, "drive", []) or [])
        ops_d = [self._op(d[0]) for d in drive]
        self.darr = (OrcOp * max(1, len(ops_d)))(*ops_d)
        coef = np.ascontiguousarray(np.array([[float(a), float(w), float(ph)] for _, a, w, ph in drive]
                                             or [[0.0, 0.0, 0.0]], dtype=np.float64))
        self.keep.append(coef)
        self.p.n_drive = len(ops_d)
        self.p.drive = ct.cast(self.darr, ct.POINTER(OrcOp))
        self.p.drive_coef = _dptr(coef)
        self.n_t = len(t)
        self.n_obs = len(ops_a)

    def _op(self, m):
        m = m.tocsr()
        rp = np.ascontiguousarray(m.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(m.indices, dtype=np.int32)
        v = np.ascontiguousarray(m.data, dtype=np.complex128).view(np.float64)
        self.keep += [rp, ci, v]
        op = OrcOp()
        op.n = int(m.shape[0])
        op.row_ptr = _iptr(rp)
        op.col = _iptr(ci)
        op.val = _dptr(v)
        return op


def philox4x64_10(counter, key):
    c = (ct.c_uint64 * 4)(*[int(x) & (2**64 - 1) for x in counter])
    k = (ct.c_uint64 * 2)(*[int(x) & (2**64 - 1) for x in key])
    o = (ct.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def uniforms(seed: int, traj: int, k: int):
    r = ct.c_double()
    c = ct.c_double()
    lib().orc_uniforms(seed, traj, k, ct.byref(r), ct.byref(c))
    return r.value, c.value


def effective_matrix(prob) -> np.ndarray:
    m = _Marshalled(prob)
    n = m.p.dim
    out = np.zeros((n, n), dtype=np.complex128)
    st = lib().orc_effective_matrix(ct.byref(m.p), _dptr(out.view(np.float64)))
    if st:
        raise RuntimeError(f"orc_effective_matrix failed: {st}")
    return out


def dopri5_fixed(M: np.ndarray, y0: np.ndarray, h: float, nsteps: int, theta: float = 0.5):
    """Fixed-step DOPRI5 on dy/dt = M y.  Returns (y_end, last-step error estimate,
    continuous extension at theta inside the last step)."""
    M = np.ascontiguousarray(M, dtype=np.complex128)
    y0 = np.ascontiguousarray(y0, dtype=np.complex128)
    n = len(y0)
    y = np.zeros(n, np.complex128)
    e = np.zeros(n, np.complex128)
    yd = np.zeros(n, np.complex128)
    st = lib().orc_dopri5_fixed(n, _dptr(M.view(np.float64)), _dptr(y0.view(np.float64)), h, nsteps,
                                theta, _dptr(y.view(np.float64)), _dptr(e.view(np.float64)),
                                _dptr(yd.view(np.float64)))
    if st:
        raise RuntimeError(f"orc_dopri5_fixed failed: {st}")
    return y, e, yd


def dense_weights(theta: float) -> np.ndarray:
    w = np.zeros(7)
    lib().orc_dense_weights(theta, _dptr(w))
    return w


def step_trace(prob, traj: int, seed=None, max_rec: int = 1 << 20):
    """Every attempted Dormand-Prince step of trajectory `traj`: array of rows
    (start time, step size, accepted 1 / rejected 0)."""
    seed = prob.seed if seed is None else seed
    m = _Marshalled(prob)
    rec = np.zeros((max_rec, 3))
    n = ct.c_int64()
    st = lib().orc_step_trace(ct.byref(m.p), seed, traj, max_rec, _dptr(rec), ct.byref(n))
    if st:
        raise RuntimeError(f"orc_step_trace failed: {st}")
    return rec[:n.value].copy()


def mcwf(prob, seed=None, traj0: int = 0, ntraj=None, nthreads=None, max_jumps: int = 64):
    """Runs trajectories traj0 .. traj0+ntraj-1 (Algorithm 1) and returns per-trajectory data."""
    seed = prob.seed if seed is None else seed
    ntraj = prob.ntraj if ntraj is None else ntraj
    nthreads = nthreads or os.cpu_count() or 1
    m = _Marshalled(prob)
    obs = np.zeros((ntraj, m.n_t, m.n_obs))
    obs_im = np.zeros((ntraj, m.n_t, m.n_obs))
    n_jumps = np.zeros(ntraj, np.int32)
    jump_t = np.full((ntraj, max_jumps), np.nan)
    jump_ch = np.full((ntraj, max_jumps), -1, np.int32)
    jump_norm = np.full((ntraj, max_jumps), np.nan)
    status = np.zeros(ntraj, np.int32)
    counts = np.zeros((ntraj, 4), np.int64)
    res = OrcResult(_dptr(obs), _dptr(obs_im), max_jumps, _iptr(n_jumps), _dptr(jump_t),
                    _iptr(jump_ch), _dptr(jump_norm), _iptr(status),
                    counts.ctypes.data_as(ct.POINTER(ct.c_int64)))
    rc = lib().orc_mcwf(ct.byref(m.p), seed, traj0, ntraj, int(nthreads), ct.byref(res))
    return dict(rc=rc, obs=obs, obs_im=obs_im, n_jumps=n_jumps, jump_t=jump_t, jump_ch=jump_ch,
                jump_norm=jump_norm, status=status, accepted=counts[:, 0], rejected=counts[:, 1],
                rhs=counts[:, 2], jumps=counts[:, 3])


def ensemble(obs: np.ndarray):
    """Mean over trajectories and its standard error (sample variance, n - 1)."""
    n = obs.shape[0]
    mean = obs.mean(axis=0)
    se = obs.std(axis=0, ddof=1) / np.sqrt(n) if n > 1 else np.zeros_like(mean)
    return mean, se


def lindblad(prob, rtol: float = 1e-11, atol: float = 1e-13):
    """Tr(A_k rho(t_j)), shape (n_t, n_obs), for rho(0) = |psi0><psi0|."""
    m = _Marshalled(prob)
    out = np.zeros((m.n_t, m.n_obs))
    out_im = np.zeros((m.n_t, m.n_obs))
    st = lib().orc_lindblad(ct.byref(m.p), rtol, atol, _dptr(out), _dptr(out_im))
    if st:
        raise RuntimeError(f"orc_lindblad failed: {st}")
    return out, out_im
