"""Exact trajectories of Algorithm 1 (Sec. 2.2): the oracle of the exponential
propagation.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing in the library imports this
module, and this module imports nothing from the library.

Between two jumps a trajectory obeys d psi/dt = -i H_eff psi = M psi
(Sec. 2.2, Eq. eqn:effective:hamiltonian, hbar = 1), a linear equation with a
constant operator, so psi(t) = exp(M (t - t_k)) psi_k exactly after the k-th jump
at t_k.  Algorithm 1 then reads:

  (A) r_0, c_0 from the random stream; psi = psi0;
  (B) the jump happens at the first time tau at which ||psi(tau)||^2 = r_k.  The
      squared norm cannot increase (d||psi||^2/dt = -sum_n ||C_n psi||^2 <= 0),
      so if ||psi(t_j)||^2 >= r_k at an output time t_j no jump happened before
      it, and otherwise the crossing in (t_prev, t_j) is the unique root there;
  (C) the channel is n* = min{n : sum_{i<=n} w_i >= c_k sum_i w_i} with
      w_i = ||C_i psi(tau)||^2 (Eq. eqn:probability:of:cn), and
      psi <- C_n* psi(tau) / ||C_n* psi(tau)|| (Eq. eqn:state:for:new:time);
  (D) k <- k + 1, fresh r_k, c_k, and the evolution restarts at tau.

This module writes that definition out with library routines as its steps:
``scipy.linalg.expm`` for the exponential, ``scipy.optimize.brentq`` for the
root, scipy's sparse products for C_n psi and A_k psi.  M comes from the C
oracle's effective matrix and (r_k, c_k) from its Philox stream, both pinned on
their own.  There is no step-size control and no interpolation: the results
differ from the exact trajectory by rounding and by the root tolerance only.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.optimize

from oracle import oracle as _orc


class _Propagators:
    """exp(M d) for the durations d met so far (the output grid repeats a few)."""

    def __init__(self, M):
        self.M = M
        self.cache = {}

    def __call__(self, d: float) -> np.ndarray:
        E = self.cache.get(d)
        if E is None:
            E = scipy.linalg.expm(self.M * d)
            if len(self.cache) < 4096:
                self.cache[d] = E
        return E


def _norm2(y) -> float:
    return float(np.vdot(y, y).real)


def _values(prob, y) -> np.ndarray:
    """Re<y|A_k|y> / <y|y> for every observable (Sec. 3: expectation operators)."""
    nn = _norm2(y)
    return np.array([float(np.vdot(y, A @ y).real) / nn for A in prob.A])


def trajectory(prob, M, seed: int, traj: int, prop: _Propagators, max_jumps: int = 64):
    """One trajectory (global id traj) on the output grid prob.t."""
    t = np.asarray(prob.t, dtype=np.float64)
    psi = np.asarray(prob.psi0, dtype=np.complex128)
    psi = psi / math.sqrt(_norm2(psi))
    obs = np.zeros((len(t), len(prob.A)))
    jumps = []
    k = 0
    r, c = _orc.uniforms(seed, traj, k)
    t_cur = float(t[0])
    obs[0] = _values(prob, psi)
    for j in range(1, len(t)):
        while True:
            d = float(t[j]) - t_cur
            y = prop(d) @ psi
            if _norm2(y) >= r:
                psi, t_cur = y, float(t[j])
                obs[j] = _values(prob, y)
                break
            # (B): the crossing lies in (t_cur, t_j)
            base = psi
            f = lambda s: _norm2(scipy.linalg.expm(M * s) @ base) - r
            s = scipy.optimize.brentq(f, 0.0, d, xtol=1e-15 * max(1.0, abs(t_cur)), rtol=4 * np.finfo(float).eps,
                                      maxiter=200)
            y = scipy.linalg.expm(M * s) @ base
            # (C)
            w = np.array([_norm2(C @ y) for C in prob.C])
            total = float(w.sum())
            if not total > 0.0:
                raise RuntimeError("no channel: every ||C_n psi|| is zero")
            cum = np.cumsum(w)
            ch = int(np.argmax(cum >= c * total)) if np.any(cum >= c * total) else len(w) - 1
            psi = (prob.C[ch] @ y) / math.sqrt(w[ch])
            t_cur = t_cur + s
            jumps.append((t_cur, ch))
            # (D)
            k += 1
            r, c = _orc.uniforms(seed, traj, k)
    n = len(jumps)
    jt = np.full(max_jumps, np.nan)
    jc = np.full(max_jumps, -1, np.int32)
    for q, (tau, ch) in enumerate(jumps[:max_jumps]):
        jt[q], jc[q] = tau, ch
    return obs, n, jt, jc


def mcwf(prob, seed=None, traj0: int = 0, ntraj=None, max_jumps: int = 64):
    """Trajectories traj0 .. traj0+ntraj-1; the same fields as the C oracle's mcwf."""
    seed = prob.seed if seed is None else seed
    ntraj = prob.ntraj if ntraj is None else ntraj
    M = _orc.effective_matrix(prob)
    prop = _Propagators(M)
    obs = np.zeros((ntraj, len(prob.t), len(prob.A)))
    n_jumps = np.zeros(ntraj, np.int32)
    jump_t = np.full((ntraj, max_jumps), np.nan)
    jump_ch = np.full((ntraj, max_jumps), -1, np.int32)
    for i in range(ntraj):
        obs[i], n_jumps[i], jump_t[i], jump_ch[i] = trajectory(prob, M, seed, traj0 + i, prop, max_jumps)
    return dict(rc=0, obs=obs, n_jumps=n_jumps, jump_t=jump_t, jump_ch=jump_ch)
