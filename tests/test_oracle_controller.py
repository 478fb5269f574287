"""The oracle's step-size controller and starting step, pinned against scipy's RK45.

scipy.integrate.RK45 is an independent implementation of the same published
integrator the oracle uses between jumps (Dormand & Prince 1980; Hairer,
Norsett & Wanner I, Sec. II.4): the same 5(4) pair with the FSAL stage, the same
RMS error norm with scale atol + rtol max(|y|, |y_new|), the HNW starting-step
heuristic, safety 0.9, growth factor clamped to [0.2, 10] with exponent 1/5 and
no growth on the step that follows a rejection.  On a trajectory that makes no
jump the oracle integrates dpsi/dt = M psi with nothing else in the loop, so its
accepted and rejected step counts must equal RK45's exactly: a wrong exponent,
clamp, safety factor, error norm or starting-step formula changes the step
sequence within a few steps and the counts with it.

One difference is by design: when the step would end within 1 % of the last
output time the oracle stretches it to end there (RK45 would leave a sliver of
a step).  The end times here are chosen from RK45's own step sequence so that
the plain comparison is unaffected, and one test pins the stretch itself.
"""

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from paper_1810_03047_gb300 import systems as S


def _rk45(M, y0, t_end, rtol, atol):
    """RK45's step sequence on dy/dt = M y: accepted step end times, the step
    size proposed after each accepted step, and the accepted / rejected counts."""
    sol = scipy.integrate.RK45(lambda t, y: M @ y, 0.0, y0.astype(np.complex128), t_end,
                               rtol=rtol, atol=atol)
    ends, props = [], []
    while sol.status == "running":
        sol.step()
        ends.append(sol.t)
        props.append(sol.h_abs)
    assert sol.status == "finished"
    acc = len(ends)
    # one evaluation for f(t0), one for the starting-step estimate, six per attempt (FSAL)
    att, rem = divmod(sol.nfev - 2, 6)
    assert rem == 0
    return np.array(ends), np.array(props), acc, att - acc


def _rk45_attempts(M, y0, t0, t_end, rtol, atol, first_step=None):
    """Every attempted RK45 step as rows (start time, size, accepted 1 / rejected 0),
    read from the times at which RK45 evaluates the right-hand side: after f(t0)
    (and the starting-step estimate) each attempt makes six evaluations, the
    fifth at the stage time t + h (c_6 = 1) and the sixth at t + h for FSAL."""
    calls = []

    def f(t, y):
        calls.append(t)
        return M @ y

    sol = scipy.integrate.RK45(f, t0, y0.astype(np.complex128), t_end, rtol=rtol, atol=atol,
                               first_step=first_step)
    ends = []
    while sol.status == "running":
        sol.step()
        ends.append(sol.t)
    assert sol.status == "finished"
    head = 1 if first_step is not None else 2
    groups = np.array(calls[head:]).reshape(-1, 6)
    rows, t = [], t0
    for g in groups:
        h = (g[4] - g[0]) * 5.0 / 4.0   # stage times t + h/5 and t + h
        acc = 1.0 if np.isclose(g[4], ends[len([r for r in rows if r[2]])], rtol=0, atol=1e-13 * max(1.0, abs(g[4]))) else 0.0
        rows.append((t, h, acc))
        if acc:
            t = g[4]
    return np.array(rows)


def _same_sequence(orc_rows, ref_rows):
    """The oracle's attempts equal RK45's: the same accept/reject pattern, and the
    same start times and step sizes up to the rounding of the error estimate.
    That estimate is a sum of stage terms that cancel; for components near atol
    the cancellation leaves only a few correct digits in FP64, and the two
    implementations sum in different orders (RK45 through a BLAS product), so
    their error norms differ in the 7th digit and their step sizes by ~1e-7
    relative -- far below the percent-level changes a wrong controller makes."""
    assert orc_rows.shape == ref_rows.shape, (orc_rows.shape, ref_rows.shape)
    np.testing.assert_array_equal(orc_rows[:, 2], ref_rows[:, 2])
    np.testing.assert_allclose(orc_rows[:, 0], ref_rows[:, 0], rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(orc_rows[:, 1], ref_rows[:, 1], rtol=1e-6)


def _no_jump_ids(orc, prob, M, t_end, want, search=4000):
    """Trajectory ids whose first threshold r_0 lies below the no-jump squared norm
    at t_end: those trajectories integrate psi' = M psi from t0 to t_end untouched."""
    psi0 = prob.psi0 / np.linalg.norm(prob.psi0)
    nn = float(np.linalg.norm(scipy.linalg.expm(M * t_end) @ psi0) ** 2)
    ids = [i for i in range(search) if orc.uniforms(prob.seed, i, 0)[0] < 0.999 * nn]
    assert len(ids) >= want, (len(ids), nn)
    return ids[:want]


def _end_inside_step(ends, props, m, frac):
    """An end time a fraction `frac` of the way into RK45's (m+1)-th accepted step,
    taken where that step needed no retry (its size is the proposal of step m)."""
    for i in range(m, len(ends) - 2):
        h = ends[i + 1] - ends[i]
        if np.isclose(h, props[i], rtol=1e-12, atol=0):
            return ends[i] + frac * h, i + 1
    raise AssertionError("no un-retried step found")


CASES = [
    # (system builder, rtol, atol, approximate end time, step index to end in)
    ("closed_jcm", 1e-8, 1e-10, 6.0, 60),
    ("closed_jcm", 1e-6, 1e-9, 6.0, 20),
    ("jaynes_cummings", 1e-8, 1e-10, 4.0, 40),
    ("two_level", 1e-8, 1e-10, 12.0, 40),
    ("dense16", 1e-7, 1e-10, 3.0, 30),
]


def _system(name):
    if name == "closed_jcm":
        return S.paper_jaynes_cummings(n_fock=20, n_t=11, t_end=6.0)
    if name == "jaynes_cummings":
        return S.jaynes_cummings_driven(ntraj=4, n_fock=12, n_t=11, t_end=4.0)
    if name == "two_level":
        return S.two_level_driven(ntraj=4, n_t=11, t_end=12.0)
    if name == "dense16":
        return S.dense_random(ntraj=4, N=16, n_c=2, n_t=11, t_end=3.0, c_norm=0.5)
    raise KeyError(name)


@pytest.mark.parametrize("name,rtol,atol,t_big,m", CASES)
def test_step_counts_equal_rk45(orc, name, rtol, atol, t_big, m):
    prob = _system(name).with_(rtol=rtol, atol=atol)
    M = orc.effective_matrix(prob)
    y0 = prob.psi0 / np.linalg.norm(prob.psi0)
    ends, props, _, _ = _rk45(M, y0, 4 * t_big, rtol, atol)
    t_end, _ = _end_inside_step(ends, props, m, 0.5)
    _, _, acc, rej = _rk45(M, y0, t_end, rtol, atol)
    assert acc > 10
    run = prob.with_(t=np.linspace(0.0, t_end, 7))
    if prob.C:
        ids = _no_jump_ids(orc, run, M, t_end, 3)
    else:
        ids = [0]
    ref = _rk45_attempts(M, y0, 0.0, t_end, rtol, atol)
    assert len(ref) == acc + rej and ref[:, 2].sum() == acc
    for i in ids:
        res = orc.mcwf(run, traj0=i, ntraj=1, nthreads=1)
        assert res["rc"] == 0 and res["n_jumps"][0] == 0
        assert int(res["accepted"][0]) == acc, (name, i, int(res["accepted"][0]), acc)
        assert int(res["rejected"][0]) == rej, (name, i, int(res["rejected"][0]), rej)
        # f(t0), the starting-step estimate and six evaluations per attempt
        assert int(res["rhs"][0]) == 2 + 6 * (acc + rej)
        _same_sequence(orc.step_trace(run, i), ref)


def test_rejections_are_exercised(orc):
    """A long run of the closed Sec. 4.3 system at rtol 1e-7 makes the controller
    reject dozens of steps, and on several of them the step accepted right
    after the rejection has so small an error that it would grow without the
    rule "no growth right after a rejection" (RK45's step size is then left
    unchanged, which the loop below counts): both the rejection branch and that
    rule are part of the comparison, not only the accept branch."""
    prob = S.paper_jaynes_cummings(n_fock=20, n_t=11, t_end=6.0).with_(rtol=1e-7, atol=1e-10)
    M = orc.effective_matrix(prob)
    y0 = (prob.psi0 / np.linalg.norm(prob.psi0)).astype(np.complex128)
    ends, props, _, _ = _rk45(M, y0, 40.0, prob.rtol, prob.atol)
    t_end, _ = _end_inside_step(ends, props, 1100, 0.5)
    sol = scipy.integrate.RK45(lambda t, y: M @ y, 0.0, y0, t_end, rtol=prob.rtol, atol=prob.atol)
    held = 0
    while sol.status == "running":
        nf = sol.nfev
        sol.step()
        if sol.nfev - nf > 6 and sol.h_abs == abs(sol.t - sol.t_old):
            held += 1
    acc = int(np.searchsorted(ends, t_end)) + 1
    rej = (sol.nfev - 2) // 6 - acc
    assert rej >= 30 and held >= 3, (rej, held)
    run = prob.with_(t=np.linspace(0.0, t_end, 7))
    res = orc.mcwf(run, ntraj=1, nthreads=1)
    assert (int(res["accepted"][0]), int(res["rejected"][0])) == (acc, rej)
    _same_sequence(orc.step_trace(run, 0), _rk45_attempts(M, y0, 0.0, t_end, prob.rtol, prob.atol))


def test_last_step_is_stretched_to_the_end_time(orc):
    """By design the oracle ends on the last output time with one step when the
    controller's step would fall short of it by under 1 %: with the end time
    0.5 % past the end of an accepted RK45 step, RK45 takes that step and then a
    sliver of 0.5 % of it, while the oracle takes one step 1.005 times as long.
    Where RK45's error on that step was at most 0.9, the stretched step's error
    (1.005^5 times as large, about 0.92) is still accepted, so the oracle makes
    exactly one accepted step fewer and the same rejections."""
    prob = S.jaynes_cummings_driven(ntraj=4, n_fock=12, n_t=11, t_end=4.0)
    M = orc.effective_matrix(prob)
    y0 = prob.psi0 / np.linalg.norm(prob.psi0)
    ends, props, _, _ = _rk45(M, y0, 16.0, prob.rtol, prob.atol)
    done = 0
    for m in range(30, len(ends) - 3):
        h = ends[m + 1] - ends[m]
        if not np.isclose(h, props[m], rtol=1e-12, atol=0):
            continue
        # the error of that step from the factor it produced: fac = 0.9 err^(-1/5)
        fac = props[m + 1] / h
        if not (fac < 10.0 and (fac / 0.9) ** -5 <= 0.9):
            continue
        t_end = ends[m] + 1.005 * h
        _, _, acc, rej = _rk45(M, y0, t_end, prob.rtol, prob.atol)
        run = prob.with_(t=np.linspace(0.0, t_end, 5))
        for i in _no_jump_ids(orc, run, M, t_end, 2):
            res = orc.mcwf(run, traj0=i, ntraj=1, nthreads=1)
            assert res["n_jumps"][0] == 0
            assert int(res["accepted"][0]) == acc - 1, (m, int(res["accepted"][0]), acc)
            assert int(res["rejected"][0]) == rej
        done += 1
        if done == 3:
            break
    assert done == 3


def test_starting_step_alone(orc):
    """The starting step decides the first attempt.  With the end time 0.4 % past
    RK45's starting step (accepted at the first attempt) the oracle stretches
    its first step to the end (one step; RK45 adds a sliver), and 2 % past it
    the oracle needs a second step like RK45: so the oracle's HNW starting step
    lies within [0.994, 1.0099] of RK45's."""
    prob = S.two_level_driven(ntraj=4, n_t=11, t_end=12.0)
    M = orc.effective_matrix(prob)
    y0 = prob.psi0 / np.linalg.norm(prob.psi0)
    h_start = scipy.integrate.RK45(lambda t, y: M @ y, 0.0, y0.astype(np.complex128), 10.0,
                                   rtol=prob.rtol, atol=prob.atol).h_abs
    for frac, delta in ((1.004, 1), (1.02, 0)):
        t_end = frac * h_start
        _, _, acc, rej = _rk45(M, y0, t_end, prob.rtol, prob.atol)
        assert (acc, rej) == (2, 0)
        run = prob.with_(t=np.array([0.0, t_end]))
        for i in _no_jump_ids(orc, run, M, t_end, 2):
            res = orc.mcwf(run, traj0=i, ntraj=1, nthreads=1)
            assert (int(res["accepted"][0]), int(res["rejected"][0])) == (acc - delta, 0), (frac, i)


def _slow_then_fast(omega, gamma=0.1, t_end=40.0):
    """|0> decays slowly (no coupling), the one jump C = sqrt(gamma) |1><0| lands in
    the pair |1>, |2> that oscillates at omega: after the jump the step kept from
    the slow phase is far too large for the fast one."""
    import scipy.sparse as sp
    H = sp.csr_matrix(np.array([[0, 0, 0], [0, 0, omega], [0, omega, 0]], dtype=np.complex128))
    C = sp.csr_matrix(np.array([[0, 0, 0], [np.sqrt(gamma), 0, 0], [0, 0, 0]], dtype=np.complex128))
    A = sp.csr_matrix(np.diag([0.0, 1.0, 0.0]).astype(np.complex128))
    return S.Problem("slow_then_fast", H, [C], [A], np.array([1, 0, 0], np.complex128),
                     np.linspace(0.0, t_end, 5), 1e-8, 1e-10, 1, 1)


@pytest.mark.parametrize("omega", [5.0, 40.0])
def test_rejections_after_a_jump_match_rk45(orc, omega):
    """After a jump the oracle keeps the step size of the step that contained the
    crossing (Algorithm 1 (D) restarts at tau).  Here that step is hundreds of
    times too large for the post-jump dynamics, so the controller rejects it
    again and again, at the 0.2 floor while the error is above (0.9/0.2)^5, and
    the first accepted step after the rejections may not grow.  The trajectory's
    counts are those of two RK45 runs: from t0 up to and including the step whose
    end norm falls below r_0, then from tau with RK45's first step set to that
    step's size."""
    prob = _slow_then_fast(omega)
    M = orc.effective_matrix(prob)
    y0 = prob.psi0.astype(np.complex128)
    seed = prob.seed
    for traj in range(64):
        r0 = orc.uniforms(seed, traj, 0)[0]
        tau = -np.log(r0) / 0.1
        if 5.0 < tau < 15.0:
            break
    # (1) up to the crossing step
    sol = scipy.integrate.RK45(lambda t, y: M @ y, 0.0, y0, 1e3, rtol=prob.rtol, atol=prob.atol)
    acc1, t_prev = 0, 0.0
    while True:
        t_prev = sol.t
        sol.step()
        acc1 += 1
        if np.vdot(sol.y, sol.y).real < r0:
            break
    rej1 = (sol.nfev - 2) // 6 - acc1
    h_cross = sol.t - t_prev
    # (2) from tau in |1> with the kept step; an end time inside an un-retried step
    y1 = np.array([0, 1, 0], np.complex128)
    big = scipy.integrate.RK45(lambda t, y: M @ y, tau, y1, tau + 20.0 * h_cross, rtol=prob.rtol, atol=prob.atol,
                               first_step=h_cross)
    ends, props = [], []
    while big.status == "running" and (not ends or ends[-1] - tau < 1.5 * h_cross):
        big.step()
        ends.append(big.t)
        props.append(big.h_abs)
    # end past tau + h_cross, so the kept step is not clipped to the end time
    first = next(i for i, e in enumerate(ends) if e - tau > 1.1 * h_cross)
    t_end, _ = _end_inside_step(np.array(ends), np.array(props), first, 0.5)
    sol2 = scipy.integrate.RK45(lambda t, y: M @ y, tau, y1, t_end, rtol=prob.rtol, atol=prob.atol,
                                first_step=h_cross)
    acc2 = 0
    while sol2.status == "running":
        sol2.step()
        acc2 += 1
    rej2 = (sol2.nfev - 1) // 6 - acc2
    assert rej2 >= 3  # the post-jump rejections are really exercised
    run = prob.with_(t=np.linspace(0.0, t_end, 5))
    res = orc.mcwf(run, traj0=traj, ntraj=1, nthreads=1)
    assert res["n_jumps"][0] == 1 and abs(res["jump_t"][0, 0] - tau) <= 1e-7 * tau
    pre = _rk45_attempts(M, y0, 0.0, sol.t, prob.rtol, prob.atol)
    post = _rk45_attempts(M, y1, res["jump_t"][0, 0], t_end, prob.rtol, prob.atol, first_step=h_cross)
    _same_sequence(orc.step_trace(run, traj), np.vstack([pre, post]))
    assert (int(res["accepted"][0]), int(res["rejected"][0])) == (acc1 + acc2, rej1 + rej2), \
        (int(res["accepted"][0]), int(res["rejected"][0]), acc1, acc2, rej1, rej2)
