"""Pins of the exact-propagation oracle (``oracle/exact.py``) to facts outside it.

The oracle propagates psi(t) = exp(M (t - t_k)) psi_k with scipy's expm and finds
the jump time with brentq.  It is checked against closed-form trajectories (the
Sec. 4.1 system with C^dag C proportional to 1, Fock-state decay), against the
independent Dormand-Prince oracle at tight tolerance trajectory by trajectory,
against the Lindblad equation in the ensemble, and for independence from the
output grid (the semigroup property), so that a wrong sign, a dropped term or a
mis-indexed jump in it fails one of them.
"""

import math

import numpy as np

from paper_1810_03047_gb300 import systems as S

from test_oracle_pins import _expected_jumps


def test_exact_strong_unitary_closed_form(orc):
    """C_0 = 0.5 sigma_x: ||psi||^2 = exp(-0.25 (t - t_k)); jump times in closed form
    to 1e-12 (no integration error at all), <sigma_z> = (-1)^N cos(0.4 pi t)."""
    from oracle import exact
    prob = S.paper_unitary().with_(C=[S._csr(0.5 * S.sigma_x())])
    seed, n = 11, 120
    res = exact.mcwf(prob, seed=seed, ntraj=n)
    total = 0
    for i in range(n):
        exp_t = _expected_jumps(seed, i, lambda k: 0.25, prob.t[-1])
        nj = int(res["n_jumps"][i])
        assert nj == len(exp_t)
        total += nj
        np.testing.assert_allclose(res["jump_t"][i, :nj], exp_t, rtol=1e-12, atol=1e-12)
        for j, tj in enumerate(prob.t):
            sign = (-1) ** sum(1 for x in exp_t if x < tj)
            assert abs(res["obs"][i, j, 0] - sign * math.cos(0.4 * math.pi * tj)) < 1e-12
    assert total > 100


def test_exact_fock_decay_closed_form(orc):
    """H = w a^dag a, C = sqrt(kappa) a, psi0 = |3>: rate kappa (3 - k) after k jumps,
    <n> = 3 - (jumps before t) exactly."""
    from oracle import exact
    kappa = 0.5
    prob = S.fock_decay(n0=3, n_fock=6, kappa=kappa, ntraj=150)
    res = exact.mcwf(prob)
    for i in range(prob.ntraj):
        exp_t = _expected_jumps(prob.seed, i, lambda k: kappa * (3 - k), prob.t[-1])
        nj = int(res["n_jumps"][i])
        assert nj == len(exp_t)
        np.testing.assert_allclose(res["jump_t"][i, :nj], exp_t, rtol=1e-12, atol=1e-12)
        assert np.all(res["jump_ch"][i, :nj] == 0)
        for j, tj in enumerate(prob.t):
            assert abs(res["obs"][i, j, 0] - (3 - sum(1 for x in exp_t if x < tj))) < 1e-11


def test_exact_matches_dopri5_oracle_at_tight_tolerance(orc):
    """Two independent oracles of the same trajectories: Dormand-Prince at rtol 1e-12
    (continuous extension, Newton root find) and the exponential (expm, brentq).
    Same jumps and channels; times and outputs within the integrator's error."""
    from oracle import exact
    for prob, n in [(S.purcell_qubit(), 30), (S.jaynes_cummings_driven(), 3), (S.two_level_driven(), 40),
                    (S.paper_photon_birth_death(), 40),      # a creation channel beside the decay
                    (S.dense_random(N=16, ntraj=12), 12),    # dense operators, four channels
                    (S.ising_chain(4, ntraj=8), 8)]:         # eight channels
        e = exact.mcwf(prob, ntraj=n)
        d = orc.mcwf(prob.with_(rtol=1e-12, atol=1e-14), ntraj=n)
        assert d["rc"] == 0
        np.testing.assert_array_equal(e["n_jumps"], d["n_jumps"])
        np.testing.assert_array_equal(e["jump_ch"], d["jump_ch"])
        ok = ~np.isnan(e["jump_t"])
        assert np.abs(e["jump_t"][ok] - d["jump_t"][ok]).max(initial=0.0) <= 1e-9
        assert np.abs(e["obs"] - d["obs"]).max() <= 1e-8


def test_exact_output_grid_does_not_change_trajectories(orc):
    """exp(M (a + b)) = exp(M a) exp(M b): the jump times and the outputs at shared
    times do not depend on which other output times are requested (including a
    non-uniform grid), up to the rounding of the different products (a few 1e-12
    in the state, over decay rates of order 0.1 in the jump times)."""
    from oracle import exact
    prob = S.purcell_qubit(ntraj=12)
    fine = exact.mcwf(prob)
    t2 = np.concatenate([prob.t[::5][:10], [4.7, 4.75, 5.0], prob.t[::5][11:]])
    assert np.all(np.diff(t2) > 0)
    coarse = exact.mcwf(prob.with_(t=t2))
    np.testing.assert_array_equal(fine["n_jumps"], coarse["n_jumps"])
    ok = ~np.isnan(fine["jump_t"])
    np.testing.assert_allclose(coarse["jump_t"][ok], fine["jump_t"][ok], rtol=0, atol=1e-10)
    idx = [int(np.argmin(np.abs(prob.t - x))) for x in t2]
    shared = [q for q, x in enumerate(t2) if abs(prob.t[idx[q]] - x) < 1e-12]
    assert len(shared) >= 40
    np.testing.assert_allclose(coarse["obs"][:, shared], fine["obs"][:, [idx[q] for q in shared]], rtol=0,
                               atol=1e-10)


def test_exact_stiff_ensemble_matches_lindblad(orc):
    """The stiff Purcell system: the exact ensemble against the Lindblad solution."""
    from oracle import exact
    prob = S.purcell_qubit(ntraj=400)
    res = exact.mcwf(prob)
    mean, se = orc.ensemble(res["obs"])
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    d = np.abs(mean - L)
    floor = 1e-4 + 6.0 / prob.ntraj  # points where the sample has no spread yet
    assert np.mean(d <= np.maximum(3 * se, floor)) >= 0.99
    assert np.all(d <= np.maximum(5 * se, floor))
