"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test checks the oracle against something the paper or the mathematics fixes:
the paper's printed matrices (Sec. 4.1 listing), numpy's independent Philox,
closed-form solutions, invariants, the order of the Dormand-Prince pair against
``scipy.linalg.expm``, and the Lindblad master equation (Sec. 2.2).  A plausible
mistake in any part of the oracle -- a dropped term, a wrong sign or index, a
transposed operand, a re-used random number -- fails at least one of them.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg

from paper_1810_03047_gb300 import systems as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MASK64 = (1 << 64) - 1


def numpy_philox_block(seed, traj, k):
    """Philox4x64-10 block for counter (k, traj, 0, 0) and key (seed, 0) from numpy.

    numpy increments its 256-bit counter before producing a block, so the block
    for counter X comes from a generator whose counter is X - 1 (with borrow)."""
    X = (int(k) & MASK64) | ((int(traj) & MASK64) << 64)
    Xm1 = (X - 1) % (1 << 256)
    words = [(Xm1 >> (64 * i)) & MASK64 for i in range(4)]
    g = np.random.Philox(key=np.array([int(seed) & MASK64, 0], dtype=np.uint64),
                         counter=np.array(words, dtype=np.uint64))
    return [int(w) for w in g.random_raw(4)]


def numpy_uniforms(seed, traj, k):
    w = numpy_philox_block(seed, traj, k)
    return ((w[0] >> 11) + 0.5) * 2.0 ** -53, ((w[1] >> 11) + 0.5) * 2.0 ** -53


def read_golden_blocks(name):
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                blocks[cur] = []
                continue
            re_, im_ = (float(x) for x in line.split())
            blocks[cur].append(complex(re_, im_))
    return {k: np.array(v) for k, v in blocks.items()}


# ---------------------------------------------------------------------------
# random stream
# ---------------------------------------------------------------------------

PHILOX_CASES = [(1, 0, 0), (1, 0, 1), (1, 5, 0), (7, 12345, 17), (MASK64, 1 << 40, 1 << 33),
                (3, MASK64, MASK64), (0, 0, 0)]


@pytest.mark.parametrize("seed,traj,k", PHILOX_CASES)
def test_philox_matches_numpy(orc, seed, traj, k):
    assert orc.philox4x64_10([k, traj, 0, 0], [seed, 0]) == numpy_philox_block(seed, traj, k)


@pytest.mark.parametrize("seed,traj,k", PHILOX_CASES)
def test_uniform_mapping(orc, seed, traj, k):
    r, c = orc.uniforms(seed, traj, k)
    r_np, c_np = numpy_uniforms(seed, traj, k)
    assert r == r_np and c == c_np
    assert 0.0 < r < 1.0 and 0.0 < c < 1.0


# ---------------------------------------------------------------------------
# effective Hamiltonian (Eq. eqn:effective:hamiltonian) against printed values
# ---------------------------------------------------------------------------

def test_paper_unitary_stored_matrix(orc):
    g = read_golden_blocks("paper_unitary_stored_matrices.txt")
    prob = S.paper_unitary()
    M = orc.effective_matrix(prob)
    np.testing.assert_allclose(M.ravel(), g["H"], rtol=0, atol=5e-9)
    # the builder reproduces the other printed matrices of the listing
    np.testing.assert_allclose(prob.C[0].toarray().ravel(), g["co"], atol=0)
    np.testing.assert_allclose(prob.A[0].toarray().ravel(), g["eo"], atol=0)
    np.testing.assert_allclose(prob.psi0, g["alpha"], atol=0)


def test_effective_matrix_fock_closed_form(orc):
    prob = S.fock_decay(n0=3, n_fock=6, kappa=0.5, omega=1.3)
    M = orc.effective_matrix(prob)
    n = np.arange(6)
    np.testing.assert_allclose(M, np.diag(-1j * 1.3 * n - 0.25 * n), atol=1e-15)


@pytest.mark.parametrize("name", ["jaynes_cummings_driven", "paper_photon_birth_death", "ising_L4"])
def test_norm_decay_identity(orc, name):
    """Eq. eqn:probabil:collapse: d<psi|psi>/dt = 2 Re<psi|M psi> = -sum_n ||C_n psi||^2."""
    prob = S.by_name(name)
    M = orc.effective_matrix(prob)
    rng = np.random.default_rng(0)
    for _ in range(3):
        psi = rng.standard_normal(prob.dim) + 1j * rng.standard_normal(prob.dim)
        lhs = 2.0 * np.real(np.vdot(psi, M @ psi))
        rhs = -sum(np.linalg.norm(c @ psi) ** 2 for c in prob.C)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))
        # the coherent part is anti-Hermitian: <psi|(M - M^dag)/(-2i)|psi> = <psi|H|psi>
        herm = np.real(np.vdot(psi, ((M - M.conj().T) / (-2j)) @ psi))
        assert abs(herm - np.real(np.vdot(psi, prob.H @ psi))) <= 1e-12 * np.linalg.norm(psi) ** 2 * 10


# ---------------------------------------------------------------------------
# Dormand-Prince 5(4) and its continuous extension against expm
# ---------------------------------------------------------------------------

def _test_ode():
    rng = np.random.default_rng(42)
    n = 5
    M = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2 * n)
    y0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return M, y0


def test_dopri5_global_order_5(orc):
    M, y0 = _test_ode()
    T = 2.0
    errs = []
    for nsteps in (10, 20, 40):
        y, _, _ = orc.dopri5_fixed(M, y0, T / nsteps, nsteps)
        errs.append(np.linalg.norm(y - scipy.linalg.expm(M * T) @ y0))
    for a, b in zip(errs, errs[1:]):
        assert 4.6 < math.log2(a / b) < 5.4, errs


def test_dopri5_error_estimate_order(orc):
    """The embedded estimate h sum (b - bhat) k is the local error of the 4th-order
    solution, O(h^5)."""
    M, y0 = _test_ode()
    est = []
    for h in (0.2, 0.1, 0.05):
        _, e, _ = orc.dopri5_fixed(M, y0, h, 1)
        y4 = scipy.linalg.expm(M * h) @ y0
        y5, _, _ = orc.dopri5_fixed(M, y0, h, 1)
        # the estimate is y5 - y4hat, so the 4th-order result y5 - e misses the exact
        # solution by about -e (y5 itself is an order more accurate)
        true4 = (y5 - e) - y4
        assert np.linalg.norm(true4 + e) <= 0.2 * np.linalg.norm(e)
        est.append(np.linalg.norm(e))
    for a, b in zip(est, est[1:]):
        assert 4.6 < math.log2(a / b) < 5.4, est


@pytest.mark.parametrize("theta", [0.13, 0.5, 0.81])
def test_dense_output_order_4(orc, theta):
    """The continuous extension has local error O(h^5) at every theta."""
    M, y0 = _test_ode()
    errs = []
    for h in (0.4, 0.2, 0.1):
        _, _, yd = orc.dopri5_fixed(M, y0, h, 1, theta)
        errs.append(np.linalg.norm(yd - scipy.linalg.expm(M * theta * h) @ y0))
    for a, b in zip(errs, errs[1:]):
        assert 4.5 < math.log2(a / b) < 5.6, errs


def test_dense_output_endpoints(orc):
    M, y0 = _test_ode()
    y, _, yd1 = orc.dopri5_fixed(M, y0, 0.3, 1, 1.0)
    np.testing.assert_allclose(yd1, y, rtol=0, atol=1e-14)
    _, _, yd0 = orc.dopri5_fixed(M, y0, 0.3, 1, 0.0)
    np.testing.assert_allclose(yd0, y0, rtol=0, atol=0)


# ---------------------------------------------------------------------------
# Algorithm 1 against closed forms
# ---------------------------------------------------------------------------

def _expected_jumps(seed, traj, rate_of_k, t_end, t0=0.0, max_k=1000):
    """Jump times when ||psi||^2 = exp(-rate_k (t - t_k)) after the k-th jump."""
    out, t = [], t0
    for k in range(max_k):
        r, _ = numpy_uniforms(seed, traj, k)
        rate = rate_of_k(k)
        if rate <= 0:
            break
        t = t - math.log(r) / rate
        if t > t_end:
            break
        out.append(t)
    return out


def test_strong_unitary_example_jump_times_and_outputs(orc):
    """Sec. 4.1 system with C_0 = 0.5 sigma_x: C^dag C = 0.25 I, so the norm decays as
    exp(-0.25 (t - t_k)) exactly; jump times follow from r_k in closed form and every
    trajectory's <sigma_z>(t) is (-1)^(jumps before t) cos(0.4 pi t)."""
    prob = S.paper_unitary().with_(C=[S._csr(0.5 * S.sigma_x())], rtol=1e-10, atol=1e-12)
    ntraj, seed = 300, 11
    res = orc.mcwf(prob, seed=seed, ntraj=ntraj)
    assert res["rc"] == 0
    total = 0
    for i in range(ntraj):
        exp_t = _expected_jumps(seed, i, lambda k: 0.25, prob.t[-1])
        nj = int(res["n_jumps"][i])
        assert nj == len(exp_t), (i, nj, exp_t)
        total += nj
        np.testing.assert_allclose(res["jump_t"][i, :nj], exp_t, rtol=1e-7, atol=1e-7)
        assert np.all(res["jump_ch"][i, :nj] == 0)
        for j, tj in enumerate(prob.t):
            if any(abs(tj - x) < 1e-6 for x in exp_t):
                continue
            sign = (-1) ** sum(1 for x in exp_t if x < tj)
            assert abs(res["obs"][i, j, 0] - sign * math.cos(0.4 * math.pi * tj)) < 1e-7
    assert total > 300  # about 2.5 jumps per trajectory are exercised


def test_fock_decay_closed_form(orc):
    """H = w a^dag a, C = sqrt(kappa) a, psi0 = |3>: the norm decays at kappa n with n
    photons left, the channel is forced, and <n>(t) = 3 - (jumps before t)."""
    kappa = 0.5
    prob = S.fock_decay(n0=3, n_fock=6, kappa=kappa, ntraj=400).with_(rtol=1e-10, atol=1e-12)
    seed = prob.seed
    res = orc.mcwf(prob)
    assert res["rc"] == 0
    for i in range(prob.ntraj):
        exp_t = _expected_jumps(seed, i, lambda k: kappa * (3 - k), prob.t[-1])
        nj = int(res["n_jumps"][i])
        assert nj == len(exp_t)
        np.testing.assert_allclose(res["jump_t"][i, :nj], exp_t, rtol=1e-7, atol=1e-7)
        assert np.all(res["jump_ch"][i, :nj] == 0)
        for j, tj in enumerate(prob.t):
            if any(abs(tj - x) < 1e-6 for x in exp_t):
                continue
            assert abs(res["obs"][i, j, 0] - (3 - sum(1 for x in exp_t if x < tj))) < 1e-8
    # ensemble: each photon survives independently, <n> = 3 exp(-kappa t), Binomial variance
    mean = res["obs"][:, :, 0].mean(axis=0)
    p = np.exp(-kappa * prob.t)
    sd = np.sqrt(3 * p * (1 - p) / prob.ntraj)
    assert np.all(np.abs(mean - 3 * p) <= 5 * sd + 1e-12)


def test_paper_unitary_ensemble_closed_form(orc):
    """Sec. 4.1 example: <sigma_z>(t) = exp(-0.005 t) cos(0.4 pi t); per trajectory it is
    +-cos(0.4 pi t), so the ensemble error is bounded with the exact Poisson variance."""
    prob = S.paper_unitary(ntraj=4000)
    res = orc.mcwf(prob)
    assert res["rc"] == 0
    mean = res["obs"][:, :, 0].mean(axis=0)
    t = prob.t
    c = np.cos(0.4 * np.pi * t)
    ex = np.exp(-0.005 * t) * c
    var = (1 - np.exp(-0.01 * t)) * c ** 2  # Var[(-1)^N] cos^2, N ~ Poisson(0.0025 t)
    assert np.all(np.abs(mean - ex) <= 5 * np.sqrt(var / prob.ntraj) + 1e-7)


def test_closed_system_matches_expm(orc):
    """Sec. 4.3 Jaynes-Cummings model without collapse operators: the trajectory is the
    Schrodinger evolution (C2) of Sec. 2.2, psi(t) = exp(-i H t) psi0 (no jumps)."""
    prob = S.paper_jaynes_cummings(n_fock=20, n_t=71, t_end=7.0).with_(rtol=1e-10, atol=1e-12)
    res = orc.mcwf(prob, ntraj=1)
    assert res["rc"] == 0 and res["n_jumps"][0] == 0
    psi0 = prob.psi0 / np.linalg.norm(prob.psi0)
    states = scipy.sparse.linalg.expm_multiply(-1j * prob.H.tocsc(), psi0, start=0.0,
                                               stop=prob.t[-1], num=len(prob.t), endpoint=True)
    A = prob.A[0]
    ex = np.array([np.real(np.vdot(s, A @ s)) / np.real(np.vdot(s, s)) for s in states])
    np.testing.assert_allclose(res["obs"][0, :, 0], ex, atol=1e-7)


# ---------------------------------------------------------------------------
# Lindblad companion integrator against closed forms
# ---------------------------------------------------------------------------

def test_lindblad_torrey_two_level(orc):
    """Resonant driven two-level atom from |g>: rho_ee(t) = rho_ss [1 - exp(-3 g t/4)
    (cos l t + (3 g/(4 l)) sin l t)], l = sqrt(W^2 - g^2/16), rho_ss = (W^2/4)/(g^2/4 + W^2/2)."""
    prob = S.two_level_driven()
    L, Li = orc.lindblad(prob)
    g, W = 0.1, 1.0
    lam = math.sqrt(W * W - g * g / 16)
    rss = (W * W / 4) / (g * g / 4 + W * W / 2)
    t = prob.t
    ree = rss * (1 - np.exp(-3 * g * t / 4) * (np.cos(lam * t) + 3 * g / (4 * lam) * np.sin(lam * t)))
    np.testing.assert_allclose(L[:, 0], ree, atol=1e-9)
    np.testing.assert_allclose(L[:, 1], 0.0, atol=1e-12)  # sigma_x vanishes at Delta = 0
    assert abs(rss - 0.4975124378109453) < 1e-15


def test_lindblad_cavity_and_paper_examples(orc):
    f = S.fock_decay(n0=3, kappa=0.5)
    L, _ = orc.lindblad(f)
    np.testing.assert_allclose(L[:, 0], 3 * np.exp(-0.5 * f.t), atol=1e-10)
    e = S.paper_unitary()
    L, _ = orc.lindblad(e)
    np.testing.assert_allclose(L[:, 0], np.exp(-0.005 * e.t) * np.cos(0.4 * np.pi * e.t), atol=1e-9)
    b = S.paper_photon_birth_death()
    L, _ = orc.lindblad(b)
    kappa, nth = 1 / 0.129, 0.063
    # thermal relaxation; the N = 5 truncation costs about 2e-5
    np.testing.assert_allclose(L[:, 0], nth + (1 - nth) * np.exp(-kappa * b.t), atol=5e-5)


# ---------------------------------------------------------------------------
# ensemble of Algorithm 1 against the Lindblad solution (statistical)
# ---------------------------------------------------------------------------

def _check_against_lindblad(obs, L, floor=1e-7):
    """|mean - L| <= 3 SE for at least 99% of the points and <= 5 SE everywhere.

    Where the sample shows no spread yet (no trajectory has jumped, SE ~ rounding),
    the sample SE says nothing about the unseen jump probability p.  With none seen in
    n trajectories, p <= 3/n at 95% ("rule of three"), and the ensemble mean can then
    be off by at most p times the observable's range; that bound (with a margin of
    2) replaces 5 SE there, plus the integration tolerance ``floor``."""
    n = obs.shape[0]
    mean = obs.mean(axis=0)
    se = obs.std(axis=0, ddof=1) / np.sqrt(n)
    diff = np.abs(mean - L)
    spread = obs.max(axis=(0, 1)) - obs.min(axis=(0, 1))
    bound_flat = floor + 6.0 / n * np.broadcast_to(spread, mean.shape)
    flat = se * 3.0 <= floor
    assert np.all(diff[flat] <= bound_flat[flat]), (diff[flat] - bound_flat[flat]).max()
    z = diff[~flat] / se[~flat]
    assert np.mean(z <= 3.0) >= 0.99, np.sort(z)[-10:]
    assert np.all(z <= 5.0), z.max()


@pytest.mark.parametrize("name,ntraj", [("two_level_driven", 1000), ("paper_photon_birth_death", 1000),
                                        ("jaynes_cummings_driven", 1500), ("ising_L4", 2000)])
def test_ensemble_matches_lindblad(orc, name, ntraj):
    prob = S.by_name(name)
    if name == "two_level_driven":
        prob = S.two_level_driven(extra_sigma_y=True)
    res = orc.mcwf(prob, ntraj=ntraj)
    assert res["rc"] == 0
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _check_against_lindblad(res["obs"], L)


# ---------------------------------------------------------------------------
# invariants, determinism and argument checks
# ---------------------------------------------------------------------------

def test_invariants_two_level(orc):
    prob = S.two_level_driven(extra_sigma_y=True)
    res = orc.mcwf(prob, ntraj=300)
    nj = res["n_jumps"]
    assert nj.sum() > 100
    for i in range(300):
        np.testing.assert_allclose(res["jump_norm"][i, :nj[i]], 1.0, atol=1e-14)
    assert np.all(np.abs(res["obs_im"]) <= 1e-13)          # Hermitian observables: real values
    assert np.all(res["obs"][:, :, 1] == 0.0)               # sigma_x vanishes per trajectory
    pe = res["obs"][:, :, 0]
    assert pe.min() >= -1e-15 and pe.max() <= 1 + 1e-15


def test_invariants_jaynes_cummings(orc):
    prob = S.jaynes_cummings_driven()
    res = orc.mcwf(prob, ntraj=64)
    assert res["rc"] == 0
    nj = res["n_jumps"]
    ok = np.arange(64)
    for i in ok:
        k = min(nj[i], 64)
        np.testing.assert_allclose(res["jump_norm"][i, :k], 1.0, atol=1e-13)
        assert set(res["jump_ch"][i, :k].tolist()) <= {0, 1}
    assert np.all(np.abs(res["obs_im"]) <= 1e-12)
    n = res["obs"][:, :, 0]
    assert n.min() >= -1e-12 and n.max() <= 29 + 1e-9


def test_partition_and_threads_do_not_change_results(orc):
    prob = S.jaynes_cummings_driven()
    a = orc.mcwf(prob, traj0=0, ntraj=24, nthreads=1)
    b1 = orc.mcwf(prob, traj0=0, ntraj=10, nthreads=3)
    b2 = orc.mcwf(prob, traj0=10, ntraj=14, nthreads=2)
    np.testing.assert_array_equal(a["obs"], np.concatenate([b1["obs"], b2["obs"]]))
    np.testing.assert_array_equal(a["jump_t"], np.concatenate([b1["jump_t"], b2["jump_t"]]))


def test_argument_errors_and_limits(orc):
    prob = S.two_level_driven()
    bad_t = prob.with_(t=np.array([0.0, 1.0, 1.0, 2.0]))
    assert orc.mcwf(bad_t, ntraj=2)["rc"] == 1
    assert orc.mcwf(prob.with_(rtol=0.0), ntraj=2)["rc"] == 1
    res = orc.mcwf(S.jaynes_cummings_driven().with_(max_steps=5), ntraj=3)
    assert res["rc"] == 4 and np.all(res["status"] == 4)
    assert np.all(np.isnan(res["obs"][:, -1, :]))
    one = prob.with_(t=np.array([0.0]))
    res = orc.mcwf(one, ntraj=3)
    assert res["rc"] == 0 and res["obs"].shape == (3, 1, 2)
    assert np.all(res["obs"][:, 0, 0] == 0.0)  # |g> has no excitation


# ---------------------------------------------------------------------------
# time-dependent Hamiltonian H(t) = H + sum_k a_k cos(omega_k t + phi_k) H_k
# (Sec. 3: mpi_main accepts a function for a time-dependent Hamiltonian)
# ---------------------------------------------------------------------------

def _phase(prob):
    (_, a, w, ph), = prob.drive
    return (a / w) * (np.sin(w * prob.t + ph) - np.sin(ph))


def test_drive_dephasing_closed_form_per_trajectory(orc):
    """H(t) = a cos(wt + phi) sigma_z with sigma_z dephasing: between jumps psi0 = |+>
    only picks up the relative phase 2F(t), F = (a/w)(sin(wt+phi) - sin phi), and each
    jump flips its sign, so <sigma_x> = (-1)^N cos 2F, <sigma_y> = (-1)^N sin 2F with
    N the jumps up to t.  Checks that the stage times reach the coefficient (a drive
    evaluated at the step start would miss F by O(h))."""
    prob = S.driven_dephasing_qubit(ntraj=300).with_(rtol=1e-10, atol=1e-12)
    res = orc.mcwf(prob, ntraj=300, max_jumps=64)
    assert res["rc"] == 0 and res["n_jumps"].sum() > 150
    F = _phase(prob)
    for i in range(300):
        jt = res["jump_t"][i, :res["n_jumps"][i]]
        N = (jt[None, :] <= prob.t[:, None]).sum(axis=1)
        np.testing.assert_allclose(res["obs"][i, :, 0], (-1.0) ** N * np.cos(2 * F), atol=1e-8)
        np.testing.assert_allclose(res["obs"][i, :, 1], (-1.0) ** N * np.sin(2 * F), atol=1e-8)


def test_drive_lindblad_closed_form(orc):
    """The master equation with the same drive: <sigma_x> = exp(-2 gamma t) cos 2F."""
    prob = S.driven_dephasing_qubit()
    L, _ = orc.lindblad(prob, 1e-11, 1e-13)
    F = _phase(prob)
    decay = np.exp(-2 * 0.1 * prob.t)
    np.testing.assert_allclose(L[:, 0], decay * np.cos(2 * F), atol=1e-9)
    np.testing.assert_allclose(L[:, 1], decay * np.sin(2 * F), atol=1e-9)


def test_constant_drive_equals_static_term(orc):
    """A term with omega = phi = 0 is the constant a H_k: the same trajectories as
    with a H_k folded into H (the same jumps; rounding-level differences only)."""
    stat = S.jaynes_cummings_driven(n_fock=8, n_t=41, t_end=8.0, E=0.5)
    base = S.jaynes_cummings_driven(n_fock=8, n_t=41, t_end=8.0, E=0.0)
    a = S.kron(S.destroy(8), S.eye(2))
    drv = base.with_(drive=[(a + S.dag(a), 0.5, 0.0, 0.0)])
    r1 = orc.mcwf(stat, ntraj=60)
    r2 = orc.mcwf(drv, ntraj=60)
    np.testing.assert_array_equal(r1["n_jumps"], r2["n_jumps"])
    np.testing.assert_allclose(r1["obs"], r2["obs"], atol=1e-7)


def test_drive_ensemble_matches_lindblad(orc):
    """Algorithm 1 with a modulated cavity drive against the driven master equation."""
    prob = S.jaynes_cummings_pulsed(n_fock=8, n_t=81, t_end=8.0)
    res = orc.mcwf(prob, ntraj=1500)
    assert res["rc"] == 0
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _check_against_lindblad(res["obs"], L)
