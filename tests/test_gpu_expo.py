"""The exponential method (QTM_METHOD_EXPONENTIAL) on the GPU (run with ``-m gpu``).

Between jumps the kernel applies psi(t) = exp(M (t - t_k)) psi_k through a ladder
of precomputed propagators and a Taylor remainder, and finds each jump time by a
binary descent over the ladder and Newton's method.  The oracle is the same
definition written with scipy's expm and brentq (``oracle/exact.py``): both
follow the exact trajectory, so they agree to rounding -- much tighter than the
Dormand-Prince path's bars -- whatever the stiffness of the system.
"""

import numpy as np
import pytest

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

from test_gpu_parity import PRECS, _within_statistics, gpu_run

pytestmark = pytest.mark.gpu

MAXJ = 64
# Both sides' propagators carry rounding: the ladder (scaling and squaring, up to
# 2^L amplification of the Taylor polynomial's rounding) and scipy's expm (Pade
# with its own squarings) differ by up to ~6e-14 per output interval on the
# stiff system (3e-14 each from a third route).  Over the m intervals between
# two jumps the squared norm thus moves by ~m 1e-13, which shifts a crossing by
# that over the decay rate (~0.5 r): 1e-11 .. 1e-10 after tens of intervals.
TOL_TAU = 1e-9                # every jump time, relative to max(1, tau)
TOL_TAU_MEDIAN = {Q.QTM_PREC_C128: 1e-10, Q.QTM_PREC_DF64: 5e-10}
TOL_OBS = 1e-8                # every per-trajectory observable
TOL_ENSEMBLE = 1e-10


def expo_run(prob, ntraj, precision=Q.QTM_PREC_C128, record=MAXJ, layout=None):
    ctx = Q.qtm_create(prob, record_jumps=record, precision=precision)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    if layout:
        Q.qtm_set_layout(ctx, *layout)
    Q.qtm_run(ctx, ntraj, prob.seed)
    mean, se = Q.qtm_expect(ctx)
    out = dict(mean=mean, se=se, obs=Q.qtm_traj_expect(ctx), stats=Q.qtm_stats(ctx),
               ladder=Q.qtm_expo_ladder(ctx))
    if record:
        out["n_jumps"], out["jump_t"], out["jump_ch"] = Q.qtm_jumps(ctx)
    Q.qtm_destroy(ctx)
    return out


def exact_run(prob, ntraj):
    from oracle import exact, oracle
    o = exact.mcwf(prob, ntraj=ntraj, max_jumps=MAXJ)
    o["mean"], o["se"] = oracle.ensemble(o["obs"])
    return o


def compare_exact(g, o, ntraj, precision):
    np.testing.assert_array_equal(g["n_jumps"], o["n_jumps"])
    dts = []
    for i in range(ntraj):
        k = min(int(o["n_jumps"][i]), MAXJ)
        np.testing.assert_array_equal(g["jump_ch"][i, :k], o["jump_ch"][i, :k], err_msg=f"traj {i}")
        tau = o["jump_t"][i, :k]
        dt = np.abs(g["jump_t"][i, :k] - tau)
        assert np.all(dt <= TOL_TAU * np.maximum(1.0, np.abs(tau))), (i, dt.max())
        dts.append(dt)
    dts = np.concatenate(dts) if dts else np.zeros(0)
    if dts.size >= 20:
        assert np.median(dts) <= TOL_TAU_MEDIAN[precision], np.median(dts)
    assert np.abs(g["obs"] - o["obs"]).max() <= TOL_OBS
    assert np.abs(g["mean"] - o["mean"]).max() <= TOL_ENSEMBLE + TOL_OBS / np.sqrt(ntraj)
    assert g["stats"]["failed"] == 0 and g["stats"]["jumps"] == int(o["n_jumps"].sum())


CASES = [
    ("purcell_qubit", dict(), 200),                      # stiff, N = 10
    ("two_level_driven", dict(), 300),                   # N = 2, one lane per trajectory
    ("paper_unitary_strong", dict(), 150),               # closed-form jump times
    ("jaynes_cummings_driven", dict(), 24),              # N = 60, many jumps
    ("dense_random", dict(N=64, ntraj=16), 16),          # dense: the 64-lane layout
    ("ising_L7", dict(ntraj=6), 6),                      # N = 128: two warps per trajectory
    ("fock_decay", dict(n0=3, kappa=0.5), 100),          # closed-form jump times, forced channel
    ("paper_jaynes_cummings", dict(), 1),                # Sec. 4.3: closed system (no channel), N = 80
    ("dense_random", dict(N=256, ntraj=4), 4),           # the dense workload's size: four warps per trajectory
]


def _problem(name, kw):
    if name == "paper_unitary_strong":
        return S.paper_unitary().with_(C=[S._csr(0.5 * S.sigma_x())])
    return S.by_name(name, **kw)


@pytest.mark.parametrize("prec", [p[1] for p in PRECS], ids=[p[0] for p in PRECS])
@pytest.mark.parametrize("name,kw,ntraj", CASES, ids=[c[0] for c in CASES])
def test_expo_parity_with_exact_oracle(name, kw, ntraj, prec):
    prob = _problem(name, kw)
    g = expo_run(prob, ntraj, precision=prec)
    o = exact_run(prob, ntraj)
    compare_exact(g, o, ntraj, prec)
    levels, delta = g["ladder"]
    assert abs(delta * 2 ** (levels - 1) - (prob.t[-1] - prob.t[0]) / (len(prob.t) - 1)) <= 1e-12


@pytest.mark.parametrize("prec", [p[1] for p in PRECS], ids=[p[0] for p in PRECS])
def test_expo_non_uniform_grid(prec):
    """Output times of uneven spacing: every interval is propagated by its binary
    digits on the ladder plus the Taylor remainder."""
    base = S.purcell_qubit()
    t2 = np.concatenate([base.t[:40:3], [4.05, 4.7, 4.75, 5.0], base.t[51::4], [20.5]])
    prob = base.with_(t=t2)
    g = expo_run(prob, 100, precision=prec)
    o = exact_run(prob, 100)
    compare_exact(g, o, 100, prec)


def test_expo_stiff_ensemble_matches_lindblad(orc):
    prob = S.purcell_qubit(ntraj=4000)
    g = expo_run(prob, prob.ntraj, record=0)
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _within_statistics(g["mean"], g["se"], L, prob.ntraj)


def test_expo_against_dopri5_on_the_stiff_system():
    """Both methods on the same Philox streams: the same jumps for the bulk of the
    trajectories, and the exponential method needs a small fraction of the
    Dormand-Prince path's matrix-vector products on this stiff system."""
    prob = S.purcell_qubit(ntraj=1000)
    a = gpu_run(prob, 1000, record=MAXJ)
    b = expo_run(prob, 1000)
    assert np.mean(a["n_jumps"] == b["n_jumps"]) >= 0.99
    assert np.abs(a["mean"] - b["mean"]).max() <= 1e-5
    assert b["stats"]["rhs_evals"] * 5 < a["stats"]["rhs_evals"], (b["stats"]["rhs_evals"], a["stats"]["rhs_evals"])


def test_expo_layouts_agree():
    """The two lane layouts of N = 60 give the same trajectories (to rounding)."""
    prob = S.jaynes_cummings_driven()
    a = expo_run(prob, 64, layout=(32, 2))
    b = expo_run(prob, 64, layout=(16, 4))
    np.testing.assert_array_equal(a["n_jumps"], b["n_jumps"])
    assert np.abs(a["obs"] - b["obs"]).max() <= 1e-10
    assert b["stats"]["kernel_group"] == 16


def test_expo_switch_back_to_dopri5_is_bitwise_the_default():
    prob = S.jaynes_cummings_driven()
    ref = gpu_run(prob, 64, record=8)
    ctx = Q.qtm_create(prob, record_jumps=8)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    Q.qtm_run(ctx, 64, prob.seed)
    Q.qtm_expect(ctx)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_DOPRI5)
    Q.qtm_run(ctx, 64, prob.seed)
    np.testing.assert_array_equal(Q.qtm_traj_expect(ctx), ref["obs"])
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_expo_ladder(ctx)
    assert ei.value.status == Q.QTM_ERR_STATE
    Q.qtm_destroy(ctx)


def test_expo_argument_errors():
    prob = S.purcell_qubit(ntraj=4)
    ctx = Q.qtm_create(prob)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_method(ctx, 7)
    assert ei.value.status == Q.QTM_ERR_ARG
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_drive(ctx, [(S.kron(S.eye(5), S.sigma_z()), 1.0, 1.0, 0.0)])
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)
    drv = S.driven_dephasing_qubit(ntraj=4)
    ctx = Q.qtm_create(drv)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)
    big = Q.qtm_create(S.ising_chain(9, ntraj=2))  # N = 512
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_method(big, Q.QTM_METHOD_EXPONENTIAL)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(big)


def test_expo_in_a_batch_with_a_dopri5_context():
    """qtm_run_batch runs an exponential-method context beside a Dormand-Prince one
    in one CUDA graph; each gives its single-run result bitwise."""
    stiff = S.purcell_qubit()
    jc = S.jaynes_cummings_driven()
    a = Q.qtm_create(stiff)
    Q.qtm_set_method(a, Q.QTM_METHOD_EXPONENTIAL)
    b = Q.qtm_create(jc)
    Q.qtm_run_batch([a, b], [300, 100], seed=1)
    got_a, got_b = Q.qtm_traj_expect(a), Q.qtm_traj_expect(b)
    Q.qtm_run(a, 300, 1)
    Q.qtm_run(b, 100, 1)
    np.testing.assert_array_equal(got_a, Q.qtm_traj_expect(a))
    np.testing.assert_array_equal(got_b, Q.qtm_traj_expect(b))
    Q.qtm_destroy(a)
    Q.qtm_destroy(b)


@pytest.mark.parametrize("name,kw,ntraj", [("purcell_qubit", dict(), 400), ("jaynes_cummings_driven", dict(), 200),
                                           ("dense_random", dict(N=64, ntraj=100), 100)])
def test_expo_complex64_statistics(orc, name, kw, ntraj):
    """complex64 (FP32 propagators and state, double-float norms): the same jump
    count as the exact oracle for the bulk of the trajectories, jump times within
    the FP32 rounding over the decay rate, and the ensemble within its statistics
    of the Lindblad solution."""
    prob = S.by_name(name, **kw)
    g = expo_run(prob, ntraj, precision=Q.QTM_PREC_C64)
    o = exact_run(prob, ntraj)
    same = g["n_jumps"] == o["n_jumps"]
    assert same.mean() >= 0.95
    dts = []
    for i in np.where(same)[0]:
        k = min(int(o["n_jumps"][i]), MAXJ)
        dts.append(np.abs(g["jump_t"][i, :k] - o["jump_t"][i, :k]))
    dts = np.concatenate(dts)
    assert np.median(dts) <= 1e-4, np.median(dts)
    assert g["stats"]["failed"] == 0
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _within_statistics(g["mean"], g["se"], L, ntraj)


def test_expo_shards_equal_one_run():
    """Contiguous id ranges (one per GPU in a multi-GPU run) reproduce one run
    over all ids bitwise under the exponential method too: every draw is keyed
    by (seed, global trajectory id)."""
    from paper_1810_03047_gb300 import shards
    prob = S.purcell_qubit()
    n, world = 301, 3
    ctx = Q.qtm_create(prob, record_jumps=16)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    Q.qtm_run(ctx, n, 5)
    whole = Q.qtm_traj_expect(ctx)
    parts = []
    for rank in range(world):
        first, count = shards.shard(n, world, rank)
        Q.qtm_run_range(ctx, first, count, 5)
        parts.append(Q.qtm_traj_expect(ctx))
    Q.qtm_destroy(ctx)
    np.testing.assert_array_equal(np.concatenate(parts), whole)
