"""The learned jump-time proposal on the GPU (run with ``-m gpu``): the training
kernels' gradient against the FP64 backprop of oracle/mlp.py, and the whole
pipeline -- pairs generated by the plain method, training on the GPU, inference
fused in the trajectory kernel -- with the exact root find still deciding the
jumps."""

import numpy as np
import pytest

from oracle import mlp
from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 64, 300, 4097])
def test_training_kernel_gradient_matches_fp64_backprop(n):
    rng = np.random.default_rng(n)
    p = (rng.standard_normal(mlp.N_PARAMS) * 0.2).astype(np.float32)
    x = rng.standard_normal((n, 6)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    loss, g = Q.qtm_mlp_loss_grad(np.concatenate([p, np.zeros(12, np.float32)]), x, t)
    l_ref, g_ref = mlp.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - l_ref) <= 1e-5 * max(1.0, abs(l_ref))
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-4 * scale, np.abs(g - g_ref).max() / scale


def _run(prob, ntraj, seed, proposal, prec=Q.QTM_PREC_DF64, params=None, record=64):
    ctx = Q.qtm_create(prob, precision=prec, record_jumps=record)
    if params is not None:
        Q.qtm_proposal_set(ctx, params)
        Q.qtm_proposal_enable(ctx, proposal)
    Q.qtm_run(ctx, ntraj, seed)
    mean, se = Q.qtm_expect(ctx)
    nj, jt, jc = Q.qtm_jumps(ctx)
    st = Q.qtm_stats(ctx)
    Q.qtm_destroy(ctx)
    return dict(mean=mean, se=se, n_jumps=nj, jump_t=jt, jump_ch=jc, stats=st)


@pytest.fixture(scope="module")
def trained():
    """Pairs from 4,000 JC trajectories of the plain method, network trained on the GPU."""
    prob = S.jaynes_cummings_driven()
    ctx = Q.qtm_create(prob, precision=Q.QTM_PREC_DF64)
    npairs = Q.qtm_proposal_collect(ctx, 4000, 11, stride=8, max_per_traj=96)
    f, dt = Q.qtm_proposal_pairs(ctx, npairs)
    loss, base = Q.qtm_proposal_train(ctx, steps=1500, batch=4096, lr=2e-3, seed=11)
    params = Q.qtm_proposal_get(ctx)
    Q.qtm_destroy(ctx)
    return dict(prob=prob, npairs=npairs, f=f, dt=dt, loss=loss, base=base, params=params)


def test_pairs_are_consistent(trained):
    f, dt = trained["f"], trained["dt"]
    assert trained["npairs"] > 50000
    assert np.all(f[:, 0] > 0) and np.all(dt > 0)           # decay rate and time left positive
    assert np.all(f[:, 2] > 0) and np.all(f[:, 2] <= 1 + 1e-6)  # norm in (0, 1]
    assert np.all(np.log(f[:, 2]) >= f[:, 3] - 1e-6)          # not yet crossed: norm >= r
    est = (np.log(f[:, 2]) - f[:, 3]) / f[:, 0]
    # the constant-rate estimate is the right order of magnitude for the time left
    assert 0.2 < np.median(dt / est) < 5.0


def test_network_improves_on_constant_rate_estimate(trained):
    assert np.isfinite(trained["loss"]) and trained["loss"] < 0.8 * trained["base"], (trained["loss"], trained["base"])


def test_proposal_keeps_jumps_and_reports_gain(trained, capsys):
    """The root find still decides: with the proposal on, every trajectory makes
    the same jumps through the same channels at the same times up to the
    integration tolerance; only the step sequence changes.

    The step count is reported, not required to fall.  With a continuous
    extension the step that contains a crossing is kept up to the crossing and
    the next step starts there, so the only work a jump discards is the tail of
    that one step; shortening the step to end just past the predicted crossing
    saves none of it, and a prediction that lands early adds a step.  The bar is
    therefore that the proposal costs at most 2 % in attempted steps."""
    prob, params = trained["prob"], trained["params"]
    n = 2000
    off = _run(prob, n, 1, False, params=params)
    on = _run(prob, n, 1, True, params=params)
    np.testing.assert_array_equal(on["n_jumps"], off["n_jumps"])
    for i in range(n):
        k = min(int(off["n_jumps"][i]), 64)
        np.testing.assert_array_equal(on["jump_ch"][i, :k], off["jump_ch"][i, :k])
        dt = np.abs(on["jump_t"][i, :k] - off["jump_t"][i, :k])
        assert np.all(dt <= 1e-6 * np.maximum(1.0, off["jump_t"][i, :k])), (i, dt.max())
    # the two step sequences move jump times by ~rtol; an output flips only where a
    # jump time crosses an output time, which none does here
    assert np.abs(on["mean"] - off["mean"]).max() <= 1e-5
    s_off = off["stats"]["accepted"] + off["stats"]["rejected"]
    s_on = on["stats"]["accepted"] + on["stats"]["rejected"]
    with capsys.disabled():
        print(f"\nproposal: attempted steps per trajectory {s_off / n:.1f} -> {s_on / n:.1f} "
              f"({100 * (s_off - s_on) / s_off:+.2f} %), loss {trained['loss']:.4f} vs "
              f"rate estimate {trained['base']:.4f}")
    assert s_on <= 1.02 * s_off


# Bars against the exact oracle at rtol 1e-10, atol 1e-12.  Measured on the CPU,
# the Dormand-Prince oracle itself meets them with room: on the first 200 JC
# trajectories identical jumps and channels, jump times within 8.7e-10 relative
# (median 2.4e-11), outputs within 1.3e-7, ensemble 1.6e-9.  The proposal-on and
# proposal-off GPU runs are held to the same bars.
EXACT_NTRAJ = 160
EXACT_TAU_MAX = 5e-9      # every jump time, relative to max(1, tau)
EXACT_TAU_MEDIAN = 2e-10
EXACT_OBS = 1e-6          # every per-trajectory output
EXACT_ENSEMBLE = 1e-8


@pytest.fixture(scope="module")
def exact_jc():
    from oracle import exact, oracle
    prob = S.jaynes_cummings_driven().with_(rtol=1e-10, atol=1e-12)
    o = exact.mcwf(prob, ntraj=EXACT_NTRAJ, max_jumps=64)
    o["mean"], _ = oracle.ensemble(o["obs"])
    return prob, o


@pytest.mark.parametrize("prec", [Q.QTM_PREC_C128, Q.QTM_PREC_DF64])
@pytest.mark.parametrize("proposal", [False, True])
def test_proposal_path_against_the_exact_oracle(trained, exact_jc, prec, proposal):
    """The proposal-on kernels against the exact trajectory (expm between jumps,
    brentq for the crossing), trajectory by trajectory, at the same bars as the
    proposal-off kernels: the learned step choice leaves every jump decision to
    the root find and changes results only within the integration tolerance."""
    prob, ex = exact_jc
    ctx = Q.qtm_create(prob, precision=prec, record_jumps=64)
    Q.qtm_proposal_set(ctx, trained["params"])
    Q.qtm_proposal_enable(ctx, proposal)
    Q.qtm_run(ctx, EXACT_NTRAJ, prob.seed)
    mean, _ = Q.qtm_expect(ctx)
    obs = Q.qtm_traj_expect(ctx)
    nj, jt, jc = Q.qtm_jumps(ctx)
    Q.qtm_destroy(ctx)
    np.testing.assert_array_equal(nj, ex["n_jumps"])
    rel = []
    for i in range(EXACT_NTRAJ):
        k = min(int(nj[i]), 64)
        np.testing.assert_array_equal(jc[i, :k], ex["jump_ch"][i, :k])
        rel.append(np.abs(jt[i, :k] - ex["jump_t"][i, :k]) / np.maximum(1.0, ex["jump_t"][i, :k]))
    rel = np.concatenate(rel)
    assert rel.max() <= EXACT_TAU_MAX, rel.max()
    assert np.median(rel) <= EXACT_TAU_MEDIAN, np.median(rel)
    assert np.abs(obs - ex["obs"]).max() <= EXACT_OBS
    assert np.abs(mean - ex["mean"]).max() <= EXACT_ENSEMBLE


def test_proposal_refused_where_it_is_not_compiled():
    """Only the complex128 / double-float single-warp kernels carry the proposal."""
    prob = S.jaynes_cummings_driven()
    ctx = Q.qtm_create(prob, precision=Q.QTM_PREC_C64)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_proposal_collect(ctx, 8, 1)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)
    big = S.ising_chain(7)  # N = 128: a multi-warp lane layout
    ctx = Q.qtm_create(big, precision=Q.QTM_PREC_DF64)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_proposal_collect(ctx, 8, 1)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)
