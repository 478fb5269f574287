"""The learned proposal inside the exponential method's crossing search (run with
``-m gpu``).

Pairs come from the exponential method itself (one per crossing: the features of
the output interval that contains it, and the time from the interval's start to
the crossing); the network, trained by the library's kernels, corrects the
constant-rate estimate of that time; the search then tries the ladder bracket that
holds the prediction first.  The root find still decides every crossing, so the
jumps are those of the search without a prediction -- bit for bit where the
bracket was hit, since the bracket's state is formed by the same products in the
same order -- and the products per trajectory fall.  Checked against the exact
oracle (expm between jumps, brentq) with the exponential method's bars.
"""

import numpy as np
import pytest

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

from test_gpu_expo import MAXJ, compare_exact, exact_run

pytestmark = pytest.mark.gpu


def _expo_ctx(prob, prec, params=None, on=False):
    ctx = Q.qtm_create(prob, precision=prec, record_jumps=MAXJ)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    if params is not None:
        Q.qtm_proposal_set(ctx, params)
        Q.qtm_proposal_enable(ctx, on)
    return ctx


def _run(prob, ntraj, prec, params=None, on=False):
    ctx = _expo_ctx(prob, prec, params, on)
    Q.qtm_run(ctx, ntraj, prob.seed)
    mean, se = Q.qtm_expect(ctx)
    out = dict(mean=mean, se=se, obs=Q.qtm_traj_expect(ctx), stats=Q.qtm_stats(ctx))
    out["n_jumps"], out["jump_t"], out["jump_ch"] = Q.qtm_jumps(ctx)
    Q.qtm_destroy(ctx)
    return out


@pytest.fixture(scope="module")
def trained_expo():
    """Pairs from 4,000 JC trajectories of the exponential method (seed 11), trained on the GPU."""
    prob = S.jaynes_cummings_driven()
    ctx = _expo_ctx(prob, Q.QTM_PREC_DF64)
    npairs = Q.qtm_proposal_collect(ctx, 4000, 11, stride=1, max_per_traj=96)
    f, dt = Q.qtm_proposal_pairs(ctx, npairs)
    loss, base = Q.qtm_proposal_train(ctx, steps=1500, batch=4096, lr=2e-3, seed=11)
    params = Q.qtm_proposal_get(ctx)
    Q.qtm_destroy(ctx)
    return dict(prob=prob, npairs=npairs, f=f, dt=dt, loss=loss, base=base, params=params)


def test_expo_pairs_are_consistent(trained_expo):
    f, dt = trained_expo["f"], trained_expo["dt"]
    prob = trained_expo["prob"]
    spacing = float(prob.t[1] - prob.t[0])
    assert trained_expo["npairs"] > 100000                     # ~39 crossings per trajectory
    assert np.all(f[:, 0] > 0) and np.all(dt > 0) and np.all(dt <= spacing * (1 + 1e-6))
    assert np.all(np.log(f[:, 2]) >= f[:, 3] - 1e-6)           # the norm is still above r at the start
    est = (np.log(f[:, 2]) - f[:, 3]) / f[:, 0]
    # the constant-rate estimate within the interval is already close: the network corrects it
    assert np.median(np.abs(np.log(dt / est))) < 0.2
    assert np.isfinite(trained_expo["loss"]) and trained_expo["loss"] <= trained_expo["base"]


# on-vs-off bar per arithmetic: a missed bracket forms the bracket's state through
# another product sequence, which moves a crossing by the arithmetic's rounding
# (measured ~1e-12 for double-float, whose unit round-off is about 2^-48)
ON_OFF_TAU = {Q.QTM_PREC_C128: 1e-12, Q.QTM_PREC_DF64: 1e-10}


@pytest.mark.parametrize("prec", [Q.QTM_PREC_C128, Q.QTM_PREC_DF64], ids=["c128", "df64"])
def test_expo_proposal_same_jumps_fewer_products(trained_expo, prec, capsys):
    prob, params = trained_expo["prob"], trained_expo["params"]
    n = 2000
    off = _run(prob, n, prec, params, on=False)
    on = _run(prob, n, prec, params, on=True)
    jumps = on["stats"]["jumps"]
    misses = on["stats"]["proposal_misses"]
    p_off = off["stats"]["rhs_evals"] / n
    p_on = on["stats"]["rhs_evals"] / n
    same, total, worst = 0, 0, 0.0
    for i in range(n):
        k = min(int(off["n_jumps"][i]), MAXJ, int(on["n_jumps"][i]))
        tau = off["jump_t"][i, :k]
        dt = np.abs(on["jump_t"][i, :k] - tau)
        same += int((dt == 0).sum())
        total += k
        if k:
            worst = max(worst, float((dt / np.maximum(1.0, tau)).max()))
    with capsys.disabled():
        print(f"\nexponential method + proposal ({'c128' if prec == Q.QTM_PREC_C128 else 'df64'}): products per "
              f"trajectory {p_off:.1f} -> {p_on:.1f} ({100 * (p_off - p_on) / p_off:+.2f} %), bracket hits "
              f"{100 * (1 - misses / max(jumps, 1)):.1f} %, jump times bitwise equal "
              f"{100 * same / max(total, 1):.1f} %, largest relative difference {worst:.2e}, loss "
              f"{trained_expo['loss']:.3e} vs constant-rate {trained_expo['base']:.3e}")
    np.testing.assert_array_equal(on["n_jumps"], off["n_jumps"])
    for i in range(n):
        k = min(int(off["n_jumps"][i]), MAXJ)
        np.testing.assert_array_equal(on["jump_ch"][i, :k], off["jump_ch"][i, :k])
    assert worst <= ON_OFF_TAU[prec], worst
    assert np.abs(on["mean"] - off["mean"]).max() <= 1e-12
    assert p_on < p_off
    assert misses < 0.5 * jumps
    assert same >= 0.5 * total


@pytest.mark.parametrize("prec", [Q.QTM_PREC_C128, Q.QTM_PREC_DF64], ids=["c128", "df64"])
def test_expo_proposal_against_exact_oracle(trained_expo, prec):
    prob = trained_expo["prob"]
    ntraj = 64
    g = _run(prob, ntraj, prec, trained_expo["params"], on=True)
    o = exact_run(prob, ntraj)
    compare_exact(g, o, ntraj, prec)


def test_expo_proposal_refused_where_it_is_not_compiled():
    prob = S.jaynes_cummings_driven()
    ctx = _expo_ctx(prob, Q.QTM_PREC_C64)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_proposal_collect(ctx, 8, 1)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)
