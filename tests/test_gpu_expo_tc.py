"""The exponential method on the tensor cores (QTM_PREC_BF16X6 + QTM_METHOD_EXPONENTIAL),
run with ``-m gpu``.

On a uniform output grid every output interval of every trajectory starts with
the same product P_L psi (P_L = exp(M dt)), so the library advances all
trajectories of a run together: per interval one tcgen05 product forms
(P_L - I) psi for every column (both operands split into three bf16 terms, FP32
accumulation), y = psi + that is added in FP32, and a per-interval kernel
finishes each column in complex64 arithmetic -- the outputs, or, for a column
whose norm crosses its threshold, the crossing search on the ladder, the jump
and the propagation on to the output time (in a catch-up launch every sixteen
intervals, after which the column rejoins the lock step).

Bars: the complex64 ones against the exact oracle (expm between jumps, brentq
for the crossing) -- the same jump count for the bulk of the trajectories, the
median jump-time error within 1e-4, and the ensemble within its statistics of
the Lindblad solution.  (Forming P_L psi itself on the tensor cores gave a
median of 1e-3: their accumulation error, several times that of an FP32
product, meets the state once per interval; the increment form scales it by
||P_L - I|| and measured 1e-6 .. 1e-5.)
"""

import numpy as np
import pytest

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

from test_gpu_expo import MAXJ, exact_run, expo_run
from test_gpu_parity import _within_statistics

pytestmark = pytest.mark.gpu

TC = Q.QTM_PREC_BF16X6


def _jump_bars(g, o, same_frac=0.95, median=1e-4):
    same = g["n_jumps"] == o["n_jumps"]
    assert same.mean() >= same_frac, same.mean()
    dts = []
    for i in np.where(same)[0]:
        k = min(int(o["n_jumps"][i]), MAXJ)
        dts.append(np.abs(g["jump_t"][i, :k] - o["jump_t"][i, :k]))
    dts = np.concatenate(dts)
    print(f"\nsame jumps {same.mean():.3f}, median jump-time error {np.median(dts) if dts.size else 0:.2e}")
    if dts.size:
        assert np.median(dts) <= median, np.median(dts)
    assert g["stats"]["failed"] == 0


@pytest.mark.parametrize("name,kw,ntraj", [
    ("dense_random", dict(N=64, ntraj=100), 100),           # padded 64, layout 32 x 2
    ("dense_random", dict(N=100, ntraj=100), 100),          # padded 128, layout 64 x 2
    ("jaynes_cummings_driven", dict(), 200),                # sparse N = 60, many jumps
    ("purcell_qubit", dict(), 400),                         # stiff, N = 10
])
def test_against_exact_oracle_and_lindblad(orc, name, kw, ntraj):
    prob = S.by_name(name, **kw)
    g = expo_run(prob, ntraj, precision=TC)
    o = exact_run(prob, ntraj)
    _jump_bars(g, o)
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _within_statistics(g["mean"], g["se"], L, ntraj)
    # one product per output interval per trajectory, plus the ladder's
    assert g["stats"]["rhs_evals"] >= ntraj * (len(prob.t) - 1)


def test_dense_workload_size_against_exact_oracle():
    """N = 256 (layout 128 x 2, the full 512 x 512 real form on the tensor cores)."""
    prob = S.dense_random(ntraj=64)
    g = expo_run(prob, 64, precision=TC)
    o = exact_run(prob, 64)
    _jump_bars(g, o)
    assert np.abs(g["obs"] - o["obs"]).max() <= 0.05


def test_same_trajectories_as_the_simt_complex64_path():
    """The lock-step path and the per-trajectory complex64 kernel on the same
    Philox streams (2,000 ids of the dense workload): the same jumps for the bulk,
    the ensembles within a few 1e-4."""
    prob = S.dense_random(ntraj=2000)
    a = expo_run(prob, 2000, precision=Q.QTM_PREC_C64, record=8)
    b = expo_run(prob, 2000, precision=TC, record=8)
    assert np.mean(a["n_jumps"] == b["n_jumps"]) >= 0.98
    assert np.abs(a["mean"] - b["mean"]).max() <= 5e-4
    assert b["stats"]["failed"] == 0 and b["stats"]["jumps"] > 1000


def test_full_size_run_against_the_simt_complex64_path():
    """The dense workload at the bench's size (20,000 trajectories: 157 product
    tiles, so the last wave is split by output chunk, and about 18,000 deferred
    crossings over seven catch-up launches) against the per-trajectory complex64
    kernel on the same ids: the same jumps for the bulk, the ensembles within a
    few 1e-4, no failed trajectory, every output finite."""
    prob = S.dense_random(ntraj=20000)
    a = expo_run(prob, 20000, precision=Q.QTM_PREC_C64, record=4)
    b = expo_run(prob, 20000, precision=TC, record=4)
    assert np.mean(a["n_jumps"] == b["n_jumps"]) >= 0.98
    assert np.abs(a["mean"] - b["mean"]).max() <= 5e-4
    assert b["stats"]["failed"] == 0 and b["stats"]["jumps"] > 15000
    assert np.all(np.isfinite(b["obs"]))


@pytest.mark.parametrize("ntraj", [1, 127, 130, 300])
def test_ragged_column_counts(ntraj):
    """Partial 128-column tiles of the product and a partial last wave of the
    per-interval kernel: every trajectory equals its run inside a larger batch
    (each column's product depends on its own column only, and a deferred
    column's catch-up does not depend on which group takes it)."""
    prob = S.dense_random(N=64, ntraj=300)
    whole = expo_run(prob, 300, precision=TC, record=8)
    part = expo_run(prob, ntraj, precision=TC, record=8)
    np.testing.assert_array_equal(part["obs"], whole["obs"][:ntraj])
    np.testing.assert_array_equal(part["n_jumps"], whole["n_jumps"][:ntraj])


def test_bitwise_reproducible_and_switch_back():
    prob = S.dense_random(N=128, ntraj=200)
    a = expo_run(prob, 200, precision=TC, record=8)
    b = expo_run(prob, 200, precision=TC, record=8)
    np.testing.assert_array_equal(a["obs"], b["obs"])
    np.testing.assert_array_equal(a["jump_t"], b["jump_t"])
    # the same context back on Dormand-Prince reproduces a fresh engine run
    ref = Q.qtm_create(prob, precision=TC)
    Q.qtm_run(ref, 200, prob.seed)
    want = Q.qtm_traj_expect(ref)
    Q.qtm_destroy(ref)
    ctx = Q.qtm_create(prob, precision=TC)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    Q.qtm_run(ctx, 200, prob.seed)
    Q.qtm_expect(ctx)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_DOPRI5)
    Q.qtm_run(ctx, 200, prob.seed)
    np.testing.assert_array_equal(Q.qtm_traj_expect(ctx), want)
    Q.qtm_destroy(ctx)


def test_non_uniform_grid_is_refused():
    base = S.purcell_qubit()
    prob = base.with_(t=np.concatenate([base.t[:40], [4.05], base.t[41:]]))
    ctx = Q.qtm_create(prob, precision=TC)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)


def test_bounded_wait_reports_timeout_and_context_recovers():
    """A 1 ns bound makes the tensor-core product's first wait give up: the run
    reports QTM_ERR_TIMEOUT (no fault, no hang), and the same context then runs
    normally and reproduces a fresh run."""
    prob = S.dense_random(N=64, ntraj=150)
    ref = expo_run(prob, 150, precision=TC, record=0)
    ctx = Q.qtm_create(prob, precision=TC)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    Q.qtm_set_wait_limit(ctx, 1)
    Q.qtm_run(ctx, 150, prob.seed)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_expect(ctx)
    assert ei.value.status == Q.QTM_ERR_TIMEOUT
    Q.qtm_set_wait_limit(ctx, 0)
    Q.qtm_run(ctx, 150, prob.seed)
    np.testing.assert_array_equal(Q.qtm_traj_expect(ctx), ref["obs"])
    Q.qtm_destroy(ctx)


def test_product_time_is_reported():
    prob = S.dense_random(N=64, ntraj=300)
    g = expo_run(prob, 300, precision=TC, record=0)
    assert g["stats"]["product_ms"] > 0.0
