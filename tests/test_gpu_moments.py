"""The exact ensemble moments on the GPU (run with ``-m gpu``): the device
reduction applies the same quantisation rule as the host (its words equal
qtm_moments_of_values of the run's own per-trajectory values, bit for bit), so
qtm_expect / qtm_sums equal the host combination of those words, and shards run
with qtm_run_range combine to exactly the bits of one run over all ids -- the
two-level average of Sec. 3 without any dependence on how the ensemble was cut."""

import numpy as np
import pytest

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [Q.QTM_PREC_C128, Q.QTM_PREC_DF64, Q.QTM_PREC_C64])
@pytest.mark.parametrize("ntraj", [1, 5, 200, 1537])
def test_device_words_follow_the_host_rule(prec, ntraj):
    prob = S.jaynes_cummings_driven(n_t=81, t_end=8.0)
    ctx = Q.qtm_create(prob, precision=prec)
    Q.qtm_run(ctx, ntraj, 1)
    w, n, E = Q.qtm_moments(ctx)
    vals = Q.qtm_traj_expect(ctx)
    mean, se = Q.qtm_expect(ctx)
    s1, s2, _ = Q.qtm_sums(ctx)
    Q.qtm_destroy(ctx)
    assert n == ntraj
    np.testing.assert_array_equal(E, Q.qtm_scale_exponents(prob))
    np.testing.assert_array_equal(w, Q.qtm_moments_of_values(vals, len(prob.A), E))
    cm, cse, cs1, cs2 = Q.qtm_combine_moments(w, [n], len(prob.A), E)
    np.testing.assert_array_equal(mean.ravel(), cm)
    np.testing.assert_array_equal(se.ravel(), cse)
    np.testing.assert_array_equal(s1.ravel(), cs1)
    np.testing.assert_array_equal(s2.ravel(), cs2)
    # and the plain FP64 statistics of the same values to rounding
    np.testing.assert_allclose(mean, vals.mean(axis=0), rtol=1e-13, atol=1e-15)
    if ntraj > 1:
        np.testing.assert_allclose(se, vals.std(axis=0, ddof=1) / np.sqrt(ntraj), rtol=1e-10, atol=1e-15)


def test_shards_combine_to_the_single_run_bitwise():
    prob = S.jaynes_cummings_driven(n_t=101, t_end=10.0)
    ntraj = 3001
    ctx = Q.qtm_create(prob, precision=Q.QTM_PREC_DF64)
    Q.qtm_run(ctx, ntraj, 1)
    mean, se = Q.qtm_expect(ctx)
    E = Q.qtm_moments(ctx)[2]
    for cuts in ((1500,), (7, 1000, 2999), (128, 256, 384, 2048)):
        bounds = [0, *cuts, ntraj]
        words, counts = [], []
        for a, b in zip(bounds[:-1], bounds[1:]):
            Q.qtm_run_range(ctx, a, b - a, 1)
            w, n, _ = Q.qtm_moments(ctx)
            words.append(w)
            counts.append(n)
        cm, cse, _, _ = Q.qtm_combine_moments(np.stack(words[::-1]), counts[::-1], len(prob.A), E)
        np.testing.assert_array_equal(cm, mean.ravel())
        np.testing.assert_array_equal(cse, se.ravel())
    Q.qtm_destroy(ctx)


def test_device_copy_of_the_words_for_a_collective():
    torch = pytest.importorskip("torch")
    prob = S.jaynes_cummings_driven(n_t=41, t_end=4.0)
    ctx = Q.qtm_create(prob, stream=Q.current_stream(), precision=Q.QTM_PREC_DF64)
    Q.qtm_run(ctx, 300, 1)
    P = len(prob.t) * len(prob.A)
    dev = torch.zeros((P, Q.QTM_MOMENT_WORDS), dtype=torch.int64, device="cuda")
    Q.qtm_moments_device(ctx, dev.data_ptr())
    torch.cuda.synchronize()
    w, _, _ = Q.qtm_moments(ctx)
    np.testing.assert_array_equal(dev.cpu().numpy(), w)
    Q.qtm_destroy(ctx)


def test_failed_trajectories_make_the_mean_nan():
    """A trajectory that stops (here: the step limit) leaves NaN outputs; they are
    counted as non-representable and the affected means are NaN, as before."""
    prob = S.jaynes_cummings_driven(n_t=41, t_end=4.0).with_(max_steps=20)
    ctx = Q.qtm_create(prob)
    Q.qtm_run(ctx, 8, 1)
    with pytest.raises(Q.QtmError):
        Q.qtm_expect(ctx)
    mean, _ = Q.qtm_expect(ctx, check=False)
    assert np.isnan(mean[-1]).all() and np.isfinite(mean[0]).all()
    Q.qtm_destroy(ctx)
