"""The library's exact ensemble moments, on the host (no GPU needed).

The trajectory average of Sec. 3 is formed from integer sums of quantised values
(qtm_moments_of_values / qtm_combine_moments, the same rule the device reduction
applies).  Checked here against exact rational arithmetic (fractions.Fraction):
values that lie on the quantisation grid give sums equal to the exact sums and a
mean and standard error within an ulp or two of the exact ones -- including a
spread 1e-9 of the mean, where the one-pass formula sum x^2 - (sum x)^2/n in FP64
would lose every digit -- and any split into shards and any order of the shards
gives the same bits.
"""

import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S


def _exact(vals):
    """Exact mean, sample standard error, sum and sum of squares of 1-d values."""
    f = [Fraction(float(v)) for v in vals]
    n = len(f)
    s1 = sum(f, Fraction(0))
    s2 = sum((x * x for x in f), Fraction(0))
    mean = s1 / n
    var = (s2 - s1 * s1 / n) / (n - 1)
    return mean, math.sqrt(var / n), s1, s2


def _ulps(a, b):
    return abs(a - b) / math.ulp(abs(b)) if b != 0 else abs(a)


def _grid_values(rng, n, P, scale, mean=0.0, spread=1.0):
    """Values on the quantisation grid of exponent E (multiples of 2^(E-100)) whose
    squares are too: multiples of 2^-40 times `scale`."""
    x = mean + spread * rng.standard_normal((n, P))
    return np.round(x * 2.0 ** 40) / 2.0 ** 40 * scale


@pytest.mark.parametrize("n,P", [(1, 3), (2, 4), (7, 6), (300, 8), (5000, 2)])
def test_sums_and_moments_match_exact_arithmetic(n, P):
    rng = np.random.default_rng(n * 31 + P)
    E = np.array([3], np.int32)  # values below 2^2
    x = _grid_values(rng, n, P, 0.5)
    w = Q.qtm_moments_of_values(x, 1, E)
    mean, se, s, s2 = Q.qtm_combine_moments(w, [n], 1, E)
    for p in range(P):
        m_ex, se_ex, s1_ex, s2_ex = _exact(x[:, p]) if n > 1 else (Fraction(float(x[0, p])), 0.0,
                                                                      Fraction(float(x[0, p])),
                                                                      Fraction(float(x[0, p])) ** 2)
        assert s[p] == float(s1_ex)           # exact sum, correctly rounded
        assert s2[p] == float(s2_ex)
        assert _ulps(mean[p], float(m_ex)) <= 1.0
        if n > 1:
            assert _ulps(se[p], se_ex) <= 4.0, (se[p], se_ex)
        else:
            assert se[p] == 0.0


def test_small_spread_around_a_large_mean():
    """Mean 6, standard deviation 6e-9: sum x^2 - (sum x)^2/n cancels 17 digits,
    which FP64 does not hold; the integer form is exact, so the standard error
    keeps full precision."""
    rng = np.random.default_rng(5)
    n = 2000
    x = (6.0 + 6e-9 * rng.standard_normal((n, 1)))
    x = np.round(x * 2.0 ** 80) / 2.0 ** 80  # on the grid of E = 4 (quanta 2^-96); squares truncated by 2^-92
    E = np.array([4], np.int32)
    mean, se, _, _ = Q.qtm_combine_moments(Q.qtm_moments_of_values(x, 1, E), [n], 1, E)
    m_ex, se_ex, _, _ = _exact(x[:, 0])
    assert _ulps(mean[0], float(m_ex)) <= 1.0
    assert abs(se[0] - se_ex) <= 1e-12 * se_ex
    s1, s2 = x.sum(), (x * x).sum()
    one_pass = math.sqrt(max((s2 - s1 * s1 / n) / (n - 1), 0.0) / n)
    assert abs(one_pass - se_ex) > 1e-3 * se_ex  # what the identity would have given in FP64


def test_any_split_and_order_gives_the_same_bits():
    rng = np.random.default_rng(11)
    n, n_obs, n_t = 997, 3, 5
    x = rng.standard_normal((n, n_t, n_obs)) * np.array([0.3, 7.0, 100.0])
    E = np.array([4, 6, 10], np.int32)  # bounds 4, 16, 256 (well above every value here)
    x = np.clip(x, -3.9, 3.9) * np.array([1.0, 4.0, 60.0])
    ref = Q.qtm_combine_moments(Q.qtm_moments_of_values(x, n_obs, E), [n], n_obs, E)
    for shards in (2, 3, 8, 61):
        cuts = np.sort(rng.choice(np.arange(1, n), shards - 1, replace=False))
        parts = np.split(np.arange(n), cuts)
        words = [Q.qtm_moments_of_values(x[idx], n_obs, E) for idx in parts]
        counts = [len(idx) for idx in parts]
        order = rng.permutation(shards)
        got = Q.qtm_combine_moments(np.stack([words[i] for i in order]), [counts[i] for i in order], n_obs, E)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
    # and the values within one shard in any order
    perm = rng.permutation(n)
    got = Q.qtm_combine_moments(Q.qtm_moments_of_values(x[perm], n_obs, E), [n], n_obs, E)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_close_to_plain_fp64_on_general_values():
    """Values off the grid are truncated by under 2^-99 of the bound: the mean and
    standard error agree with numpy's FP64 ones to rounding."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.9, 0.95, (4000, 6))
    E = np.array([2], np.int32)
    mean, se, _, _ = Q.qtm_combine_moments(Q.qtm_moments_of_values(x, 1, E), [len(x)], 1, E)
    np.testing.assert_allclose(mean, x.mean(axis=0), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(se, x.std(axis=0, ddof=1) / np.sqrt(len(x)), rtol=1e-12)


def test_non_representable_values_make_the_output_nan():
    E = np.array([1], np.int32)  # values must lie below 2^1
    x = np.array([[0.5, 0.25, 1.0], [np.nan, 0.5, 1.0], [0.25, np.inf, 2.5]])
    w = Q.qtm_moments_of_values(x, 1, E)
    assert list(w[:, 8]) == [1, 1, 1]
    mean, se, s, s2 = Q.qtm_combine_moments(w, [3], 1, E)
    assert np.isnan(mean).all() and np.isnan(se).all() and np.isnan(s).all()


def test_empty_and_single_trajectory():
    E = np.array([2], np.int32)
    w = Q.qtm_moments_of_values(np.zeros((0, 4)), 1, E)
    mean, se, s, _ = Q.qtm_combine_moments(w, [0], 1, E)
    assert (mean == 0).all() and (se == 0).all() and (s == 0).all()
    w1 = Q.qtm_moments_of_values(np.full((1, 4), -1.5), 1, E)
    mean, se, _, _ = Q.qtm_combine_moments(np.stack([w, w1]), [0, 1], 1, E)
    assert (mean == -1.5).all() and (se == 0).all()


def test_scale_exponents_follow_the_observable_bound():
    """2^(E - 1) is the first power of two above max_i sum_j |Re A_ij| + |Im A_ij|,
    which bounds |<psi|A|psi>| / <psi|psi> for Hermitian A."""
    jc = S.jaynes_cummings_driven(n_fock=30)
    assert list(Q.qtm_scale_exponents(jc)) == [6, 2]          # a^dag a <= 29 < 32, sigma+sigma- <= 1 < 2
    two = S.two_level_driven()
    assert list(Q.qtm_scale_exponents(two)) == [2, 2]         # sigma+sigma-, sigma_x: bound 1
    z = two.with_(A=[sp.csr_matrix((2, 2), dtype=complex), sp.csr_matrix(np.diag([0.75, -0.75]))])
    assert list(Q.qtm_scale_exponents(z)) == [-400, 1]        # zero operator; bound 0.75 < 1
    dense = S.dense_random(ntraj=2, N=16)
    assert list(Q.qtm_scale_exponents(dense)) == [1]          # diag(0..15)/16 < 1


def test_argument_errors():
    E = np.array([2], np.int32)
    w = np.zeros((2, 9), np.int64)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_combine_moments(w, [-1], 1, E)
    assert ei.value.status == Q.QTM_ERR_ARG
    with pytest.raises(Q.QtmError):
        Q.qtm_combine_moments(w, [1], 1, np.array([999], np.int32))
    with pytest.raises(Q.QtmError):
        Q.qtm_moments_of_values(np.zeros((3, 5)), 2, np.array([2, 2], np.int32))  # 5 values, 2 observables
