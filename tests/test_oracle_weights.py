"""Pins for the oracle's weights, ESS and fixed-point resampling (Sec. 3).

* log-sum-exp against scipy.special.logsumexp; ESS = N for equal weights,
  1 for a one-hot vector, 2 for two equal weights among zeros;
* systematic resampling: offspring of j lie in {floor(N q_j/T), ceil(N q_j/T)},
  they sum to N, ancestors are non-decreasing, and -- the exact expectation --
  summed over every distinct offset U in [0, T) the offspring of j equal
  N q_j exactly (brute force over all U on tiny inputs);
* multinomial resampling: P(ancestor = j) = q_j / T by brute-force enumeration
  of every position and a chi-square test on random draws.
"""
import numpy as np
import pytest
from scipy import special, stats

import oracle


def test_normalise_matches_scipy_and_special_cases():
    rng = np.random.default_rng(0)
    lw = rng.standard_normal(1000) * 30.0 - 500.0
    lse, ess, W = oracle.normalise(lw)
    assert abs(lse - special.logsumexp(lw)) < 1e-9
    np.testing.assert_allclose(W, np.exp(lw - special.logsumexp(lw)), rtol=1e-12)
    assert abs(ess - 1.0 / np.sum(W**2)) < 1e-9 * ess
    assert abs(oracle.normalise(np.full(77, -3.0))[1] - 77.0) < 1e-9
    one_hot = np.full(50, -np.inf)
    one_hot[13] = 4.0
    lse, ess, W = oracle.normalise(one_hot)
    assert lse == 4.0 and ess == 1.0 and W[13] == 1.0
    # two equal weights and two zeros: ESS 2
    assert abs(oracle.normalise(np.array([0.0, 0.0, -np.inf, -np.inf]))[1] - 2.0) < 1e-12
    lse, ess, _ = oracle.normalise(np.full(5, -np.inf))
    assert lse == -np.inf and ess == 0.0


def test_quantise_scale_and_floor():
    W = np.array([0.5, 0.25, 0.125, 0.125])
    S, q = oracle.quantise(W)
    assert S == 62 - 2
    assert list(q) == [2**59, 2**58, 2**57, 2**57]
    S, q = oracle.quantise(np.array([1.0 / 3, 2.0 / 3, 0.0]))
    assert S == 60 and q[2] == 0 and int(q[0]) == int(np.floor((1.0 / 3) * 2.0**60))


def _offspring(anc, N):
    return np.bincount(anc, minlength=N)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 64, 1000])
def test_systematic_offspring_bounds(N):
    rng = np.random.default_rng(N)
    W = rng.gamma(0.3, size=N)
    W /= W.sum()
    _, q = oracle.quantise(W)
    for trial in range(5):
        r64 = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        T, anc = oracle.systematic(q, r64)
        assert T == int(q.astype(object).sum())
        o = _offspring(anc, N)
        assert o.sum() == N
        assert np.all(np.diff(anc) >= 0)
        exact = [int(qj) * N for qj in q]
        lo = [e // T for e in exact]
        hi = [-(-e // T) for e in exact]
        assert all(l <= oj <= h for l, oj, h in zip(lo, o, hi))


def test_systematic_exact_expectation_over_all_offsets():
    # tiny integer weights so that every offset U in [0, T) can be enumerated
    for q_list in ([1, 3, 0, 4], [5, 0, 0, 2, 1], [1, 1, 1], [7]):
        q = np.array(q_list, dtype=np.uint64)
        N, T = len(q_list), sum(q_list)
        total = np.zeros(N, dtype=np.int64)
        for U in range(T):
            r64 = -(-(U << 64) // T)             # smallest r64 with floor(r64 T / 2^64) = U
            T2, anc = oracle.systematic(q, r64)
            assert T2 == T
            total += _offspring(anc, N)
        assert list(total) == [N * x for x in q_list]


def test_systematic_extreme_offsets():
    q = np.array([3, 1], dtype=np.uint64)
    _, anc = oracle.systematic(q, 0)
    assert list(anc) == [0, 0]
    _, anc = oracle.systematic(q, 2**64 - 1)
    assert list(anc) == [0, 1]


def test_multinomial_brute_force_probabilities():
    q = np.array([1, 0, 3, 4], dtype=np.uint64)
    T, C = 8, np.cumsum([1, 0, 3, 4])
    counts = np.zeros(4, dtype=np.int64)
    for P in range(T):
        u = -(-(P << 64) // T)
        a = oracle.multinomial(q, np.array([u] * 4, dtype=np.uint64))[0]
        assert C[a] > P and (a == 0 or C[a - 1] <= P)
        counts[a] += 1
    assert list(counts) == [1, 0, 3, 4]
    rng = np.random.default_rng(9)
    u = rng.integers(0, 2**63, size=40000, dtype=np.uint64) * np.uint64(2)
    anc = np.concatenate([oracle.multinomial(q, u[i:i + 4]) for i in range(0, 40000, 4)])
    obs = np.bincount(anc, minlength=4)
    assert obs[1] == 0
    chi2, p = stats.chisquare(obs[[0, 2, 3]], 40000 * np.array([1, 3, 4]) / 8)
    assert p > 1e-4


def test_moments_weighted():
    rng = np.random.default_rng(1)
    th = rng.standard_normal((500, 3))
    lw = rng.standard_normal(500)
    W = np.exp(lw - special.logsumexp(lw))
    m, v = oracle.moments(th, lw)
    np.testing.assert_allclose(m, W @ th, rtol=1e-12)
    np.testing.assert_allclose(v, W @ (th - m) ** 2, rtol=1e-12)


def test_moments_leave_out_zero_weight_particles():
    """A particle of weight zero (possibly at a non-finite position after a
    divergent trajectory) does not enter the estimates."""
    rng = np.random.default_rng(2)
    th = rng.standard_normal((50, 2))
    lw = rng.standard_normal(50)
    m, v = oracle.moments(th, lw)
    th2 = np.vstack([th, [[np.nan, np.inf]]])
    lw2 = np.concatenate([lw, [-np.inf]])
    m2, v2 = oracle.moments(th2, lw2)
    np.testing.assert_array_equal(m2, m)
    np.testing.assert_array_equal(v2, v)
