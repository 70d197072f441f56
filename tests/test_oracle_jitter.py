"""Pins for the oracle's jitter schemes (Sec. 3.2.1), each against something
other than itself:

* the k-th prime against sympy's;
* radical inverses against the exact fraction of the reversed digits (Python
  integers), and the N-d Halton matrix against scipy's unscrambled Halton
  points; the inverse variant is the same matrix with its columns reversed;
* N-d primes and the golden-ratio sequence against a 50-digit evaluation of
  frac(n x) within the rounding bound of the FP64 evaluation;
* 1-d Sobol against scipy's unscrambled one-dimensional Sobol sequence;
* 1-d Halton in both orders of its J x K index matrix (particle-major, scheme
  1, and iteration-major, scheme 11) against scipy's unscrambled
  one-dimensional Halton sequence reshaped the two ways;
* uniform: a chi-square test; equidistant: every column a permutation of
  {1..J}/J, different per iteration; offset equidistant: within [0, 0.1) of
  it;
* the sampler's step counts follow the scheme.
"""
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle

getcontext().prec = 60


def test_primes_match_sympy():
    sympy = pytest.importorskip("sympy")
    for m in list(range(1, 200)) + [1000, 4096, 65536]:
        assert oracle.nth_prime(m) == int(sympy.prime(m))


def test_radical_inverse_exact_fraction():
    rng = np.random.default_rng(1)
    for _ in range(300):
        n = int(rng.integers(1, 2**30))
        b = int(rng.choice([2, 3, 5, 7, 11, 541, 7919, 821641]))
        num, den, x = 0, 1, n
        while x:
            num, den, x = num * b + x % b, den * b, x // b
        assert oracle.radical_inverse(n, b) == float(Fraction(num, den))


def test_halton_nd_matches_scipy_and_inverse_reverses():
    J, K = 64, 12
    H = oracle.jitter_matrix(oracle.JITTER["halton_nd"], 5, J, K)
    ref = stats.qmc.Halton(d=K, scramble=False).random(J + 1)[1:]
    np.testing.assert_allclose(H, ref, rtol=0, atol=1e-15)
    Hi = oracle.jitter_matrix(oracle.JITTER["halton_nd_inv"], 5, J, K)
    np.testing.assert_array_equal(Hi, H[:, ::-1])


def test_halton1_both_index_orders_match_scipy():
    J, K = 48, 10
    ref = stats.qmc.Halton(d=1, scramble=False).random(J * K + 1)[1:, 0]   # points n = 1 .. J K
    H1 = oracle.jitter_matrix(oracle.JITTER["halton1"], 5, J, K)
    np.testing.assert_array_equal(H1, ref.reshape(J, K))                # n = j K + k
    H11 = oracle.jitter_matrix(oracle.JITTER["halton1_iter"], 5, J, K)
    np.testing.assert_array_equal(H11, ref.reshape(K, J).T)             # n = (k - 1) J + j + 1
    # iteration-major: each iteration's J values are a stratified sample of (0, 1)
    for k in range(K):
        assert np.all(np.histogram(H11[:, k], bins=16, range=(0, 1))[0] == J // 16)


def _frac_hp(n, x_dec):
    v = Decimal(n) * x_dec
    return v - int(v)


@pytest.mark.parametrize("name", ["primes", "primes_inv", "golden"])
def test_kronecker_sequences_high_precision(name):
    J, K = 50, 9
    H = oracle.jitter_matrix(oracle.JITTER[name], 5, J, K)
    for j in range(J):
        for k in range(1, K + 1):
            if name == "golden":
                n, x = j * K + k, (Decimal(5).sqrt() - 1) / 2
            else:
                kk = k if name == "primes" else K + 1 - k
                n, x = j + 1, Decimal(oracle.nth_prime(kk)).sqrt()
            want = _frac_hp(n, x)
            # two FP64 roundings of x (sqrt, then the product n x): |err| <= 2^-52 n x
            bound = Decimal(2) ** -51 * n * x
            assert abs(Decimal(H[j, k - 1]) - want) <= bound, (name, j, k)
    if name == "primes_inv":
        np.testing.assert_array_equal(H, oracle.jitter_matrix(oracle.JITTER["primes"], 5, J, K)[:, ::-1])


def test_sobol1_matches_scipy():
    J, K = 16, 8
    H = oracle.jitter_matrix(oracle.JITTER["sobol1"], 5, J, K)
    seq = stats.qmc.Sobol(d=1, scramble=False).random_base2(8)[:, 0]
    for j in range(J):
        for k in range(1, K + 1):
            assert H[j, k - 1] == seq[j * K + k]


def test_uniform_and_equidistant():
    J, K = 500, 6
    U = oracle.jitter_matrix(oracle.JITTER["uniform"], 9, J, K)
    assert U.min() > 0 and U.max() < 1
    _, p = stats.chisquare(np.bincount((U.ravel() * 10).astype(int), minlength=10))
    assert p > 1e-4
    E = oracle.jitter_matrix(oracle.JITTER["equidistant"], 9, J, K)
    for k in range(K):
        np.testing.assert_array_equal(np.sort(E[:, k]), np.arange(1, J + 1) / J)
    assert not np.array_equal(E[:, 0], E[:, 1])
    O = oracle.jitter_matrix(oracle.JITTER["equidistant_offset"], 9, J, K)
    d = O - E
    assert d.min() >= 0 and d.max() < 0.1
    # a non-power-of-4 size exercises the cycle walk
    J2 = 37
    for k in (1, 2, 3):
        np.testing.assert_array_equal(np.sort([oracle.shuffle_index(3, k, j, J2) for j in range(J2)]),
                                      np.arange(J2))


@pytest.mark.parametrize("scheme", range(12))
def test_sampler_step_counts_follow_the_scheme(scheme):
    t = oracle.TargetSpec.gauss_dense(np.zeros(3), np.eye(3))
    cfg = oracle.SMCConfig(n_particles=64, n_iters=4, n_warmup=2, step_size=0.1, traj_len0=1.0,
                           max_steps=50, seed=13, jitter=scheme)
    st = oracle.smc_init(t, cfg)
    st["chees"] = oracle.initial_chees_state(cfg)
    for k in (1, 2):
        L = float(np.exp(st["chees"].log_L))
        out = oracle.smc_iteration(t, cfg, k, st)
        want = [oracle.step_count(oracle.jitter(scheme, 13, j, k, 64, 4), L, 0.1, 50) for j in range(64)]
        np.testing.assert_array_equal(out["steps"], want)
