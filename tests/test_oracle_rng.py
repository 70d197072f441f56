"""Pins for the oracle's random numbers, Halton jitter and step counts.

Philox4x32-10 known-answer vectors are not available offline, so the generator
is pinned by what any correct counter-based generator must satisfy: output
words uniform over 32 bits and bytes, no serial correlation, a bijection on
counters (no collisions on a large sample), and avalanche (one flipped counter
bit changes about half of the 128 output bits).  The radical inverse is pinned
by the textbook van der Corput values and by its definition as a sum of
reversed binary digits, checked against exact rational arithmetic.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle


def _words(n, seed=1234, tag=2, k=7):
    out = np.empty((n, 4), dtype=np.uint32)
    for i in range(n):
        out[i] = oracle.philox((i % 97, i // 97, k, tag), seed)
    return out


def test_philox_byte_uniformity_chi2():
    w = _words(20000)
    b = w.view(np.uint8).ravel()
    counts = np.bincount(b, minlength=256)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4, (chi2, p)


def test_philox_bit_balance_and_serial_correlation():
    w = _words(20000).astype(np.float64).ravel() / 2.0**32
    assert abs(w.mean() - 0.5) < 0.005
    r = np.corrcoef(w[:-1], w[1:])[0, 1]
    assert abs(r) < 0.01


def test_philox_no_collisions_and_key_dependence():
    a = _words(5000, seed=1)
    b = _words(5000, seed=2)
    as_int = lambda m: {tuple(r) for r in m}
    assert len(as_int(a)) == 5000
    assert len(as_int(a) & as_int(b)) == 0


def test_philox_avalanche():
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(400):
        ctr = [int(x) for x in rng.integers(0, 2**32, size=4)]
        base = oracle.philox(ctr, 99)
        word, bit = rng.integers(0, 4), rng.integers(0, 32)
        ctr2 = list(ctr)
        ctr2[word] ^= 1 << int(bit)
        other = oracle.philox(ctr2, 99)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(base, other)))
    assert abs(np.mean(flips) - 64.0) < 2.0


def test_u01_open_interval_and_resolution():
    assert oracle.u01(0, 0) == 0.5 * 2.0**-52
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 0.5 * 2.0**-52
    assert 0.0 < oracle.u01(0, 0) < oracle.u01(0, 64) < 1.0


def test_normals_distribution():
    z = np.concatenate([oracle.normals(5, oracle.TAG_MOM, 3, j, 25) for j in range(2000)])
    ks = stats.kstest(z, "norm")
    assert ks.pvalue > 1e-3
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.03
    # streams for different (tag, k, j) are distinct
    assert not np.allclose(oracle.normals(5, 2, 3, 0, 4), oracle.normals(5, 2, 4, 0, 4))
    assert not np.allclose(oracle.normals(5, 1, 3, 0, 4), oracle.normals(5, 2, 3, 0, 4))


def test_halton_van_der_corput_textbook_values():
    # base-2 radical inverse: 1 -> 1/2, 2 -> 1/4, 3 -> 3/4, 4 -> 1/8, 5 -> 5/8, 6 -> 3/8
    expect = [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875, 0.0625]
    assert [oracle.halton2(n) for n in range(1, 9)] == expect
    assert oracle.halton2(0) == 0.0


@pytest.mark.parametrize("n", [9, 1000, 123456789, 2**31 + 12345, 2**32 - 1])
def test_halton_equals_exact_digit_reversal(n):
    digits = bin(n)[2:][::-1]
    exact = sum(Fraction(int(d), 2 ** (i + 1)) for i, d in enumerate(digits))
    assert oracle.halton2(n) == float(exact)


def test_step_count_ceil_and_clip():
    # ceil(h L / eps) for values away from rounding boundaries
    assert oracle.step_count(0.5, 1.0, 0.1, 500) == 5
    assert oracle.step_count(0.51, 1.0, 0.1, 500) == 6
    assert oracle.step_count(0.75, 5.0, 0.001, 500) == 500       # clipped at the cap
    assert oracle.step_count(1e-9, 1.0, 0.1, 500) == 1           # at least one step
    assert oracle.step_count(float("nan"), 1.0, 0.1, 500) == 1
    rng = np.random.default_rng(3)
    for _ in range(200):
        h, L = rng.uniform(), rng.uniform(0.01, 3.0)
        s = oracle.step_count(h, L, 0.01, 10**6)
        assert s == max(1, math.ceil((h * L) / 0.01))
