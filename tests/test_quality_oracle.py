"""Pins of the oracle's statistics for the paper's tests 35 and 100 (Sec. 4.2)
and of the host-side chi-square helpers.

Every expected value here is constructed by hand (sequences whose visits or
block weights are placed on purpose) or follows from a closed form, so a
dropped term, an off-by-one in the gap count or a wrong bit field fails one
of them.
"""
import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import quality

NO_VISIT = np.uint32(0xFFFFFFFF)   # every field bit set


def _seq(n, visits):
    x = np.full(n, NO_VISIT, np.uint32)
    x[list(visits)] = 0
    return x


def test_gap_constructed_positions():
    # visits at 0, 5, 6, 40, 1000: gaps 0 (nothing before index 0), 4, 0, 33, 959
    h = oracle.gap_histogram(_seq(1200, [0, 5, 6, 40, 1000]), t=64)
    expect = np.zeros(65, np.uint64)
    expect[0] = 2
    expect[4] = 1
    expect[33] = 1
    expect[64] = 1          # 959 >= t
    np.testing.assert_array_equal(h, expect)


def test_gap_trailing_run_is_not_a_gap():
    h = oracle.gap_histogram(_seq(100, [10]), t=32)
    assert h.sum() == 1 and h[10] == 1
    assert oracle.gap_histogram(_seq(100, []), t=32).sum() == 0


def test_gap_bit_field():
    """r = 25, b = 5: u = (x * 2^25 mod 2^32) / 2^32 < 1/32 exactly when
    bits 6..2 of x are zero; bits 31..7 (dropped) and 1..0 (below the field)
    do not matter."""
    x = np.array([1 << 2, 1 << 6, 1 << 1, 1 << 7, (1 << 31) | 3, 0x7C, 0x80], np.uint32)
    visits = [not (v & 0x7C) for v in x.tolist()]
    assert visits == [False, False, True, True, True, False, True]
    # gaps: index 2 -> 2, index 3 -> 0, index 4 -> 0, index 6 -> 1
    h = oracle.gap_histogram(x, r=25, b=5, t=8)
    np.testing.assert_array_equal(h[:3], [2, 1, 1])
    assert h.sum() == 4
    # r = 0, b = 1: visit iff the top bit is clear; visits at 1 and 3, one
    # non-visit before each
    h = oracle.gap_histogram(np.array([0x80000000, 0x7FFFFFFF, 0x80000000, 0], np.uint32), r=0, b=1, t=4)
    np.testing.assert_array_equal(h, [0, 2, 0, 0, 0])


@pytest.mark.parametrize("k", [1, 2, 7, 32, 100])
def test_gap_period_k(k):
    """A visit at every k-th value: n // k gaps, all of length k - 1."""
    n = 5000
    x = _seq(n, [j for j in range(n) if j % k == k - 1])
    h = oracle.gap_histogram(x, t=64)
    assert h.sum() == n // k
    assert h[min(k - 1, 64)] == n // k


def test_gap_lengths_add_up():
    """With t beyond every gap: sum over gaps of (length + 1) equals the index
    of the last visit plus one."""
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    h = oracle.gap_histogram(x, t=4096)
    assert h[4096] == 0
    last = np.nonzero((x & 0x7C) == 0)[0][-1]
    assert int(np.sum((np.arange(4096) + 1) * h[:4096])) == last + 1


def test_hamming_constant_and_alternating_blocks():
    L, per = 1200, 240
    bounds = [590, 600, 610]
    zeros = np.zeros(per, np.uint32)
    ones = np.full(per, 0x7C, np.uint32)        # the 5-bit field all ones: weight L
    t = oracle.hamming_pairs(np.concatenate([zeros] * 6), bounds=bounds)
    assert t[0, 0] == 3 and t.sum() == 3
    t = oracle.hamming_pairs(np.concatenate([ones] * 4), bounds=bounds)
    assert t[3, 3] == 2 and t.sum() == 2
    t = oracle.hamming_pairs(np.concatenate([zeros, ones, ones, zeros, zeros, ones]), bounds=bounds)
    assert t[0, 3] == 2 and t[3, 0] == 1 and t.sum() == 3
    assert L == 5 * per


def _block_of_weight(w, per=240, s=5):
    """per outputs whose s-bit fields hold exactly w ones in total."""
    x = np.zeros(per, np.uint32)
    for k in range(w):
        j, bit = divmod(k, s)
        x[j] |= np.uint32(1 << (2 + bit))      # bits 2..6 = the field for r = 25
    return x


def test_hamming_classes_follow_the_bounds():
    bounds = [590, 600, 610]
    pairs = [(589, 590), (599, 600), (609, 610), (0, 1200)]
    x = np.concatenate([np.concatenate([_block_of_weight(a), _block_of_weight(b)]) for a, b in pairs])
    t = oracle.hamming_pairs(x, bounds=bounds)
    expect = np.zeros((4, 4), np.uint64)
    for a, b in pairs:
        ca = sum(1 for q in bounds if q <= a)
        cb = sum(1 for q in bounds if q <= b)
        expect[ca, cb] += 1
    np.testing.assert_array_equal(t, expect)
    assert expect[0, 1] == 1 and expect[1, 2] == 1 and expect[2, 3] == 1 and expect[0, 3] == 1


def test_hamming_pairs_count_and_bits_outside_the_field():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 2 ** 32, 240 * 9 + 17, dtype=np.uint64).astype(np.uint32)
    t = oracle.hamming_pairs(x, bounds=[600])
    assert t.sum() == 4            # 9 complete blocks -> 4 complete pairs
    # bits outside the 5-bit field (31..7 and 1..0) do not change anything
    ref = oracle.hamming_pairs(x & np.uint32(0x7C), bounds=[600])
    np.testing.assert_array_equal(oracle.hamming_pairs(x | np.uint32(0xFFFFFF83), bounds=[600]), ref)
    np.testing.assert_array_equal(oracle.hamming_pairs(x, bounds=[600]), ref)


def test_probability_helpers():
    p = quality.gap_probabilities(5, 100)
    assert p.size == 101 and abs(p.sum() - 1.0) < 1e-12
    assert abs(p[0] - 1 / 32) < 1e-15 and abs(p[1] - 31 / 1024) < 1e-15
    q = quality.binomial_class_probabilities(1200, quality.default_hamming_bounds(1200, 4))
    assert abs(q.sum() - 1.0) < 1e-12 and np.all(np.abs(q - 0.25) < 0.03)
    # Binomial(4, 1/2) with bounds [1, 3]: classes {0}, {1, 2}, {3, 4}
    np.testing.assert_allclose(quality.binomial_class_probabilities(4, [1, 3]),
                               [1 / 16, 10 / 16, 5 / 16])


def test_chi2_accepts_an_independent_generator_and_rejects_a_biased_one():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(2024)
    x = rng.integers(0, 2 ** 32, 4_000_000, dtype=np.uint64).astype(np.uint32)
    g = quality.gap_test(oracle.gap_histogram(x, t=128), b=5)
    bounds = quality.default_hamming_bounds(1200, 4)
    h = quality.hamming_test(oracle.hamming_pairs(x, bounds=bounds), L=1200, bounds=bounds)
    assert g["p_value"] > 1e-6 and h["p_value"] > 1e-6
    # too regular: a visit exactly every 32 values
    biased = np.full(400000, NO_VISIT, np.uint32)
    biased[31::32] = 0
    assert quality.gap_test(oracle.gap_histogram(biased, t=128), b=5)["p_value"] < 1e-12
    # dependent successive blocks: each block repeats the one before it
    rep = np.repeat(x[:240 * 2000].reshape(2000, 240), 2, axis=0).ravel()
    hd = quality.hamming_test(oracle.hamming_pairs(rep, bounds=bounds), L=1200, bounds=bounds)
    assert hd["p_value"] < 1e-12
