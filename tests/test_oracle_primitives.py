"""Pins for the oracle's random stream and arithmetic primitives.

Philox4x32-10 is pinned to the published known-answer values; the uniform
mapping to its exact end points; the logarithm to a correctly rounded
reference (mpmath at 120 bits); the bounded-integer routine to uniformity,
including the residue pattern a multiply-shift without rejection would show.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert orc.philox4x32_10(ctr, key) == want


def test_philox_counter_sensitivity(orc):
    # every counter word and key word changes the output
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert orc.philox4x32_10(c, [5, 6]) != base
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert orc.philox4x32_10([1, 2, 3, 4], k) != base


def test_u01_end_points_and_open_interval(orc):
    assert orc.u01(0, 0) == 2.0 ** -53
    assert orc.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # the low 12 bits of the first word are discarded
    assert orc.u01(0xFFF, 0) == orc.u01(0, 0)
    assert orc.u01(0x1000, 0) == 3.0 * 2.0 ** -53
    # the second word supplies the high 32 of the 52 bits
    assert orc.u01(0, 1) == (2.0 ** 20 + 0.5) * 2.0 ** -52
    rng = np.random.default_rng(5)
    a = rng.integers(0, 2 ** 32, 2000)
    b = rng.integers(0, 2 ** 32, 2000)
    for x, y in zip(a, b):
        r = orc.u01(x, y)
        assert 0.0 < r < 1.0
        k = (int(y) << 20) | (int(x) >> 12)
        assert r == (k + 0.5) / 2.0 ** 52


def test_log_is_within_one_ulp_of_correct_rounding(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    rng = np.random.default_rng(11)
    xs = list(rng.random(3000)) + list(np.exp(rng.uniform(-700, 700, 2000)))
    xs += [2.0 ** -53, 1.0 - 2.0 ** -53, 0.5, 2.0, 1.4142135623730951,
           0.7071067811865476, 1e-300, 5e-324, 1.7976931348623157e308]
    worst = 0.0
    for x in xs:
        y = orc.log(x)
        ref = float(mpmath.log(mpmath.mpf(float(x))))
        worst = max(worst, abs(y - ref) / math.ulp(ref))
    assert worst <= 1.0


def test_log_special_values(orc):
    assert orc.log(1.0) == 0.0
    assert orc.log(0.0) == -math.inf
    assert math.isnan(orc.log(-1.0))
    assert orc.log(math.inf) == math.inf
    for k in (-1074, -60, -1, 1, 7, 1023):
        y = orc.log(2.0 ** k)
        assert abs(y - k * math.log(2.0)) <= math.ulp(k * math.log(2.0))
    # monotone on a fine grid around 1
    xs = np.linspace(0.5, 2.0, 20001)
    ys = np.array([orc.log(x) for x in xs])
    assert np.all(np.diff(ys) > 0)


def test_bounded_range_one_is_zero(orc):
    out = orc.bounded_sequence(7, 3, 0, np.ones(50, dtype=np.uint32))
    assert np.all(out == 0)


def test_bounded_uniform_small_range(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    # 6000 draws of range 6 spread over 1000 independent event streams
    counts = np.zeros(6)
    for e in range(1000):
        out = orc.bounded_sequence(99, e, 0, np.full(6, 6, dtype=np.uint32))
        assert np.all(out < 6)
        counts += np.bincount(out, minlength=6)
    p = scipy_stats.chisquare(counts).pvalue
    assert p > 1e-3


def test_bounded_rejects_multiply_shift_bias(orc):
    # For s = 3 * 2^30 a multiply-shift without rejection returns values
    # divisible by 3 with probability 1/2; an unbiased routine gives 1/3.
    s = 3 * 2 ** 30
    res = []
    for e in range(400):
        res.append(orc.bounded_sequence(1234, e, 2, np.full(25, s, dtype=np.uint32)))
    res = np.concatenate(res)
    assert np.all(res < s)
    frac0 = np.mean(res % 3 == 0)
    se = math.sqrt((1 / 3) * (2 / 3) / res.size)
    assert abs(frac0 - 1 / 3) < 5 * se


def test_bounded_streams_depend_on_event_and_replicate(orc):
    r = np.full(8, 1000, dtype=np.uint32)
    a = orc.bounded_sequence(1, 0, 0, r)
    assert not np.array_equal(a, orc.bounded_sequence(1, 1, 0, r))
    assert not np.array_equal(a, orc.bounded_sequence(1, 0, 1, r))
    assert not np.array_equal(a, orc.bounded_sequence(2, 0, 0, r))
    assert np.array_equal(a, orc.bounded_sequence(1, 0, 0, r))
