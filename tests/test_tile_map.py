"""The FP32 kernels split a tile index t into (row, column) = divmod(t, d)
without an integer division: q = trunc(rn(t * rn(1 / d))) in single
precision, then one correction step.  The same arithmetic in numpy float32
(IEEE single, round to nearest like the device's __frcp_rn and __fmul_rn)
must give divmod exactly for every 0 <= t < 2^24 and d >= 1, the range the
library admits (it refuses grids of 2^24 tiles or more).

Bound: t and 1/d are each off by at most a relative 2^-24 after rounding,
so the estimate of t / d is off by less than (t / d) 2^-23 < 2 / d, i.e. by
less than one for d >= 2 (d = 1 is exact): one correction suffices."""
import numpy as np


def split(t, d):
    f32 = np.float32
    inv = f32(1.0) / f32(d)
    q = np.trunc(f32(t) * inv).astype(np.int64)
    r = t - q * d
    lo = r < 0
    hi = r >= d
    q = np.where(lo, q - 1, np.where(hi, q + 1, q))
    r = np.where(lo, r + d, np.where(hi, r - d, r))
    return q, r


def _check(t, d):
    q, r = split(t, d)
    qe, re = np.divmod(t, d)
    bad = np.nonzero((q != qe) | (r != re))[0]
    assert bad.size == 0, (d, t[bad[:5]], q[bad[:5]], qe[bad[:5]])


def test_exact_near_every_multiple_below_2_24():
    # the estimate is least accurate right at and beside multiples of d, and
    # at the top of the range; check those for many divisors, including the
    # tile-column counts of power-of-two grids (2^k / 32 + 1)
    top = 1 << 24
    divisors = list(range(1, 300)) + [2 ** k // 32 + 1 for k in range(5, 20)] + [4099, 65537, 1 << 20, top - 1]
    for d in divisors:
        k = np.arange(0, top // d + 1, max(1, (top // d) // 4096), dtype=np.int64)
        t = np.concatenate([k * d - 1, k * d, k * d + 1, np.arange(top - 64, top, dtype=np.int64)])
        t = t[(t >= 0) & (t < top)]
        _check(t, d)


def test_exact_on_random_pairs():
    rng = np.random.default_rng(24)
    for _ in range(20):
        d = int(rng.integers(1, 1 << 20))
        t = rng.integers(0, 1 << 24, size=200_000, dtype=np.int64)
        _check(t, d)


def test_fails_above_the_admitted_range():
    # above 2^24 the single-precision image of t is no longer exact and the
    # quotient estimate can be off by more than one: the library's limit is
    # needed, not a formality
    d = 3
    t = np.arange((1 << 26) - 3000, 1 << 26, dtype=np.int64)
    q, r = split(t, d)
    assert np.any(q != t // d)
