"""The BF16 storage rounding used as reference by the parity tests (CPU only): one rounding from
FP64 to the nearest value with 8 significant bits, ties to even, checked against a brute-force
search over the BF16 grid and against the double-rounding counterexample (FP64 -> FP32 -> BF16)."""
import numpy as np

from helpers import round_bf16


def _bf16_grid_neighbours(x):
    """The two BF16 values around x > 0 (normal range) and whether the lower one has an even
    significand: enumerate the 2^7 significands of x's binade and its successor."""
    e = int(np.floor(np.log2(x)))
    cand = [(1.0 + k / 128.0) * 2.0**e for k in range(128)] + [2.0 ** (e + 1)]
    lo = max(c for c in cand if c <= x)
    hi = min(c for c in cand if c >= x)
    return lo, hi, e


def test_round_bf16_matches_brute_force():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(0.5, 4.0, 3000), 10.0 ** rng.uniform(-30, 30, 3000)])
    got = round_bf16(xs)
    for x, g in zip(xs, got):
        lo, hi, e = _bf16_grid_neighbours(x)
        if lo == hi:
            assert g == x
            continue
        if x - lo < hi - x:
            expect = lo
        elif hi - x < x - lo:
            expect = hi
        else:  # tie: the neighbour whose last significand bit is zero
            k_lo = round((lo / 2.0**e - 1.0) * 128.0)
            expect = lo if k_lo % 2 == 0 else hi
        assert g == expect, (x, g, expect)
    np.testing.assert_array_equal(round_bf16(-xs), -got)


def test_single_rounding_not_double_rounding():
    # 1 + 3 2^-8 - 2^-40 lies below the midpoint of 1 + 2^-7 and 1 + 2^-6: nearest is 1 + 2^-7.
    # Through FP32 it first becomes the midpoint itself, which then rounds to the even 1 + 2^-6.
    x = 1.0 + 3.0 * 2.0**-8 - 2.0**-40
    assert round_bf16(x) == 1.0 + 2.0**-7
    via_f32 = np.float32(x)
    assert float(via_f32) == 1.0 + 3.0 * 2.0**-8
    assert round_bf16(np.float64(via_f32)) == 1.0 + 2.0**-6
    # exact ties go to the even significand
    assert round_bf16(1.0 + 2.0**-8) == 1.0
    assert round_bf16(1.0 + 3.0 * 2.0**-8) == 1.0 + 2.0**-6
    assert round_bf16(0.0) == 0.0
