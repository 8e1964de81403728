"""The test-side TF32 rounding used to pin the TF32 form (host only)."""
import numpy as np

from numerics import round_tf32


def test_round_tf32_ties_go_to_even_and_specials_pass():
    x = np.array([1.0, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -10 + 2.0 ** -12,
                  -2.5, np.inf, -0.0], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -9, 1.0 + 2.0 ** -10, -2.5, np.inf, -0.0], dtype=np.float32)
    assert np.array_equal(round_tf32(x), want)
    assert np.isnan(round_tf32(np.array([np.nan], dtype=np.float32)))[0]


def test_round_tf32_is_within_half_an_ulp_of_ten_bits():
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 100
    r = round_tf32(x)
    assert np.all((r.view(np.uint32) & 0x1FFF) == 0)            # 13 low mantissa bits cleared
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -11)      # half a unit of the 10-bit mantissa
