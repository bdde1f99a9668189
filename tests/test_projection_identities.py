"""The exact identities the render kernels' projection relies on (Sec. 3.1),
checked on the host over every float32 exponent and the special values.

The kernels compute s = (c / w * 0.5 + 0.5) * size with each step rounded in
float32, but write the two middle steps as one fused multiply-add, and take
the culling tests as integer compares of bit patterns:

- fma(ndc, 0.5, 0.5) equals RN(RN(ndc * 0.5) + 0.5);
- w lies in (0, inf) exactly when bits(w) - 1 < 0x7F7FFFFF (unsigned);
- for s != -0, 0 <= s < size exactly when bits(s) < bits(size), and the
  kernels' s is never -0.

numpy float32 arithmetic rounds every operation to nearest-even, keeps
denormals and never fuses.  The fused result is emulated in float64: ndc *
0.5 + 0.5 is exact there when |ndc| >= 2^-27, and otherwise both the float64
sum and the exact one lie within 2^-28 of 0.5, so both round to 0.5 in
float32.
"""
import numpy as np

F32, U32 = np.float32, np.uint32
SPECIAL = np.array([0.0, -0.0, 1e-45, -1e-45, 1.1754942e-38, 1.17549435e-38, -1.17549435e-38, 3.4028235e38,
                    -3.4028235e38, np.inf, -np.inf, np.nan, 0.5, -0.5, 1.0, -1.0, 2.0, -2.0, 0.99999994, -0.99999994,
                    1.0000001, -1.0000001, 2.0 ** -126, 2.0 ** -125, -(2.0 ** -125), 2.0 ** -27, -(2.0 ** -27),
                    2.0 ** -28, 3.0, -3.0], dtype=F32)


def float32_sample(count: int, seed: int) -> np.ndarray:
    """Random bit patterns (every exponent, both signs, NaNs included),
    values spread over [-4, 4], and the special values."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 1 << 32, size=count, dtype=np.uint64).astype(U32).view(F32)
    near = rng.uniform(-4.0, 4.0, size=count).astype(F32)
    return np.concatenate([bits, near, SPECIAL])


def fused_half(ndc: np.ndarray) -> np.ndarray:
    return (ndc.astype(np.float64) * 0.5 + 0.5).astype(F32)


def two_roundings(ndc: np.ndarray) -> np.ndarray:
    return (ndc * F32(0.5)) + F32(0.5)


def same_bits(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (a.view(U32) == b.view(U32)) | (np.isnan(a) & np.isnan(b))


def test_fused_half_equals_two_roundings():
    with np.errstate(all="ignore"):
        ndc = float32_sample(2_000_000, 1)
        assert same_bits(fused_half(ndc), two_roundings(ndc)).all()
        # every float32 in [-2^-24, 2^-24] near the underflow edge, by bit pattern
        tiny = np.arange(0, 1 << 20, dtype=U32).view(F32)
        for t in (tiny, -tiny):
            assert same_bits(fused_half(t), two_roundings(t)).all()


def test_integer_depth_test_equals_float_test():
    with np.errstate(all="ignore"):
        w = float32_sample(2_000_000, 2)
        float_test = (w > F32(0.0)) & (w < F32(np.inf))
        int_test = (w.view(U32) - U32(1)) < U32(0x7F7FFFFF)
        assert np.array_equal(float_test, int_test)
        # the boundaries by bit pattern: +0, the smallest denormal, FLT_MAX, +inf, -0
        edge = np.array([0, 1, 0x7F7FFFFF, 0x7F800000, 0x80000000, 0x7FC00000, 0xFFFFFFFF], dtype=U32)
        assert ((edge - U32(1)) < U32(0x7F7FFFFF)).tolist() == [False, True, True, False, False, False, False]


def test_integer_viewport_test_equals_float_test():
    with np.errstate(all="ignore"):
        s = float32_sample(500_000, 3)
        s = s[s.view(U32) != U32(0x80000000)]  # -0 is excluded (next test)
        for size in (1, 2, 3, 7, 31, 640, 1080, 1920, 4096, 16383, 16384):
            fs = F32(size)
            float_test = (s >= F32(0.0)) & (s < fs)
            int_test = s.view(U32) < fs.view(U32)
            assert np.array_equal(float_test, int_test), size
            grid = np.linspace(-1.0, size + 1.0, 20_001).astype(F32)
            grid = grid[grid.view(U32) != U32(0x80000000)]
            assert np.array_equal((grid >= F32(0.0)) & (grid < fs), grid.view(U32) < fs.view(U32)), size


def test_screen_coordinate_is_never_negative_zero():
    """t = fma(ndc, 0.5, 0.5) is +0 or at least 2^-25 in magnitude, so
    t * size (size >= 1) cannot round to -0."""
    with np.errstate(all="ignore"):
        ndc = float32_sample(2_000_000, 4)
        # the values of ndc just below -1, where t is a tiny negative number
        below = (np.arange(1, 1 << 16, dtype=U32) + F32(-1.0).view(U32)).view(F32)
        ndc = np.concatenate([ndc, below])
        t = fused_half(ndc)
        finite_t = t[np.isfinite(t)]
        assert not (finite_t.view(U32) == U32(0x80000000)).any()
        nonzero = finite_t[finite_t != 0]
        assert np.abs(nonzero).min() >= F32(2.0 ** -25)
        for size in (1, 1920, 16384):
            s = t * F32(size)
            assert not (s.view(U32) == U32(0x80000000)).any(), size
