"""The mixed dtypes' Cholesky pivots: the FP64 square root and reciprocal of
an FP32 value, rounded to FP32, equal the correctly rounded FP32 square root
and reciprocal (double rounding is innocuous for sqrt and division when the
wider format has at least 2p + 2 significand bits: 53 >= 2 * 24 + 2;
S. A. Figueroa, 1995).  The GPU kernels rely on this to take the FP32
operations; numpy's float32 sqrt and divide are IEEE round-to-nearest."""
import numpy as np


def _samples(count, seed):
    rng = np.random.default_rng(seed)
    # every binade of positive normal floats, uniform significands
    bits = rng.integers(0x00800000, 0x7F800000, size=count, dtype=np.int64).astype(np.uint32)
    x = bits.view(np.float32)
    edge = np.array([1.0, 2.0, 4.0, 0.5, 3.0, np.finfo(np.float32).max,
                     np.finfo(np.float32).tiny, np.float32(1.0) + np.finfo(np.float32).eps,
                     np.float32(2.0) - np.finfo(np.float32).eps], dtype=np.float32)
    # subnormals too
    sub = (rng.integers(1, 0x00800000, size=count // 16, dtype=np.int64).astype(np.uint32)
           .view(np.float32))
    return np.concatenate([x, edge, sub])


def test_sqrt_via_fp64_equals_fp32_sqrt():
    x = _samples(2_000_000, 11)
    via64 = np.sqrt(x.astype(np.float64)).astype(np.float32)
    direct = np.sqrt(x)
    assert np.array_equal(via64.view(np.uint32), direct.view(np.uint32))


def test_reciprocal_via_fp64_equals_fp32_division():
    x = _samples(2_000_000, 12)
    with np.errstate(over="ignore"):
        x = x[np.isfinite(np.float32(1.0) / x)]  # 1/x overflows for the smallest subnormals
        via64 = (1.0 / x.astype(np.float64)).astype(np.float32)
        direct = np.float32(1.0) / x
    assert np.array_equal(via64.view(np.uint32), direct.view(np.uint32))


def test_a_too_narrow_format_is_not_innocuous():
    """Control: rounding the square root to 12 significand bits and then to
    11 (an intermediate narrower than 2 * 11 + 2) does differ from rounding
    to 11 bits once, so the equalities above are a property of the widths,
    not of the test."""
    rng = np.random.default_rng(13)
    x = rng.uniform(1.0, 4.0, 200_000)

    def round_bits(v, p):
        m, e = np.frexp(v)
        return np.ldexp(np.round(m * 2.0 ** p) / 2.0 ** p, e)
    direct = round_bits(np.sqrt(x), 11)
    twice = round_bits(round_bits(np.sqrt(x), 12), 11)
    assert not np.array_equal(direct, twice)
