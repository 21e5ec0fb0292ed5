"""The operand splits of the split-precision dtypes, modelled on the host:
x = hi + lo + r with hi = round(x) and lo = round(x - hi) in the narrow format
(bf16: 8 significant bits, round to nearest even; tf32: 11 significant bits,
round to nearest, ties away from zero), x - hi exact in FP32.  With p the
format's significant bits, |x - hi| <= 2^-p |x|, and since x - hi lies below
2^(e - p) for x in [2^e, 2^(e+1)) unless it equals that power of two (then
lo is exact), rounding it costs at most 2^(-2p-1) |x|:
    BF16X3 |r| <= 2^-17 |x|,  TF32X3 |r| <= 2^-23 |x|,  TF32 (hi only) 2^-11 |x|,
each attained to within a factor of two.  The tolerances of the split dtypes
start from these figures."""
import numpy as np
import pytest


def bf16_rn(x):
    """float32 -> nearest bf16 (ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def tf32_rna(x):
    """float32 -> nearest tf32 (10 stored mantissa bits, ties away), as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x1000) >> 13) << 13
    return r.astype(np.uint32).view(np.float32)


def split(x, rnd):
    hi = rnd(x)
    d = (x - hi).astype(np.float32)  # exact: x and hi share the leading bits
    lo = rnd(d)
    return hi, lo


def _inputs(seed, count=200000):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(count) * np.exp2(rng.integers(-60, 60, count))
    return x.astype(np.float32)


def test_rounding_helpers_match_known_values():
    one = np.float32(1.0)
    # 1 + 2^-8 is the midpoint between bf16 1 and 1 + 2^-7: even -> 1
    assert bf16_rn(np.float32(1 + 2.0 ** -8)) == one
    assert bf16_rn(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)
    # tf32: 1 + 2^-11 is the midpoint of 1 and 1 + 2^-10: away -> 1 + 2^-10
    assert tf32_rna(np.float32(1 + 2.0 ** -11)) == np.float32(1 + 2.0 ** -10)
    assert tf32_rna(np.float32(-(1 + 2.0 ** -11))) == np.float32(-(1 + 2.0 ** -10))
    for v in (0.0, 1.0, -2.5, 3.0 * 2.0 ** -40):
        assert bf16_rn(np.float32(v)) == np.float32(v)
        assert tf32_rna(np.float32(v)) == np.float32(v)


@pytest.mark.parametrize("name,rnd,bits", [("bf16", bf16_rn, 8), ("tf32", tf32_rna, 11)])
def test_split_residuals_meet_their_bounds(name, rnd, bits):
    x = _inputs(bits)
    hi, lo = split(x, rnd)
    xd = x.astype(np.float64)
    # the narrow values really are narrow: no bits below the format's precision
    for v in (hi, lo):
        m, _ = np.frexp(v.astype(np.float64))
        assert np.all(m * 2.0 ** bits == np.round(m * 2.0 ** bits))
    # x - hi is exact in FP32
    assert np.all((xd - hi.astype(np.float64)) == (x - hi).astype(np.float64))
    r1 = np.abs(xd - hi) / np.abs(xd)
    r2 = np.abs(xd - hi.astype(np.float64) - lo.astype(np.float64)) / np.abs(xd)
    u = 2.0 ** -bits
    assert r1.max() <= u and r1.max() > u / 2
    assert r2.max() <= u * u / 2 and r2.max() > u * u / 4
