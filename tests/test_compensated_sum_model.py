"""Host model of the compensated FP32 combination that the library uses for
all-float combinations of the split dtypes (tucker_f64.cu,
lincomb1_f32_kernel): out = sum_k c_k x_k with FP32 inputs and a float
output, each c_k split as chi + clo, each product formed as chi x = p + e
(e exact, as the FMA gives it), the sum kept as a (hi, lo) pair updated by
Knuth's two-sum.  numpy float32 operations round like the GPU's FP32 adds and
multiplies, and the exact product of two floats fits a double, which gives
the FMA's exact error term.

Pinned: the compensated result equals the FP64 evaluation rounded to float
except for results within a hair of a rounding boundary, and it is far more
accurate than plain FP32 accumulation on cancelling sums."""
import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def compensated(cs, xs):
    hi = np.zeros_like(xs[0], dtype=f32)
    lo = np.zeros_like(xs[0], dtype=f32)
    for c, x in zip(cs, xs):
        ch = f32(c)
        cl = f32(c - float(ch))
        p = f32(ch * x)
        e_exact = (ch.astype(np.float64) * x.astype(np.float64) - p.astype(np.float64)).astype(f32)  # fmaf(ch, x, -p)
        e = f32(e_exact + f32(cl * x))
        s, t = two_sum(hi, p)
        hi = s
        lo = f32(lo + f32(t + e))
    return f32(hi + lo)


def test_compensated_sum_matches_fp64_rounded_to_float():
    rng = np.random.default_rng(11)
    for trial in range(20):
        m = int(rng.integers(1, 13))
        xs = [rng.standard_normal(20000).astype(f32) * f32(10.0 ** rng.uniform(-3, 3)) for _ in range(m)]
        cs = list(rng.standard_normal(m) * 10.0 ** rng.uniform(-4, 1, m))
        exact = sum(c * x.astype(np.float64) for c, x in zip(cs, xs))
        ref = exact.astype(f32)
        got = compensated(cs, xs)
        diff_ulp = np.abs(got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
        # at most one float ulp apart, and only where the exact sum lies
        # within 2^-40 (relative) of a rounding boundary
        assert diff_ulp.max() <= 1
        off = np.nonzero(diff_ulp)[0]
        if off.size:
            a = exact[off]
            mid = (got[off].astype(np.float64) + ref[off].astype(np.float64)) / 2
            assert np.all(np.abs(a - mid) <= 2.0 ** -40 * np.abs(a))


def test_compensated_sum_survives_cancellation_where_fp32_does_not():
    rng = np.random.default_rng(12)
    x = rng.standard_normal(10000).astype(f32)
    y = (x * f32(1.0 + 2.0 ** -20)).astype(f32)
    cs, xs = [1.0 / 3.0, -1.0 / 3.0, 1e-7], [y, x, x]   # (1/3 is not a float: the products round)
    exact = sum(c * v.astype(np.float64) for c, v in zip(cs, xs))
    plain = f32(f32(f32(cs[0]) * y) + f32(f32(cs[1]) * x) + f32(f32(cs[2]) * x))
    comp = compensated(cs, xs)
    err_c = np.abs(comp - exact).max() / np.abs(exact).max()
    err_p = np.abs(plain.astype(np.float64) - exact).max() / np.abs(exact).max()
    assert err_c <= 2.0 ** -23
    assert err_p > 4 * err_c
