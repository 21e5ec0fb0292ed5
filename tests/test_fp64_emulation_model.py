"""The arithmetic of the FP64-emulated mu-mode products (PHIKS_FP64_EMU),
modelled on the host with exact integers.

The scheme is Ozaki-style splitting (Ozaki, Ogita, Oishi and Rump, 2012) with
balanced base-256 digits: each fibre x of the tensor (the n values contracted
together) and each row l of the matrix is written as x_j = Q_j 2^k with
|Q_j| < 2^55 (k from the largest element; smaller elements rounded to the
nearest integer Q_j) and Q_j = sum_s c_s 2^(8 (6 - s)), seven digits with
c_1..c_6 in [-128, 127] and |c_0| <= 128.  The dot product keeps the 28 digit
products with s + t <= 6: G_k = sum_j sum_{s+t=k} b_s c_t, accumulated in FP32
on the tensor cores, then T = sum_k 2^(8 (6 - k)) G_k, S = floor(T / 2^8) and
the result RN(S) 2^(k_x + k_l + 56).

These tests pin the two facts the GPU path relies on, independently of its
kernels: every G_k is an integer below 2^24 for n <= 128 (so FP32 sums it
exactly in any order), and the error per dot product is at most
    (n (1 + 6.03) 2^-54 + 2^-52) max|x| max|l| + 2^-53 |result|
(input rounding 2^-54 per term, the dropped products s + t >= 7 at most
6.03 2^-54 per term, the floor 2^-52, the final rounding).
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

DIGITS = 7


def fixed_point(x):
    """Q_j and k with x_j = Q_j 2^k up to rounding, |Q_j| < 2^55."""
    m = max(abs(v) for v in x)
    if m == 0:
        return [0] * len(x), 0
    k = math.frexp(m)[1] - 55  # m in [2^(k + 54), 2^(k + 55))
    scale = Fraction(2) ** k
    return [round(Fraction(v) / scale) for v in x], k


def balanced_digits(Q):
    """c_0 (most significant) .. c_6 with Q = sum_s c_s 256^(6 - s)."""
    low = []
    for _ in range(DIGITS - 1):
        r = (Q + 128) % 256 - 128
        low.append(r)
        Q = (Q - r) // 256
    return [Q] + low[::-1]


def slice_sums(cx, cl):
    """G_k = sum_j sum_{s+t=k} b_s c_t for k = 0..6 (exact integers)."""
    G = [0] * DIGITS
    for c, b in zip(cx, cl):
        for s in range(DIGITS):
            for t in range(DIGITS - s):
                G[s + t] += b[s] * c[t]
    return G


def emulated_dot(x, l):
    Qx, kx = fixed_point(x)
    Ql, kl = fixed_point(l)
    G = slice_sums([balanced_digits(q) for q in Qx], [balanced_digits(q) for q in Ql])
    T = sum(g << (8 * (DIGITS - 1 - k)) for k, g in enumerate(G))
    S = T >> 8  # floor
    return math.ldexp(float(S), kx + kl + 56), G


def bound(x, l, result):
    n = len(x)
    M = max(abs(v) for v in x) * max(abs(v) for v in l)
    return (n * 7.03 * 2.0 ** -54 + 2.0 ** -52) * M + 2.0 ** -53 * abs(result)


def exact_dot(x, l):
    return sum(Fraction(a) * Fraction(b) for a, b in zip(x, l))


def test_digits_reconstruct_and_stay_balanced():
    rng = random.Random(3)
    for _ in range(2000):
        Q = rng.randrange(-(2 ** 55) + 1, 2 ** 55)
        c = balanced_digits(Q)
        assert sum(v * 256 ** (DIGITS - 1 - s) for s, v in enumerate(c)) == Q
        assert abs(c[0]) <= 128
        assert all(-128 <= v <= 127 for v in c[1:])
    for Q in (2 ** 55 - 1, -(2 ** 55) + 1, 0, 128, -128, 127 * 2 ** 40):
        c = balanced_digits(Q)
        assert abs(c[0]) <= 128 and sum(v * 256 ** (DIGITS - 1 - s) for s, v in enumerate(c)) == Q


def test_fixed_point_rounding_is_half_a_unit():
    rng = np.random.default_rng(4)
    x = list(rng.standard_normal(64) * np.exp2(rng.integers(-70, 3, 64)))
    Q, k = fixed_point(x)
    m = max(abs(v) for v in x)
    assert max(abs(q) for q in Q) < 2 ** 55
    for v, q in zip(x, Q):
        assert abs(Fraction(v) - q * Fraction(2) ** k) <= Fraction(2) ** (k - 1)
        assert abs(Fraction(v) - q * Fraction(2) ** k) <= Fraction(m) * Fraction(2) ** -55


@pytest.mark.parametrize("n", [8, 128])
def test_slice_sums_are_exact_in_fp32_at_the_worst_digits(n):
    # every digit at its largest magnitude with equal signs: the largest |G_k|
    worst = [-128] * DIGITS
    G = slice_sums([worst] * n, [worst] * n)
    assert all(abs(g) < 2 ** 24 for g in G)
    assert G[DIGITS - 1] == DIGITS * n * 128 * 128
    # FP32 accumulation in a random order reproduces each G_k exactly
    rng = np.random.default_rng(n)
    for k in range(DIGITS):
        terms = np.full((k + 1) * n, 128.0 * 128.0, dtype=np.float32)
        terms[rng.random(terms.size) < 0.5] *= -1
        exact = int(terms.astype(np.int64).sum())
        acc = np.float32(0)
        for v in terms[rng.permutation(terms.size)]:
            acc = np.float32(acc + v)
        assert int(acc) == exact


def test_longest_exact_contraction_covers_the_supported_n():
    # (k + 1) n 2^14 < 2^24 for k = 6 needs n <= 146; the kernels accept n <= 128
    assert max(n for n in range(1, 400) if DIGITS * n * 2 ** 14 < 2 ** 24) == 146


@pytest.mark.parametrize("n,seed", [(8, 1), (64, 2), (128, 3)])
def test_error_bound_on_random_fibres(n, seed):
    rng = np.random.default_rng(seed)
    for trial in range(20):
        if trial % 2:
            x = rng.standard_normal(n)
            l = rng.standard_normal(n)
        else:  # wide dynamic range, including elements far below the largest
            x = rng.standard_normal(n) * np.exp2(rng.integers(-80, 4, n))
            l = rng.standard_normal(n) * np.exp2(rng.integers(-30, 4, n))
        x, l = [float(v) for v in x], [float(v) for v in l]
        got, G = emulated_dot(x, l)
        assert all(abs(g) < 2 ** 24 for g in G)
        err = abs(Fraction(got) - exact_dot(x, l))
        assert err <= Fraction(bound(x, l, got))


def _from_digits(c, shift):
    return math.ldexp(float(sum(v * 256 ** (DIGITS - 1 - s) for s, v in enumerate(c))), shift)


def test_error_bound_on_adversarial_digits():
    # digits near +-128 everywhere make the dropped products s + t >= 7 as
    # large as they can be; the bound must still hold
    n = 128
    x = [_from_digits([96] + [127 if (j + s) % 2 else -128 for s in range(1, DIGITS)], -48)
         for j in range(n)]
    l = [_from_digits([96] + [127 if s % 2 else -128 for s in range(1, DIGITS)], -48)] * n
    got, _ = emulated_dot(x, l)
    assert abs(Fraction(got) - exact_dot(x, l)) <= Fraction(bound(x, l, got))
    # equal signs in every low digit: the dropped products add up, past
    # n 2^-53 max|x| max|l|, so the truncation term of the bound is needed
    x = [_from_digits([96] + [-128] * (DIGITS - 1), -48)] * n
    got, _ = emulated_dot(x, x)
    err = abs(Fraction(got) - exact_dot(x, x))
    M = Fraction(max(abs(v) for v in x)) ** 2
    assert err <= Fraction(bound(x, x, got))
    assert err > n * Fraction(2) ** -53 * M


def test_a_dropped_term_breaks_the_bound():
    # the bound is tight enough to catch a slip: losing one slice sum (G_5,
    # weight 2^8 in T) exceeds it on ordinary inputs
    rng = np.random.default_rng(9)
    x = [float(v) for v in rng.standard_normal(64)]
    l = [float(v) for v in rng.standard_normal(64)]
    Qx, kx = fixed_point(x)
    Ql, kl = fixed_point(l)
    G = slice_sums([balanced_digits(q) for q in Qx], [balanced_digits(q) for q in Ql])
    G[DIGITS - 2] = 0
    T = sum(g << (8 * (DIGITS - 1 - k)) for k, g in enumerate(G))
    wrong = math.ldexp(float(T >> 8), kx + kl + 56)
    assert abs(Fraction(wrong) - exact_dot(x, l)) > Fraction(bound(x, l, wrong))


def _as_f32_bits(v):
    return int(np.array([v], dtype=np.float32).view(np.int32)[0])


@pytest.mark.parametrize("n", [8, 36, 64, 128])
def test_fp32_add_conversion_is_exact_where_the_epilogue_uses_it(n):
    """G_k + 1.5 2^23 in FP32, minus the bit pattern of 1.5 2^23, is G_k for
    |G_k| <= 2^22: the epilogue uses it for the accumulators k with
    (k + 1) n <= 256 (all seven for n <= 36, four for n <= 64, two for n <= 128)."""
    nm = {8: 7, 36: 7, 64: 4, 128: 2}[n]
    magic = _as_f32_bits(12582912.0)
    assert magic == 0x4B400000
    for k in range(nm):
        bound = (k + 1) * n * 2 ** 14
        assert bound <= 2 ** 22
        for g in (-bound, -bound + 1, -1, 0, 1, bound - 1, bound, 12345, -777777):
            if abs(g) > bound:
                continue
            s = np.float32(g) + np.float32(12582912.0)
            assert _as_f32_bits(s) - magic == g, (k, g)
    # one past the bound would not be exact: 2^22 + 1 lands above 2^24
    s = np.float32(2 ** 22 + 1) + np.float32(12582912.0)
    assert _as_f32_bits(s) - magic != 2 ** 22 + 1


def _i32(v):
    assert -2 ** 31 <= v < 2 ** 31, v   # the kernel's 32-bit partial sums must not wrap
    return v


@pytest.mark.parametrize("seed", range(4))
def test_partial_sum_assembly_matches_the_64_bit_one(seed):
    """For n <= 64 the epilogue forms S = floor(T / 2^8) from 32-bit partial
    sums A = 2^8 G_0 + G_1, B = 2^8 G_2 + G_3, C = 2^8 G_4 + G_5 + floor(G_6 / 2^8)
    as S = A 2^32 + B 2^16 + C; this is the sum T = sum_k 2^(8 (6 - k)) G_k
    floored, and no partial sum leaves 32 bits at the largest |G_k|."""
    rng = random.Random(seed)
    n = 64
    bounds = [(k + 1) * n * 2 ** 14 for k in range(DIGITS)]
    cases = [[b for b in bounds], [-b for b in bounds], [0] * DIGITS]
    cases += [[rng.randint(-b, b) for b in bounds] for _ in range(2000)]
    for g in cases:
        A = _i32(g[0] * 256 + g[1])
        B = _i32(g[2] * 256 + g[3])
        C = _i32(g[4] * 256 + g[5] + (g[6] >> 8))
        S = A * 2 ** 32 + B * 2 ** 16 + C
        T = sum(gk * 2 ** (8 * (6 - k)) for k, gk in enumerate(g))
        assert S == T // 256


def _fixed_from_sum(S, e, E):
    """The split of exact sums: Q = S 2^(e - (E - 1077)) rounded half away
    from zero, by the shifts the kernel uses (arbitrary-precision integers)."""
    if S == 0:
        return 0
    u = abs(S)
    sh = E - 1077 - e
    if sh <= 0:
        q = u << (-sh)
    elif sh < 64:
        q = (u >> sh) + ((u >> (sh - 1)) & 1)
    else:
        q = 0
    return -q if S < 0 else q


@pytest.mark.parametrize("seed", range(3))
def test_fixed_point_of_exact_sums(seed):
    """The pass after a resident GEMM pass takes the exact sums S with value
    S 2^e (e = fibre exponent + row exponent - 40) instead of rounded
    doubles: the fibre exponent is the largest value's biased exponent as a
    double, E = max(bitlength(S) + e + 1022), and every Q is the value in
    units of 2^(E - 1077), rounded half away from zero, with |Q| <= 2^55: the
    same fixed point the double path reaches (one rounding less)."""
    rng = random.Random(seed)
    for _ in range(300):
        fib = []
        for _ in range(8):
            L = rng.randint(0, 62)
            S = 0 if L == 0 else rng.choice((-1, 1)) * rng.randint(2 ** (L - 1), 2 ** L - 1)
            fib.append((S, rng.randint(-80, 40)))
        nz = [(S, e) for S, e in fib if S]
        if not nz:
            continue
        E = max(abs(S).bit_length() + e + 1022 for S, e in nz)
        for S, e in fib:
            q = _fixed_from_sum(S, e, E)
            assert abs(q) <= 2 ** 55
            exact = Fraction(S) * Fraction(2) ** (e + 1077 - E)
            want = math.floor(abs(exact) + Fraction(1, 2)) * (1 if exact >= 0 else -1)
            assert q == want, (S, e, E)
        # the largest value uses the top of the range: 2^54 <= |Q| <= 2^55
        assert max(abs(_fixed_from_sum(S, e, E)) for S, e in nz) >= 2 ** 54
        # as a double the same value gives the same Q once it is exactly representable
        for S, e in nz:
            if abs(S) < 2 ** 53 and -1000 < abs(S).bit_length() + e + 1022 < 2000:
                x = math.ldexp(float(S), e)
                if x != 0.0 and math.isfinite(x):
                    m, ex = math.frexp(abs(x))                     # |x| = m 2^ex, m in [1/2, 1)
                    bexp = ex + 1022                               # biased exponent of x
                    assert bexp == abs(S).bit_length() + e + 1022
