"""The double-float arithmetic of the Gram-Schmidt (gs_arith = 1), restated in
NumPy float32 and checked against a long-double reference: the error-free
transformations it is built from (Knuth's two-sum, the FMA two-product) are
exact, and a dot product accumulated the kernel's way (k_mdot_df: per
component pair a running (s, c) sum, renormalised after every step, hi*hi
exact, the cross terms in FP32, lo*lo dropped) stays within a small multiple
of 2^-47 of the sum of |terms|, far below FP32 and close to FP64.  This pins
the arithmetic's design; the kernels themselves are checked against the
oracle on the GPU."""
import numpy as np

F = np.float32
LD = np.longdouble


def fma(a, b, c):
    """fused multiply-add of float32 values: the product of two floats is exact
    in float64, so this rounds a*b + c once in float64 and once more to float32
    (a double rounding that can differ from a single one by an ulp, far below
    the bounds checked here)"""
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = F(a + b)
    bv = F(s - a)
    av = F(s - bv)
    return s, F(F(a - av) + F(b - bv))


def two_prod(a, b):
    p = F(a * b)
    return p, fma(a, b, -p)


def renorm(s, t):
    h = F(s + t)
    return h, F(t - F(h - s))


def df_acc(acc, xh, xl, yh, yl):
    """acc += x * y, x = xh + xl, y = yh + yl (one component of k_mdot_df)"""
    p, e = two_prod(xh, yh)
    e = fma(xh, yl, e)
    e = fma(xl, yh, e)
    s, t = two_sum(acc[0], p)
    return renorm(s, F(t + F(acc[1] + e)))


def split(x):
    h = F(x)
    return h, F(np.float64(x) - np.float64(h))


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a, b = F(rng.standard_normal() * 10.0 ** rng.integers(-8, 8)), F(rng.standard_normal())
        s, e = two_sum(a, b)
        assert LD(s) + LD(e) == LD(a) + LD(b)
        p, e = two_prod(a, b)
        assert LD(p) + LD(e) == LD(a) * LD(b)


def test_split_keeps_about_48_bits():
    rng = np.random.default_rng(4)
    x = rng.standard_normal(1000)
    for v in x:
        h, l = split(v)
        assert abs((np.float64(h) + np.float64(l)) - v) <= 2.0 ** -47 * abs(v)


def test_double_float_dot_is_close_to_fp64():
    rng = np.random.default_rng(5)
    n = 3000
    v = rng.standard_normal(n)
    w = rng.standard_normal(n) * 1e-3
    acc = (F(0), F(0))
    for a, b in zip(v, w):
        ah, al = split(a)
        bh, bl = split(b)
        acc = df_acc(acc, ah, al, bh, bl)
    got = LD(acc[0]) + LD(acc[1])
    exact = sum(LD(a) * LD(b) for a, b in zip(v, w))
    scale = sum(abs(LD(a) * LD(b)) for a, b in zip(v, w))
    err = abs(got - exact) / scale
    assert err <= 8 * 2.0 ** -47, float(err)
    # and far below a plain FP32 accumulation of the same terms
    plain = F(0)
    for a, b in zip(v, w):
        plain = fma(F(a), F(b), plain)
    assert abs(LD(plain) - exact) / scale > 100 * err
