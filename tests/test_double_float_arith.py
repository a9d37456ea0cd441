"""Precision of the double-float arithmetic the double-float walk (sg_opts.precision = 48) is
built on, checked on the CPU: each value an unevaluated sum hi + lo of two float32 numbers,
Knuth's two-sum, Dekker's fast two-sum and the exact product (an FMA on the GPU; here the
float64 product of two float32 numbers, which is exact), and from them the sum, the sum of two
terms of one sign, the two-term dot product, product, quotient and reciprocal square root in the
forms the walks use.  Each function here restates, operation for operation, the device function
of the same name in paper_2603_15780_gb300/csrc/walk.cuh (its FMA as a float64 multiply-add
rounded once to float32).  Their results are compared with
float64 references (whose own error, about 1e-16, is far below the bounds) over random operands
spanning the magnitudes a walk meets."""
import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def two_prod(a, b):
    p = f32(a * b)
    return p, f32(np.float64(a) * np.float64(b) - np.float64(p))


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def df_add(a, b):
    s, e = two_sum(a[0], b[0])
    t, f = two_sum(a[1], b[1])
    e = f32(e + t)
    s, e = fast_two_sum(s, e)
    e = f32(e + f)
    return fast_two_sum(s, e)


def df_add_same_sign(a, b):
    s, e = two_sum(a[0], b[0])
    e = f32(e + f32(a[1] + b[1]))
    return fast_two_sum(s, e)


def df_dot2(a, b, c, d):
    p, pe = two_prod(a[0], b[0])
    q, qe = two_prod(c[0], d[0])
    s, e = two_sum(p, q)
    lo = f32(e + f32(pe + qe))
    lo = fma(a[0], b[1], lo)
    lo = fma(a[1], b[0], lo)
    lo = fma(c[0], d[1], lo)
    lo = fma(c[1], d[0], lo)
    return fast_two_sum(s, lo)


def df_mul(a, b):
    p, e = two_prod(a[0], b[0])
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    return fast_two_sum(p, e)


def df_mul_f(a, b):
    p, e = two_prod(a[0], b)
    e = fma(a[1], b, e)
    return fast_two_sum(p, e)


def df_div(a, b):
    rb = f32(1.0 / np.float64(b[0]))           # the correctly rounded reciprocal
    q1 = f32(a[0] * rb)
    r = df_add(a, tuple(-x for x in df_mul_f(b, q1)))
    return fast_two_sum(q1, f32(r[0] * rb))


def df_rsqrt(n):
    r = f32(1.0 / np.sqrt(np.float64(n[0])))   # an FP32 estimate (the GPU's rsqrtf is within 2 ulp)
    r = f32(r * f32(1 + 2.0 ** -22))           # perturb it by that much: the Newton step must absorb it
    e = df_add((f32(1), f32(0)), tuple(-x for x in df_mul(n, two_prod(r, r))))
    return fast_two_sum(r, f32(f32(0.5) * r * e[0]))


def split(x):
    hi = f32(x)
    return hi, f32(x - np.float64(hi))


def val(a):
    return np.float64(a[0]) + np.float64(a[1])


def operands(rng, n):
    mag = 10.0 ** rng.uniform(-4, 1, n)
    return rng.choice([-1.0, 1.0], n) * mag * rng.uniform(0.5, 1.0, n)


def rel(x, ref):
    return abs(x - ref) / abs(ref)


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(3)
    a, b = (operands(rng, 2000).astype(np.float32) for _ in range(2))
    for x, y in zip(a, b):
        s, e = two_sum(x, y)
        assert np.float64(s) + np.float64(e) == np.float64(x) + np.float64(y)
        p, e = two_prod(x, y)
        assert np.float64(p) + np.float64(e) == np.float64(x) * np.float64(y)
        if abs(x) >= abs(y):
            s, e = fast_two_sum(x, y)
            assert np.float64(s) + np.float64(e) == np.float64(x) + np.float64(y)


def test_double_float_operations_keep_about_46_bits():
    """Sum, product and quotient within 2^-44 (measured about 2^-46); the reciprocal square root,
    one Newton step from an estimate 2^-22 off, within 2^-41 (the step squares the estimate's
    error: about 1.5 (2^-22)^2; measured 2^-42)."""
    rng = np.random.default_rng(4)
    xs, ys = operands(rng, 3000), operands(rng, 3000)
    bound = {"add": 2.0 ** -44, "mul": 2.0 ** -44, "div": 2.0 ** -44, "rsqrt": 2.0 ** -41}
    worst = {"add": 0.0, "mul": 0.0, "div": 0.0, "rsqrt": 0.0}
    for x, y in zip(xs, ys):
        a, b = split(x), split(y)
        A, B = val(a), val(b)
        worst["add"] = max(worst["add"], abs(val(df_add(a, b)) - (A + B)) / (abs(A) + abs(B)))
        worst["mul"] = max(worst["mul"], rel(val(df_mul(a, b)), A * B))
        worst["div"] = max(worst["div"], rel(val(df_div(a, b)), A / B))
        worst["rsqrt"] = max(worst["rsqrt"], rel(val(df_rsqrt(split(abs(x)))), 1.0 / np.sqrt(abs(A))))
    assert all(worst[k] < bound[k] for k in worst), worst


def test_sum_is_accurate_under_cancellation():
    """The walk subtracts nearly equal coordinates (c - x near a vertex): the double-float sum
    of two close values keeps a small absolute error relative to its operands."""
    rng = np.random.default_rng(5)
    for x in operands(rng, 2000):
        y = -x * (1.0 + rng.uniform(-1e-9, 1e-9))
        a, b = split(x), split(y)
        err = abs(val(df_add(a, b)) - (val(a) + val(b)))
        assert err <= 2.0 ** -46 * abs(x)


def test_same_sign_sum_and_dot_product():
    """The one-two-sum sum of two terms of one sign (norms, path lengths) within 2^-44 of the
    exact sum; the two-term dot product a b + c d (the mixed walk's crossing test) within 2^-44
    of |a b| + |c d| in absolute terms, including operands whose products cancel."""
    rng = np.random.default_rng(6)
    xs, ys = np.abs(operands(rng, 3000)), np.abs(operands(rng, 3000))
    sg = rng.choice([-1.0, 1.0], 3000)
    worst_s = 0.0
    for x, y, g in zip(xs, ys, sg):
        a, b = split(g * x), split(g * y)
        A, B = val(a), val(b)
        worst_s = max(worst_s, rel(val(df_add_same_sign(a, b)), A + B))
    assert worst_s < 2.0 ** -44, worst_s
    worst_d = 0.0
    for k in range(3000):
        a, b, c = (split(t) for t in operands(rng, 3))
        if k % 2:
            # c d close to -a b: the high parts cancel
            d = split(-val(a) * val(b) / val(c) * (1.0 + rng.uniform(-1e-6, 1e-6)))
        else:
            d = split(operands(rng, 1)[0])
        A, B, C, D = val(a), val(b), val(c), val(d)
        err = abs(val(df_dot2(a, b, c, d)) - (A * B + C * D))
        worst_d = max(worst_d, err / (abs(A * B) + abs(C * D)))
    assert worst_d < 2.0 ** -44, worst_d
