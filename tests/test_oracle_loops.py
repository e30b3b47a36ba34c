"""Pins for the oracle's sequential loops (CPU only).

* The "100 hours" worked example (section Accuracy, second Table 2) with the
  paper's printed results, from ``tests/golden/hundred_hours.txt``.
* The paper's remark after Example 2 that the twofold loops leave the value
  itself as direct summation computes it: value bits of sumtf, sumt (and the
  dot forms) equal those of sum.
* Theorem 2 on two items: sumt of (a, b) is TWO-SUM(a, b).
* Special cases: integer data, where every operation is exact.
* The literal dot loops (the paper's remark that a dot product runs the
  summation loop with the product of the i-th elements as the item): each
  equals its summation loop over the products rounded by numpy's own IEEE
  multiply, bit for bit; Kahan's dot also obeys the compensated-summation
  bound against the exact dot.
* The known error bound of the rigorous (TWO-SUM based) compensated sum,
  |S - (v + e)| <= u|S| + gamma_{n-1}^2 sum|x_i| (Ogita, Rump, Oishi 2005,
  "Accurate sum and dot product", Prop. 4.5 / 5.5), against the exact oracle.
* The magnitude pattern of the paper's accuracy table (first Table 2).
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1401_0248_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hundred_hours.txt")


def golden_rows():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, res, dev, est = line.split()
        rows[name] = (float(res), float(dev), None if est == "-" else float(est))
    return rows


def close6(a, b):
    """equal to the six significant digits the paper prints"""
    if b == 0:
        return a == 0
    return abs(a - b) <= 5e-6 * abs(b) + 1e-12


def test_hundred_hours_matches_paper():
    G = golden_rows()
    x = np.full(3600000, 0.1, dtype=np.float32)
    direct, _ = O.loop("sum", x)
    double, _ = O.loop("sumd", x)
    kahan, _ = O.loop("sumk", x)
    v, e = O.loop("sumtf", x)
    vt, et = O.loop("sumt", x)
    assert (vt, et) == (v, e)      # here |s| >= |y| after the first step: tf == t
    got = {
        "direct": float(direct) / 3600,
        "double": float(double) / 3600,
        "kahan": float(kahan) / 3600,
        "twofold": (float(v) + float(e)) / 3600,   # value + error taken in binary64
    }
    for name, (res, dev, est) in G.items():
        assert close6(got[name], res), (name, got[name], res)
        assert close6(abs(got[name] - 100.0), dev), (name, got[name], dev)
    assert close6(float(e) / 3600, G["twofold"][2])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_twofold_value_is_the_direct_sum(dtype):
    x = I.normal(50001, "f32" if dtype == np.float32 else "f64", seed=7).numpy()
    y = I.uniform(50001, "f32" if dtype == np.float32 else "f64", seed=7, stream=3).numpy()
    s, _ = O.loop("sum", x)
    for m in ("sumtf", "sumt"):
        assert O.loop(m, x)[0] == s
    d, _ = O.loop("dot", x, y)
    for m in ("dottf", "dott", "dottf2", "dott2"):
        assert O.loop(m, x, y)[0] == d


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_sumt_two_items_is_two_sum(dtype):
    a = I.normal(2000, "f32" if dtype == np.float32 else "f64", seed=8).numpy()
    b = (I.normal(2000, "f32" if dtype == np.float32 else "f64", seed=8, stream=5).numpy()
         * dtype(1e-3)).astype(dtype)
    x2, y2 = O.two_sum(a, b)
    for i in range(a.size):
        v, e = O.loop("sumt", np.array([a[i], b[i]], dtype=dtype))
        assert v == x2[i] and e == y2[i]
        if abs(a[i]) >= abs(b[i]):
            v, e = O.loop("sumtf", np.array([a[i], b[i]], dtype=dtype))
            assert Fraction(float(v)) + Fraction(float(e)) == Fraction(float(a[i])) + Fraction(float(b[i]))


def test_integer_data_is_exact():
    rng = np.random.default_rng(3)
    x = rng.integers(-1000, 1000, size=10000).astype(np.float32)    # partial sums < 2^24
    S = float(np.sum(x.astype(np.int64)))
    for m in ("sum", "sumk", "sumtf", "sumt"):
        v, e = O.loop(m, x)
        assert float(v) == S and e == 0
    y = rng.integers(-30, 30, size=10000).astype(np.float32)
    D = float(np.sum(x.astype(np.int64) * y.astype(np.int64)))
    for m in ("dot", "dotk", "dottf", "dott", "dottf2", "dott2"):
        v, e = O.loop(m, x, y)
        assert float(v) == D and e == 0, m


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_literal_dots_are_sum_loops_over_rounded_products(dt):
    """dot, dotk, dottf, dott = sum, sumk, sumtf, sumt of RN(x_i * y_i), the
    rounding done by numpy (not by the oracle), on inexact products of mixed
    magnitudes so that every loop's compensation is non-zero."""
    n = 40001
    x = I.normal(n, dt, seed=31).numpy()
    y = I.normal(n, dt, seed=31, stream=2).numpy()
    y[::3] *= x.dtype.type(1e-3)
    p = np.multiply(x, y)                 # RN(x_i * y_i) in the data type
    assert p.dtype == x.dtype
    for dm, sm in (("dot", "sum"), ("dotk", "sumk"), ("dottf", "sumtf"), ("dott", "sumt")):
        vd, ed = O.loop(dm, x, y)
        vs, es = O.loop(sm, p)
        assert vd.tobytes() == vs.tobytes() and ed.tobytes() == es.tobytes(), dm
        if dm != "dot":
            assert ed != 0, dm


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_kahan_dot_bound(dt):
    """Kahan's dot (Example 2 with the rounded product as the item) against
    the exact dot: |s - sum x_i y_i| <= u sum|x_i y_i| (the products' own
    roundings) + (2u + 4 n u^2)(1 + u) sum|x_i y_i| (compensated summation of
    the rounded products, Goldberg 1991 / Higham 2002 Thm 4.8); the
    compensated value beats the direct dot on the same data."""
    n = 100000
    u = 2.0 ** -24 if dt == "f32" else 2.0 ** -53
    x = I.uniform(n, dt, seed=32, lo=0.0).numpy()
    y = I.uniform(n, dt, seed=32, stream=4, lo=0.0).numpy()
    s, c = O.loop("dotk", x, y)
    r = O.exact(x, y, v=float(s))
    assert abs(r.rv) <= (u + (2 * u + 4 * n * u * u) * (1 + u)) * r.sabs
    d, _ = O.loop("dot", x, y)
    rd = O.exact(x, y, v=float(d))
    assert abs(r.rv) < abs(rd.rv)


def gamma(k, u):
    return k * u / (1 - k * u)


@pytest.mark.parametrize("dt,cond", [("f32", 1e3), ("f32", 1e6), ("f64", 1e8), ("f64", 1e14)])
def test_rigorous_sum_error_bound(dt, cond):
    n = 20000
    ic = I.ill_conditioned(n, dt, cond, seed=11)
    x = ic.x.numpy()
    u = 2.0 ** -24 if dt == "f32" else 2.0 ** -53
    v, e = O.loop("sumt", x)
    r = O.exact(x, v=float(v), e=float(e))
    assert abs(r.r) <= u * abs(r.s) + gamma(n - 1, u) ** 2 * r.sabs
    # the plain value alone is far worse on such data
    assert abs(r.rv) > abs(r.r)
    # and the TwoProduct dot obeys the same bound on its terms
    icd = I.ill_conditioned(n, dt, cond, seed=12, dot=True)
    v, e = O.loop("dott2", icd.x.numpy(), icd.y.numpy())
    rd = O.exact(icd.x.numpy(), icd.y.numpy(), v=float(v), e=float(e))
    assert abs(rd.r) <= u * abs(rd.s) + gamma(2 * n, u) ** 2 * rd.sabs


def test_dot_twoproduct_on_inexact_products():
    x = I.normal(30000, "f32", seed=13).numpy()
    y = I.normal(30000, "f32", seed=13, stream=7).numpy()
    u = 2.0 ** -24
    v, e = O.loop("dott2", x, y)
    r = O.exact(x, y, v=float(v), e=float(e))
    assert abs(r.r) <= u * abs(r.s) + gamma(2 * x.size, u) ** 2 * r.sabs
    # without TwoProduct the lost product errors dominate the residual
    v1, e1 = O.loop("dott", x, y)
    r1 = O.exact(x, y, v=float(v1), e=float(e1))
    assert abs(r1.r) > 10 * abs(r.r)


def test_kahan_bound():
    x = I.uniform(100000, "f32", seed=14, lo=0.0).numpy()
    s, _ = O.loop("sumk", x)
    r = O.exact(x, v=float(s))
    u = 2.0 ** -24
    assert abs(r.rv) <= (2 * u + 4 * x.size * u * u) * r.sabs


def test_wide_accumulators():
    x = I.normal(100000, "f32", seed=15).numpy()
    y = I.normal(100000, "f32", seed=15, stream=9).numpy()
    s, _ = O.loop("sumd", x)
    d, _ = O.loop("dotd", x, y)
    u = 2.0 ** -53
    rs = O.exact(x, v=float(s))
    rd = O.exact(x, y, v=float(d))
    assert abs(rs.rv) <= gamma(x.size, u) * rs.sabs
    assert abs(rd.rv) <= gamma(x.size, u) * rd.sabs
    xd = I.normal(100000, "f64", seed=15).numpy()
    q, ql = O.loop("sumq", xd)
    rq = O.exact(xd, v=float(q), e=float(ql))
    assert abs(rq.r) <= gamma(xd.size, 2.0 ** -113) * rq.sabs + 2.0 ** -1074


@pytest.mark.parametrize("lo", [0.0, -1.0])
def test_accuracy_table_magnitudes(lo):
    """First Table 2: 1M uniform binary32 numbers; twofold fast tracks the
    exact sum to ~1e-10 relative or better, direct summation to 1e-7..1e-3."""
    x = I.uniform(1000000, "f32", seed=16, lo=lo).numpy()
    s, _ = O.loop("sum", x)
    v, e = O.loop("sumtf", x)
    k, _ = O.loop("sumk", x)
    ex = O.exact(x, v=float(v), e=float(e))
    S = ex.s
    rel_direct = abs(float(s) - S) / abs(S)
    rel_tf = abs(ex.r) / abs(S)
    rel_k = abs(float(k) - S) / abs(S)
    assert 1e-9 < rel_direct < 1e-2
    assert rel_tf < 1e-9
    assert rel_k < 1e-6


def test_error_growth_with_n():
    """Accuracy against N (the paper's closing remarks on how the errors
    grow): on positive uniform binary32 data the direct sum's relative error
    grows with N and stays within its gamma_{N-1} bound, while the rigorous
    twofold pair stays near u^2 N, far below the direct error, for all
    N < 1/u."""
    u = 2.0 ** -24
    prev = 0.0
    for k in (10, 14, 18, 22):
        n = 1 << k
        x = I.uniform(n, "f32", seed=20 + k, lo=0.0).numpy()
        s, _ = O.loop("sum", x)
        v, e = O.loop("sumt", x)
        ex = O.exact(x, v=float(v), e=float(e))
        S = ex.s
        rel_direct = abs(float(s) - S) / S
        rel_twofold = abs(ex.r) / S
        assert rel_direct <= (n - 1) * u / (1 - (n - 1) * u)
        assert rel_twofold <= u + 4 * (n * u) ** 2
        assert rel_twofold < rel_direct * 1e-3 or rel_direct == 0.0
        if k >= 14:
            assert rel_direct > prev          # grows with N on this data
        prev = rel_direct
