"""Pins for the oracle's error-free transforms (CPU only).

The statements pinned here are Theorem 1 (Dekker FAST-TWO-SUM: x + y = a + b
when |a| >= |b|) and Theorem 2 (Knuth TWO-SUM: x + y = a + b for any a, b,
p >= 3) of the Algorithms section, and the definition of TwoProduct
(p = RN(ab), e = RN(ab - p), so p + e = ab unless ab underflows).

1. The algorithms themselves are checked exhaustively in tiny binary formats
   (p = 3..5 bits, every pair of values) built on exact rationals.
2. The oracle's C primitives are checked exhaustively on structured binary32
   sets (all pairs) and on random binary64 samples against exact rationals.
"""
from fractions import Fraction
import itertools
import math

import numpy as np
import pytest

import oracle as O


# ----------------------------------------------------------- tiny formats
class Tiny:
    """binary format with p significand bits, normal exponents emin..emax,
    gradual underflow and round-to-nearest-even; values are Fractions."""

    def __init__(self, p, emin, emax):
        self.p, self.emin, self.emax = p, emin, emax
        self.q0 = Fraction(2) ** (emin - p + 1)            # smallest quantum
        self.big = (2 - Fraction(2) ** (1 - p)) * Fraction(2) ** emax

    def values(self):
        out = {Fraction(0)}
        for m in range(1, 2 ** self.p):                     # subnormals and exponent emin
            out.add(m * self.q0)
        for e in range(self.emin + 1, self.emax + 1):
            for m in range(2 ** (self.p - 1), 2 ** self.p):
                out.add(m * Fraction(2) ** (e - self.p + 1))
        pos = sorted(out)
        return [-v for v in reversed(pos[1:])] + pos

    def rn(self, x):
        """round a rational to the format; None on overflow"""
        if x == 0:
            return Fraction(0)
        s = -1 if x < 0 else 1
        a = abs(x)
        e = math.floor(math.log2(a))
        while Fraction(2) ** e > a:
            e -= 1
        while Fraction(2) ** (e + 1) <= a:
            e += 1
        q = max(Fraction(2) ** (e - self.p + 1), self.q0)
        k = a / q
        f = math.floor(k)
        r = k - f
        if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
            f += 1
        v = f * q
        if v > self.big:
            return None
        return s * v


class _Overflow(Exception):
    pass


def _r(F, v):
    r = F.rn(v)
    if r is None:
        raise _Overflow
    return r


def tiny_fast_two_sum(F, a, b):
    """FAST-TWO-SUM steps 1-3 in the tiny format; None if a step overflows"""
    try:
        x = _r(F, a + b)
        bv = _r(F, x - a)
        y = _r(F, b - bv)
    except _Overflow:
        return None
    return x, y


def tiny_two_sum(F, a, b):
    """TWO-SUM steps 1-6 in the tiny format; None if a step overflows"""
    try:
        x = _r(F, a + b)
        bv = _r(F, x - a)
        av = _r(F, x - bv)
        bs = _r(F, b - bv)
        as_ = _r(F, a - av)
        y = _r(F, as_ + bs)
    except _Overflow:
        return None
    return x, y


def tiny_two_product(F, a, b):
    try:
        p = _r(F, a * b)
        return p, _r(F, a * b - p)
    except _Overflow:
        return None


@pytest.mark.parametrize("p,emin,emax", [(3, -3, 3), (4, -3, 3), (5, -2, 2)])
def test_tiny_two_sum_error_free_all_pairs(p, emin, emax):
    F = Tiny(p, emin, emax)
    vals = F.values()
    n = 0
    for a, b in itertools.product(vals, vals):
        r = tiny_two_sum(F, a, b)
        if r is None:
            continue
        x, y = r
        assert x + y == a + b, (a, b, x, y)
        assert x == F.rn(a + b)
        n += 1
    assert n > 0.9 * len(vals) ** 2


@pytest.mark.parametrize("p,emin,emax", [(3, -3, 3), (4, -3, 3), (5, -2, 2)])
def test_tiny_fast_two_sum_precondition_and_counterexamples(p, emin, emax):
    F = Tiny(p, emin, emax)
    vals = F.values()
    bad = 0
    for a, b in itertools.product(vals, vals):
        r = tiny_fast_two_sum(F, a, b)
        if r is None:
            continue
        x, y = r
        if abs(a) >= abs(b):
            assert x + y == a + b, (a, b, x, y)
        elif x + y != a + b:
            bad += 1
    # without the precondition the transform is not error-free (Theorem 1's
    # hypothesis matters): counterexamples exist in every format
    assert bad > 0


@pytest.mark.parametrize("p,emin,emax", [(3, -4, 3), (4, -4, 3)])
def test_tiny_two_product_definition(p, emin, emax):
    F = Tiny(p, emin, emax)
    vals = F.values()
    lost = 0
    for a, b in itertools.product(vals, vals):
        r = tiny_two_product(F, a, b)
        if r is None:
            continue
        pp, e = r
        # exact whenever the residual is representable, i.e. no underflow
        if pp + e != a * b:
            lost += 1
            assert abs(a * b) < Fraction(2) ** (emin + p), (a, b)
    assert lost > 0      # underflow does break it, as the definition predicts


# ------------------------------------------------- binary32, C primitives
def structured_f32(exps, nsig=48, seed=1):
    rng = np.random.default_rng(seed)
    sig = rng.integers(1 << 23, 1 << 24, size=nsig, dtype=np.int64)
    sig[0], sig[1] = 1 << 23, (1 << 24) - 1
    vals = []
    for e in exps:
        for m in sig:
            for s in (1.0, -1.0):
                vals.append(s * math.ldexp(float(m), int(e) - 23))
    return np.array(vals, dtype=np.float32)


def all_pairs(v):
    a = np.repeat(v, v.size)
    b = np.tile(v, v.size)
    return a, b


@pytest.mark.parametrize("exps", [range(-8, 8), range(100, 116), range(-126, -110)])
def test_c_two_sum_f32_exhaustive_structured(exps):
    a, b = all_pairs(structured_f32(exps))
    x, y = O.two_sum(a, b)
    ad, bd = a.astype(np.float64), b.astype(np.float64)
    exact = ad + bd                      # exact: exponents within 16, 24-bit significands
    assert np.all(x == exact.astype(np.float32))
    assert np.all(x.astype(np.float64) + y.astype(np.float64) == exact)


@pytest.mark.parametrize("exps", [range(-8, 8), range(-149, -133)])
def test_c_fast_two_sum_f32_exhaustive_structured(exps):
    a, b = all_pairs(structured_f32(exps))
    x, y = O.fast_two_sum(a, b)
    exact = a.astype(np.float64) + b.astype(np.float64)
    ok = np.abs(a) >= np.abs(b)
    assert np.all((x.astype(np.float64) + y.astype(np.float64) == exact)[ok])
    assert np.all(x == exact.astype(np.float32))
    if exps[0] > -140:        # in the subnormal window every sum is exact
        assert np.any((x.astype(np.float64) + y.astype(np.float64) != exact)[~ok])


def test_c_two_sum_f32_subnormal_and_overflow():
    tiny = structured_f32(range(-149, -133))
    a, b = all_pairs(tiny)
    x, y = O.two_sum(a, b)
    assert np.all(y == 0)                            # sums of subnormals are exact
    assert np.all(x.astype(np.float64) == a.astype(np.float64) + b.astype(np.float64))
    big = structured_f32(range(120, 128))
    a, b = all_pairs(big)
    x, y = O.two_sum(a, b)
    exact = a.astype(np.float64) + b.astype(np.float64)
    ovf = np.abs(exact) >= 2.0 ** 128 - 2.0 ** 103      # RN overflow threshold
    assert np.all(np.isinf(x[ovf]))
    assert np.all(np.isfinite(x[~ovf]))
    # Theorem 2 assumes no overflow in any step; where a step overflows the
    # error term is not finite, otherwise the identity holds
    fin = ~ovf & np.isfinite(y)
    assert fin.sum() > 0.5 * (~ovf).sum()
    assert np.all(x[fin].astype(np.float64) + y[fin].astype(np.float64) == exact[fin])


@pytest.mark.parametrize("exps", [range(-8, 8), range(-80, -64), range(56, 72)])
def test_c_two_product_f32_exhaustive_structured(exps):
    a, b = all_pairs(structured_f32(exps))
    p, e = O.two_product(a, b)
    ab = a.astype(np.float64) * b.astype(np.float64)           # exact in binary64
    with np.errstate(over="ignore"):
        assert np.all(p == (a * b))                                # p = RN32(ab)
        fin = np.isfinite(p)
        # e = RN32(ab - p): ab - p is exact in binary64
        assert np.all(e[fin] == (ab[fin] - p[fin].astype(np.float64)).astype(np.float32))
        normal = fin & (np.abs(ab) >= 2.0 ** -102)
        assert np.all(p[normal].astype(np.float64) + e[normal].astype(np.float64) == ab[normal])
        # overflow: p infinite, e the opposite infinity
        assert np.all(np.isinf(e[~fin]) & (np.sign(e[~fin]) == -np.sign(p[~fin])))


def test_c_two_product_f32_underflow_sign_of_zero():
    a = np.array([1e-30, -1e-30, 1e-30, 3e-39], dtype=np.float32)
    b = np.array([1e-30, 1e-30, -1e-25, 0.5], dtype=np.float32)
    p, e = O.two_product(a, b)
    ab = a.astype(np.float64) * b.astype(np.float64)
    assert np.all(p == a * b)
    assert np.all(np.signbit(p) == np.signbit(ab))
    assert np.all(e == (ab - p.astype(np.float64)).astype(np.float32))
    assert np.all(np.signbit(e[:3]) == np.signbit(ab[:3]))   # lost residual keeps its sign


# ------------------------------------------------- binary64, C primitives
def random_f64(n, seed, emin=-1074, emax=1023):
    rng = np.random.default_rng(seed)
    m = rng.random(n) + 1.0
    e = rng.integers(emin, emax, size=n)
    s = rng.choice([-1.0, 1.0], size=n)
    return np.array([s[i] * math.ldexp(m[i], int(e[i])) for i in range(n)], dtype=np.float64)


def test_c_two_sum_f64_random_exact_rationals():
    a = random_f64(20000, 2, -60, 60)
    b = random_f64(20000, 3, -60, 60)
    b[:5000] = a[:5000] * (1 + 2.0 ** -40)          # near cancellation
    x, y = O.two_sum(a, b)
    for i in range(a.size):
        assert x[i] == a[i] + b[i]
        assert Fraction(x[i]) + Fraction(y[i]) == Fraction(a[i]) + Fraction(b[i])
    xf, yf = O.fast_two_sum(a, b)
    ok = np.abs(a) >= np.abs(b)
    for i in np.nonzero(ok)[0][:5000]:
        assert Fraction(xf[i]) + Fraction(yf[i]) == Fraction(a[i]) + Fraction(b[i])


def test_c_two_product_f64_random_exact_rationals():
    a = np.concatenate([random_f64(8000, 4, -600, 600), random_f64(2000, 5, -1074, -900),
                        random_f64(1000, 6, 500, 1023)])
    b = np.concatenate([random_f64(8000, 7, -600, 600), random_f64(2000, 8, -200, 100),
                        random_f64(1000, 9, 0, 600)])
    p, e = O.two_product(a, b)
    with np.errstate(over="ignore", under="ignore"):
        assert np.all(p == a * b)
    for i in range(a.size):
        if not math.isfinite(p[i]):
            assert math.isinf(e[i]) and (e[i] > 0) != (p[i] > 0)
            continue
        ab = Fraction(a[i]) * Fraction(b[i])
        d = ab - Fraction(p[i])
        want = float(d) if d != 0 else 0.0     # int/int division in Python rounds correctly
        assert e[i] == want and (d == 0 or math.copysign(1, e[i]) == (1 if d > 0 else -1)), i
        if abs(ab) >= Fraction(2) ** -969:
            assert Fraction(p[i]) + Fraction(e[i]) == ab


def test_c_specials_propagate():
    a = np.array([np.inf, np.nan, np.inf, 0.0], dtype=np.float64)
    b = np.array([1.0, 1.0, 0.0, np.inf], dtype=np.float64)
    p, e = O.two_product(a, b)
    assert np.isinf(p[0]) and np.isnan(e[0])
    assert np.isnan(p[1]) and np.isnan(p[2]) and np.isnan(p[3])
    x, y = O.two_sum(a, b)
    assert np.isinf(x[0]) and np.isnan(y[0])
