"""Pins for the oracle's exact superaccumulator (CPU only).

The superaccumulator is the plain definition S = sum x_i (or sum x_i*y_i,
products unrounded), rounded once.  It is pinned by brute force with Python's
exact rationals on small random sets spanning the whole exponent range, by
closed forms, by invariances (permutation, thread count, negation) and by a
construction whose exact sum is known independently (the ill-conditioned
recipe of the input module).
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle as O
from paper_1401_0248_gb300 import inputs as I


def rn32(F):
    """nearest binary32 to a rational, ties to even, by search"""
    if abs(F) >= 2 ** 128 - 2 ** 103:                   # RN overflow threshold
        return np.float32(np.inf) if F > 0 else np.float32(-np.inf)
    c = np.float32(float(F))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        if not np.isfinite(cand):
            continue
        d = abs(Fraction(float(cand)) - F)
        key = (d, int(np.frombuffer(np.float32(cand).tobytes(), np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def rand_wide(n, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.float32:
        e = rng.integers(-149, 126, size=n)
    else:
        e = rng.integers(-1074, 1020, size=n)
    m = rng.random(n) + 1.0
    s = rng.choice([-1.0, 1.0], size=n)
    v = np.array([s[i] * math.ldexp(m[i], int(e[i])) for i in range(n)])
    return v.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("seed", range(6))
def test_exact_sum_brute_force(dtype, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 40))
    if seed % 2:
        x = rand_wide(n, dtype, seed)
    else:   # clustered exponents, cancellation
        x = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4)).astype(dtype)
        x = np.concatenate([x, -x[: n // 2]]).astype(dtype)
    F = sum((Fraction(float(v)) for v in x), Fraction(0))
    v = float(x[0]) if x.size else 0.0
    e = float(x[-1]) * 2.0 ** -30
    r = O.exact(x, v=v, e=e)
    assert r.cls == 0
    assert r.s == float(F)
    assert r.s32 == rn32(F)
    assert r.s_lo == float(F - Fraction(r.s))
    assert r.rv == float(F - Fraction(v))
    assert r.r == float(F - Fraction(v) - Fraction(e))
    assert r.sabs == float(sum((abs(Fraction(float(t))) for t in x), Fraction(0)))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("seed", range(4))
def test_exact_dot_brute_force(dtype, seed):
    n = 30
    x = rand_wide(n, dtype, 10 + seed)
    y = rand_wide(n, dtype, 20 + seed)
    if dtype == np.float32:      # keep products finite: exponent sum within range
        y = (y / np.float32(2.0 ** 60)).astype(dtype)
    else:
        x = (x / 2.0 ** 500).astype(dtype)
        y = (y / 2.0 ** 500).astype(dtype)
    F = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))
    r = O.exact(x, y)
    assert r.s == float(F)
    assert r.s32 == rn32(F)
    assert r.s_lo == float(F - Fraction(r.s))


def test_exact_closed_forms():
    # k copies of 2^j
    for j in (-149, -20, 0, 100):
        x = np.full(1000, 2.0 ** j, dtype=np.float32)
        assert O.exact(x).s == 1000 * 2.0 ** j
    # x and -x interleaved: exactly zero
    x = I.normal(10001, "f64", seed=3).numpy()
    z = np.empty(2 * x.size)
    z[0::2], z[1::2] = x, -x
    r = O.exact(z)
    assert r.s == 0.0 and r.s_lo == 0.0 and r.cls == 0
    # carries: many copies of the largest finite value
    big = np.full(3 << 20, np.finfo(np.float64).max)
    assert O.exact(big).s == math.inf   # exact sum exceeds the binary64 range
    big32 = np.full(3 << 20, np.finfo(np.float32).max, dtype=np.float32)
    r = O.exact(big32)
    assert r.s == float(Fraction(float(np.finfo(np.float32).max)) * (3 << 20))
    # 3.6e6 copies of 0.1f: the exact real is 3.6e6 * RN32(0.1)
    t = np.full(3600000, 0.1, dtype=np.float32)
    assert O.exact(t).s == float(Fraction(float(np.float32(0.1))) * 3600000)


def test_exact_invariances():
    x = I.uniform(300001, "f64", seed=5).numpy()
    y = I.uniform(300001, "f64", seed=5, stream=1).numpy()
    r1 = O.exact(x, y, nthreads=1)
    r8 = O.exact(x, y, nthreads=8)
    perm = np.random.default_rng(0).permutation(x.size)
    rp = O.exact(x[perm], y[perm], nthreads=3)
    rn = O.exact(-x, y, nthreads=2)
    assert r1.s == r8.s == rp.s and r1.s_lo == r8.s_lo == rp.s_lo
    assert rn.s == -r1.s and rn.s_lo == -r1.s_lo


def test_exact_matches_constructed_sum():
    for dt, cond in (("f32", 1e4), ("f32", 1e8), ("f64", 1e16), ("f64", 1e30)):
        ic = I.ill_conditioned(1 << 15, dt, cond, seed=2)
        r = O.exact(ic.x.numpy())
        assert r.s == float(ic.S)
        assert r.s_lo == float(ic.S - Fraction(r.s))
        icd = I.ill_conditioned(1 << 15, dt, cond, seed=2, dot=True)
        rd = O.exact(icd.x.numpy(), icd.y.numpy())
        assert rd.s == float(icd.S)


def test_exact_specials():
    x = np.array([1.0, np.inf, 2.0])
    assert O.exact(x).cls == 2 and O.exact(x).s == math.inf
    x = np.array([1.0, -np.inf])
    assert O.exact(x).cls == 3
    x = np.array([np.inf, -np.inf])
    assert O.exact(x).cls == 1
    x = np.array([1.0, np.nan])
    assert O.exact(x).cls == 1
    a = np.array([np.inf, 1.0], dtype=np.float32)
    b = np.array([0.0, 1.0], dtype=np.float32)
    assert O.exact(a, b).cls == 1                 # Inf * 0
    assert O.exact(np.zeros(0)).s == 0.0


def test_exact_batched_equals_per_segment():
    L = I.csr_lengths(200, 1, 3000, seed=4)
    L[5] = 0
    L[17] = 0
    off = I.csr_offsets(L)
    x = I.normal(int(off[-1]), "f32", seed=4).numpy()
    y = I.uniform(int(off[-1]), "f32", seed=4).numpy()
    v = np.linspace(-1, 1, 200)
    out = O.exact_batched(x, off, y, v=v, e=v * 1e-9)
    for s in range(200):
        r = O.exact(x[off[s]:off[s + 1]], y[off[s]:off[s + 1]], v=v[s], e=v[s] * 1e-9)
        assert out[s]["s"] == r.s and out[s]["r"] == r.r and out[s]["sabs"] == r.sabs
    with pytest.raises(ValueError):
        O.exact_batched(x, np.array([0, 5, 3], dtype=np.int64))


def test_exact_add():
    assert O.exact_add(1.0, 2.0 ** -60) == 1.0
    assert O.exact_add(1.0, 2.0 ** -53, 2.0 ** -105) == 1.0 + 2.0 ** -52


def test_ill_conditioned_reaches_its_condition_number():
    """The generator's achieved cond = sum|x| / |sum x| (from the exact
    oracle) lies within a factor of 10 of the target, for sums and dots."""
    for dt, cond in (("f32", 1e4), ("f32", 1e8), ("f64", 1e8), ("f64", 1e16), ("f64", 1e24)):
        for dot in (False, True):
            ic = I.ill_conditioned(1 << 16, dt, cond, seed=4, dot=dot)
            r = O.exact(ic.x.numpy(), ic.y.numpy() if dot else None)
            got = r.sabs / abs(r.s)
            assert cond / 10 <= got <= cond * 10, (dt, cond, dot, got)
