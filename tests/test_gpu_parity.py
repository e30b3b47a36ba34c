"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar: the error-free transforms are bit-identical to the oracle's; every
reduction's (value, error) is bit-identical to the oracle's sequential replay
of the documented order for the launch shape in use; rigorous results also
satisfy |S - (v+e)| <= u|S| + gamma_D^2 sum|x| against the exact oracle.
Sizes span several blocks / tiles and ragged tails; edge cases: n = 0, 1,
< one vector, misaligned pointers, empty segments, invalid offsets.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_0248_gb300 import inputs as I
from paper_1401_0248_gb300 import twofold as tf
from _helpers import U32, U64, csr_depth, flat_depth, same_bits, twofold_bound

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TD = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(DEV)
    assert tf.sm_count() > 0, "libtwofold.so does not see an sm_103a device"


def _np(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------ primitives
def structured_f32(exps, nsig=40, seed=1):
    rng = np.random.default_rng(seed)
    sig = rng.integers(1 << 23, 1 << 24, size=nsig, dtype=np.int64)
    sig[0], sig[1] = 1 << 23, (1 << 24) - 1
    v = [s * np.ldexp(float(m), int(e) - 23) for e in exps for m in sig for s in (1.0, -1.0)]
    return np.array(v, dtype=np.float32)


def pairs(v):
    return np.repeat(v, v.size), np.tile(v, v.size)


F32_SETS = [range(-8, 8), range(-149, -133), range(-70, -54), range(112, 128)]


@pytest.mark.parametrize("name", ["fast_two_sum", "two_sum", "two_product"])
@pytest.mark.parametrize("exps", F32_SETS)
def test_prims_f32_bit_exact_structured(name, exps):
    a, b = pairs(structured_f32(exps))
    with np.errstate(all="ignore"):
        wx, wy = getattr(O, name)(a, b)
    gx, gy = tf.prim(name, torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV))
    assert same_bits(_np(gx), wx) and same_bits(_np(gy), wy)


def wide_f64(n, seed):
    rng = np.random.default_rng(seed)
    e = rng.integers(-1074, 1023, size=n)
    m = rng.random(n) + 1.0
    s = rng.choice([-1.0, 1.0], size=n)
    return (s * np.ldexp(m, e)).astype(np.float64)


@pytest.mark.parametrize("name", ["fast_two_sum", "two_sum", "two_product"])
def test_prims_f64_bit_exact_random(name):
    n = 1 << 20
    a = wide_f64(n, 1)
    b = wide_f64(n, 2)
    b[: n // 4] = a[: n // 4] * (1 + 2.0 ** -30)            # near cancellation
    b[n // 4: n // 2] = np.ldexp(np.random.default_rng(3).random(n // 4) + 1, -540)
    a[n // 4: n // 2] = np.ldexp(np.random.default_rng(4).random(n // 4) + 1, -530)  # subnormal products
    with np.errstate(all="ignore"):
        wx, wy = getattr(O, name)(a, b)
    gx, gy = tf.prim(name, torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV))
    assert same_bits(_np(gx), wx) and same_bits(_np(gy), wy)


def int_two_sum_cases(n, seed):
    """binary64 pairs that exercise every branch of the integer-pipe TWO-SUM:
    exponent gaps 0..60, ties, cancellation, carries into a new binade,
    near-overflow, tiny and subnormal operands, zeros and specials."""
    rng = np.random.default_rng(seed)
    k = n // 8
    a = np.ldexp(rng.random(n) + 1.0, rng.integers(-60, 60, size=n))
    gap = rng.integers(0, 61, size=n)
    b = np.ldexp(rng.random(n) + 1.0, (np.frexp(a)[1] - 1 - gap))
    sgn = rng.choice([-1.0, 1.0], size=(2, n))
    a, b = a * sgn[0], b * sgn[1]
    # ties: b = +-half an ulp of a (times an odd multiple of lower powers)
    ulp = np.spacing(np.abs(a[:k]))
    b[:k] = ulp * 0.5 * rng.choice([-1.0, 1.0], size=k) * (1 + 2.0 ** -rng.integers(1, 40, size=k))
    b[k:k + k // 2] = ulp[: k // 2] * 0.5 * rng.choice([-1.0, 1.0], size=k // 2)      # exact ties
    # cancellation and binade carries
    b[k + k // 2: 2 * k] = -a[k + k // 2: 2 * k] * (1 + np.ldexp(1.0, -rng.integers(1, 52, size=k - k // 2)))
    a[2 * k: 3 * k] = np.nextafter(np.ldexp(1.0, rng.integers(-20, 20, size=k)), 0)
    b[2 * k: 3 * k] = np.spacing(a[2 * k: 3 * k]) * rng.random(k) * 2
    # near overflow and near the lower limit of the integer path
    a[3 * k: 3 * k + 64] = np.finfo(np.float64).max * rng.random(64)
    b[3 * k: 3 * k + 64] = np.finfo(np.float64).max * rng.random(64)
    a[3 * k + 64: 3 * k + 128] = np.ldexp(rng.random(64) + 1, rng.integers(-1000, -960, size=64))
    b[3 * k + 64: 3 * k + 128] = np.ldexp(rng.random(64) + 1, rng.integers(-1074, -960, size=64))
    a[3 * k + 128: 3 * k + 136] = [0.0, -0.0, 0.0, 1.0, np.inf, -np.inf, np.nan, 5e-324]
    b[3 * k + 128: 3 * k + 136] = [0.0, -0.0, -0.0, -1.0, 1.0, np.inf, 1.0, -5e-324]
    return a, b


def test_int_two_sum_f64_bit_exact():
    a, b = int_two_sum_cases(1 << 21, 5)
    with np.errstate(all="ignore"):
        wx, wy = O.two_sum(a, b)
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    gx, gy = tf.prim("two_sum_int", ta, tb)
    hx, hy = tf.prim("two_sum", ta, tb)
    assert same_bits(_np(gx), wx) and same_bits(_np(gy), wy)
    assert same_bits(_np(gx), _np(hx)) and same_bits(_np(gy), _np(hy))
    gx, gy = tf.prim("two_sum_int", tb, ta)          # operand order
    assert same_bits(_np(gx), wx) and same_bits(_np(gy), wy)


def test_int_fast_two_sum_f64_bit_exact():
    """FAST-TWO-SUM on the integer pipe: the literal algorithm's bits for any
    order of magnitudes, including |a| < |b| where it loses error."""
    a, b = int_two_sum_cases(1 << 21, 8)
    rng = np.random.default_rng(10)
    k = 1 << 18
    a2 = np.ldexp(rng.random(k) + 1, rng.integers(-60, 2, size=k)) * rng.choice([-1.0, 1.0], size=k)
    b2 = np.ldexp(1.0, rng.integers(0, 10, size=k)) * rng.choice([-1.0, 1.0], size=k)
    b2[k // 2:] *= 1 + np.ldexp(1.0, -52) * rng.integers(0, 8, size=k - k // 2)
    a = np.concatenate([a, a2, b2])
    b = np.concatenate([b, b2, a2])
    with np.errstate(all="ignore"):
        wx, wy = O.fast_two_sum(a, b)
    gx, gy = tf.prim("fast_two_sum_int", torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV))
    assert same_bits(_np(gx), wx) and same_bits(_np(gy), wy)


def int_two_product_cases(n, seed):
    rng = np.random.default_rng(seed)
    a = np.ldexp(rng.random(n) + 1, rng.integers(-560, 560, size=n)) * rng.choice([-1.0, 1.0], size=n)
    b = np.ldexp(rng.random(n) + 1, rng.integers(-560, 560, size=n)) * rng.choice([-1.0, 1.0], size=n)
    k = n // 8
    b[:k] = np.ldexp(1.0, rng.integers(-10, 10, size=k))                        # exact products
    a[k:2 * k] = np.ldexp(np.floor(rng.random(k) * 2 ** 26) + 2 ** 26, -26)      # short significands,
    b[k:2 * k] = np.ldexp(np.floor(rng.random(k) * 2 ** 27) + 2 ** 27, -27)      # ties and carries
    a[2 * k:3 * k] = np.ldexp(rng.random(k) + 1, rng.integers(-1022, -400, size=k))   # near underflow
    b[2 * k:3 * k] = np.ldexp(rng.random(k) + 1, rng.integers(-700, -100, size=k))
    a[3 * k:4 * k] = np.ldexp(rng.random(k) + 1, rng.integers(400, 1023, size=k))     # near overflow
    b[3 * k:4 * k] = np.ldexp(rng.random(k) + 1, rng.integers(300, 1023, size=k))
    a[4 * k: 4 * k + 8] = [0.0, -0.0, np.inf, np.nan, 5e-324, 1e-310, 1e308, -1e-300]
    b[4 * k: 4 * k + 8] = [3.0, 2.0, 0.0, 1.0, 1e300, 1e10, 10.0, 1e-300]
    return a, b


def test_int_two_product_f64_bit_exact():
    a, b = int_two_product_cases(1 << 21, 6)
    with np.errstate(all="ignore"):
        wp, we = O.two_product(a, b)
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    gp, ge = tf.prim("two_product_int", ta, tb)
    assert same_bits(_np(gp), wp) and same_bits(_np(ge), we)
    gp, ge = tf.prim("two_product_int", tb, ta)
    assert same_bits(_np(gp), wp) and same_bits(_np(ge), we)


# ------------------------------------------------------------ flat path
VARIANTS = [("sum", "plain"), ("sum", "fast"), ("sum", "rigorous"), ("dot", "plain"),
            ("dot", "fast"), ("dot", "rigorous")]
SIZES = [0, 1, 3, 5, 1000, 65537, (1 << 20) + 13]


def run_flat(op, variant, x, y, out_f64=False):
    if op == "sum":
        return tf.sum(x, variant, out_f64=out_f64)
    return tf.dot(x, y, variant, out_f64=out_f64)


def check_flat(op, variant, dt, x, y, out_f64=False):
    out = _np(run_flat(op, variant, x, y, out_f64))
    xh, yh = _np(x), (_np(y) if y is not None else None)
    block, unroll, grid, _ = tf.launch_shape(op, False, TD[dt], variant, xh.size)
    want = O.replay_flat(op, variant, xh, yh, block=block, unroll=unroll, grid=grid, out_f64=out_f64)
    assert same_bits(out, want), (op, variant, dt, xh.size, out, want)
    return out, (block, unroll, grid)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("op,variant", VARIANTS + [("sum", "wide"), ("dot", "wide")])
@pytest.mark.parametrize("n", SIZES)
def test_flat_bit_exact_vs_replay(dt, op, variant, n):
    x = I.normal(n, dt, seed=n % 4000, device=DEV)
    y = I.normal(n, dt, seed=n % 4000, stream=3, device=DEV) if op == "dot" else None
    out, (block, unroll, grid) = check_flat(op, variant, dt, x, y)
    if dt == "f32" and variant != "plain":
        check_flat(op, variant, dt, x, y, out_f64=True)
    if n and variant == "rigorous":
        ex = O.exact(_np(x), _np(y) if y is not None else None, v=float(out[0]), e=float(out[1]))
        u = U32 if dt == "f32" else U64
        D = flat_depth(n, 4 if dt == "f32" else 2, block, unroll, grid)
        assert abs(ex.r) <= twofold_bound(ex.s, ex.sabs, u, D)


@pytest.mark.parametrize("dt,cond", [("f64", 1e8), ("f64", 1e16), ("f64", 1e30), ("f32", 1e8)])
def test_flat_ill_conditioned_bit_exact(dt, cond):
    """cancelling data makes |s| < |y| common, which exercises the binary64
    FAST-TWO-SUM's non-error-free branch and the exact-sum branches"""
    n = (1 << 20) + 7
    ic = I.ill_conditioned(n, dt, cond, seed=3, device=DEV)
    icd = I.ill_conditioned(n, dt, cond, seed=4, device=DEV, dot=True)
    for variant in ("fast", "rigorous", "plain"):
        check_flat("sum", variant, dt, ic.x, None)
        check_flat("dot", variant, dt, icd.x, icd.y)


def test_flat_wide_f64_binary128_special_values_bit_exact():
    """binary64 data in the binary128 accumulator: zeros, subnormals, huge
    values, and Inf/NaN propagation"""
    rng = np.random.default_rng(21)
    n = 100003
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    y = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    x[::7] = 0.0
    x[1::11] = -0.0
    x[2::13] = 5e-324
    y[3::17] = -2.5e-310
    tx, ty = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    check_flat("sum", "wide", "f64", tx, None)
    check_flat("dot", "wide", "f64", tx, ty)
    # exactness where every partial sum fits in 113 bits: integers
    xi = torch.from_numpy(rng.integers(-2 ** 50, 2 ** 50, size=n).astype(np.float64)).to(DEV)
    out = _np(tf.sum(xi, "wide"))
    ex = O.exact(_np(xi))
    assert out[0] == ex.s and out[1] == ex.s_lo
    xs = x.copy()
    xs[5] = np.inf
    check_flat("sum", "wide", "f64", torch.from_numpy(xs).to(DEV), None)
    xs[6] = -np.inf
    check_flat("sum", "wide", "f64", torch.from_numpy(xs).to(DEV), None)


def test_flat_wide_special_values_bit_exact():
    """zeros, subnormals and huge binary32 values take the hardware widening"""
    rng = np.random.default_rng(12)
    n = 200003
    x = (rng.standard_normal(n) * 10.0 ** rng.integers(-45, 38, size=n)).astype(np.float32)
    y = (rng.standard_normal(n) * 10.0 ** rng.integers(-45, 38, size=n)).astype(np.float32)
    x[::7] = 0.0
    x[1::11] = -0.0
    y[2::13] = np.float32(1e-45)
    x[3::17] = np.float32(3e-39)
    with np.errstate(over="ignore"):
        assert np.isfinite(x).all() and np.isfinite(y).all()
    tx, ty = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    check_flat("sum", "wide", "f32", tx, None)
    check_flat("dot", "wide", "f32", tx, ty)
    check_flat("sum", "wide", "f32", tx, None, out_f64=True)
    check_flat("dot", "wide", "f32", tx, ty, out_f64=True)


# the paper's Kahan summation (Example 2) and its literal dot forms
EXTRA = [("sum", "kahan", False), ("dot", "kahan", False), ("dot", "fast", True),
         ("dot", "rigorous", True)]


def oracle_variant(variant, literal):
    return variant + "_literal" if literal else variant


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("op,variant,literal", EXTRA)
@pytest.mark.parametrize("n", [1, 7, 65537, (1 << 20) + 3])
def test_flat_kahan_and_literal_dots_bit_exact(dt, op, variant, literal, n):
    x = I.normal(n, dt, seed=n % 4000 + 7, device=DEV)
    y = I.normal(n, dt, seed=n % 4000 + 7, stream=3, device=DEV)
    for out_f64 in ((False, True) if dt == "f32" else (False,)):
        if op == "sum":
            got = _np(tf.sum(x, variant, out_f64=out_f64))
        else:
            got = _np(tf.dot(x, y, variant, out_f64=out_f64, literal=literal))
        block, unroll, grid, _ = tf.launch_shape(op, False, TD[dt], variant, n)
        want = O.replay_flat(op, oracle_variant(variant, literal), _np(x),
                             _np(y) if op == "dot" else None, block=block, unroll=unroll,
                             grid=grid, out_f64=out_f64)
        assert same_bits(got, want), (dt, op, variant, literal, n)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_csr_kahan_and_literal_dots_bit_exact(dt):
    off_h = make_csr(200, 1, 30000, seed=15, empties=(3, 4))
    n = int(off_h[-1])
    x = I.normal(n, dt, seed=16, device=DEV)
    y = I.normal(n, dt, seed=16, stream=2, device=DEV)
    off = torch.from_numpy(off_h).to(DEV)
    for op, variant, literal in EXTRA:
        if op == "sum":
            got = _np(tf.sum_batched(x, off, variant))
        else:
            got = _np(tf.dot_batched(x, y, off, variant, literal=literal))
        _, unroll, _, tile = tf.launch_shape(op, True, TD[dt], variant, n)
        want = O.replay_csr(op, oracle_variant(variant, literal), _np(x), off_h,
                            _np(y) if op == "dot" else None, unroll=unroll, tile=tile)
        assert same_bits(got, want), (dt, op, variant, literal)


def test_kahan_accuracy_between_direct_and_twofold():
    """the paper's accuracy table ordering on uniform data: direct worst,
    Kahan and twofold fast far better (binary32, 1M elements)"""
    x = I.uniform(1 << 20, "f32", seed=17, lo=0.0, device=DEV)
    ex = O.exact(_np(x))
    d = _np(tf.sum(x, "plain", out_f64=True))
    k = _np(tf.sum(x, "kahan", out_f64=True))
    t = _np(tf.sum(x, "fast", out_f64=True))
    err = lambda v, e=0.0: abs(float(O.exact_add(ex.s, ex.s_lo, -v, -e))) / ex.s
    assert err(k[0], k[1]) < err(d[0]) and err(t[0], t[1]) < err(d[0])


def test_count_large_errors():
    rng = np.random.default_rng(18)
    for dt in (np.float32, np.float64):
        pairs = np.stack([rng.standard_normal(100000), rng.standard_normal(100000) * 1e-6], 1).astype(dt)
        pairs[::97, 1] = pairs[::97, 0] * 0.5           # large relative errors
        pairs[5, 0] = np.nan
        pairs[6, 1] = np.inf
        tau = 1e-3
        want = int(np.sum(~((np.abs(pairs[:, 1].astype(np.float64)) <= tau * np.abs(pairs[:, 0].astype(np.float64)))
                            & np.isfinite(pairs[:, 0]) & np.isfinite(pairs[:, 1]))))
        got = tf.count_large_errors(torch.from_numpy(pairs).to(DEV), tau)
        assert int(got.item()) == want
    # chained after a batched reduction, on the device
    off_h = make_csr(50, 1, 1000, seed=19)
    x = I.normal(int(off_h[-1]), "f32", seed=19, device=DEV)
    out = tf.sum_batched(x, torch.from_numpy(off_h).to(DEV), "rigorous")
    cnt = tf.count_large_errors(out, 0.0)
    o = _np(out)
    assert int(cnt.item()) == int(np.sum(o[:, 1] != 0))


@pytest.mark.parametrize("block,unroll,bps", [(128, 1, 1), (256, 4, 8), (512, 2, 4), (128, 4, 2)])
def test_flat_every_plan_shape(block, unroll, bps):
    n = 300007
    for dt in ("f32", "f64"):
        x = I.uniform(n, dt, seed=9, device=DEV)
        y = I.uniform(n, dt, seed=9, stream=1, device=DEV)
        cls = tf.plan_class(n)
        for op, variant in VARIANTS:
            before = tf.plan_get(op, cls, TD[dt], variant)
            try:
                tf.plan_set(op, cls, TD[dt], variant, block, unroll, bps)
                assert tf.launch_shape(op, False, TD[dt], variant, n)[:2] == (block, unroll)
                check_flat(op, variant, dt, x, y if op == "dot" else None)
            finally:
                tf.plan_set(op, cls, TD[dt], variant, before["block"], before["unroll"],
                            before["blocks_per_sm"])


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("blocks", [1, 2, 3, 7])
def test_flat_last_block_done_with_few_blocks(dt, blocks):
    """The last-block-done grid fold with 1, 2 and odd block counts (and a
    partial last vector), bit for bit against the replay."""
    V = 4 if dt == "f32" else 2
    n = 128 * V * blocks - (V - 1)
    cls = tf.plan_class(n)
    x = I.normal(n, dt, seed=blocks, device=DEV)
    y = I.normal(n, dt, seed=blocks, stream=2, device=DEV)
    for op, variant in (("sum", "rigorous"), ("dot", "fast"), ("sum", "kahan")):
        before = tf.plan_get(op, cls, TD[dt], variant)
        try:
            tf.plan_set(op, cls, TD[dt], variant, 128, 1, 8)
            assert tf.launch_shape(op, False, TD[dt], variant, n)[2] == blocks
            check_flat(op, variant, dt, x, y if op == "dot" else None)
        finally:
            tf.plan_set(op, cls, TD[dt], variant, before["block"], before["unroll"],
                        before["blocks_per_sm"])


def test_flat_partial_sums_overflow_with_finite_exact_sum():
    """Partial sums that overflow while the exact sum is 0: the result follows
    the documented order (Inf/NaN where its additions overflow), matching the
    replay; reported, not bound-checked."""
    big = np.full(4096, 1.5e308)
    x = np.concatenate([big, -big])
    xt = torch.from_numpy(x).to(DEV)
    for variant in ("fast", "rigorous", "plain"):
        check_flat("sum", variant, "f64", xt, None)
    xi = torch.from_numpy(np.ascontiguousarray(np.stack([big, -big], 1).reshape(-1))).to(DEV)
    for variant in ("fast", "rigorous"):
        check_flat("sum", variant, "f64", xi, None)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_flat_misaligned_pointers_same_bits(dt):
    n = 200003
    base = I.normal(n + 3, dt, seed=4, device=DEV)
    ybase = I.normal(n + 3, dt, seed=4, stream=1, device=DEV)
    for off in (1, 2, 3):
        x = base[off:off + n]               # element-aligned, not 16-byte aligned
        y = ybase[off:off + n]
        xc, yc = x.clone(), y.clone()      # 16-byte aligned copies
        for variant in ("fast", "rigorous", "plain"):
            a = _np(tf.sum(x, variant))
            b = _np(tf.sum(xc, variant))
            assert same_bits(a, b)
            a = _np(tf.dot(x, yc, variant))
            b = _np(tf.dot(xc, yc, variant))
            assert same_bits(a, b)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_csr_misaligned_pointers_same_bits(dt):
    """Batched inputs that are element-aligned but not 16-byte aligned load
    through registers (no shared-memory ring); the order, hence the bits, is
    the aligned call's."""
    off_h = make_csr(300, 1, 20000, seed=47, empties=(5, 6))
    n = int(off_h[-1])
    off = torch.from_numpy(off_h).to(DEV)
    base = I.normal(n + 3, dt, seed=5, device=DEV)
    ybase = I.normal(n + 3, dt, seed=5, stream=1, device=DEV)
    for k in (1, 3):
        x, y = base[k:k + n], ybase[k:k + n]
        xc, yc = x.clone(), y.clone()
        for variant in ("fast", "rigorous"):
            assert same_bits(_np(tf.sum_batched(x, off, variant)), _np(tf.sum_batched(xc, off, variant)))
            assert same_bits(_np(tf.dot_batched(x, y, off, variant)),
                             _np(tf.dot_batched(xc, yc, off, variant)))


def test_flat_special_values():
    x = torch.tensor([1.0, float("inf"), 2.0], device=DEV)
    out = _np(tf.sum(x, "fast"))
    assert np.isinf(out[0]) and np.isnan(out[1])
    x = torch.tensor([1.0, float("nan")], dtype=torch.float64, device=DEV)
    assert np.isnan(_np(tf.sum(x, "rigorous"))[0])
    z = torch.zeros(0, device=DEV)
    out = _np(tf.sum(z, "rigorous"))
    assert out[0] == 0 and out[1] == 0 and not np.signbit(out[0])
    # integers: every operation exact, so value = exact sum and error = 0
    xi = torch.randint(-100, 100, (1 << 20,), device=DEV).float()
    out = _np(tf.sum(xi, "rigorous"))
    assert float(out[0]) == float(xi.long().sum().item()) and out[1] == 0


# ------------------------------------------------------------ CSR path
def make_csr(nseg, lmin, lmax, seed, empties=()):
    L = I.csr_lengths(nseg, lmin, lmax, seed=seed)
    for k in empties:
        L[k] = 0
    return I.csr_offsets(L)


def check_csr(op, variant, dt, x, y, off_h, out_f64=False):
    off = torch.from_numpy(off_h).to(DEV)
    if op == "sum":
        out = tf.sum_batched(x, off, variant, out_f64=out_f64)
    else:
        out = tf.dot_batched(x, y, off, variant, out_f64=out_f64)
    got = _np(out)
    xh, yh = _np(x), (_np(y) if y is not None else None)
    _, unroll, _, tile = tf.launch_shape(op, True, TD[dt], variant, xh.size)
    want = O.replay_csr(op, variant, xh, off_h, yh, unroll=unroll, tile=tile, out_f64=out_f64)
    assert same_bits(got, want), (op, variant, dt)
    return got, unroll, tile


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("op,variant", VARIANTS + [("sum", "wide"), ("dot", "wide")])
def test_csr_bit_exact_vs_replay(dt, op, variant):
    off_h = make_csr(300, 1, 20000, seed=5, empties=(0, 7, 8, 299))
    n = int(off_h[-1]) + 5                      # x longer than the segments cover
    x = I.normal(n, dt, seed=6, device=DEV)
    y = I.normal(n, dt, seed=6, stream=2, device=DEV) if op == "dot" else None
    got, unroll, tile = check_csr(op, variant, dt, x, y, off_h)
    if dt == "f32" and variant in ("fast", "rigorous"):
        check_csr(op, variant, dt, x, y, off_h, out_f64=True)
    if variant == "rigorous":
        ex = O.exact_batched(_np(x), off_h, _np(y) if y is not None else None,
                             v=got[:, 0].astype(np.float64), e=got[:, 1].astype(np.float64))
        u = U32 if dt == "f32" else U64
        for s in range(300):
            L = int(off_h[s + 1] - off_h[s])
            D = csr_depth(max(L, 1), 4 if dt == "f32" else 2, unroll, tile)
            assert abs(ex[s]["r"]) <= twofold_bound(ex[s]["s"], ex[s]["sabs"], u, D)


@pytest.mark.parametrize("bps", [1, 4])
@pytest.mark.parametrize("tile", [1024, 4096, 16384])
def test_csr_tiles_and_long_segments(tile, bps):
    # one segment over many tiles, many tiny ones, and segments ending on tile
    # edges; one block per SM stages through the shared-memory ring (tiles of
    # 4096 and more), four per SM leave no room for it and load into registers
    L = [tile * 40 + 17, 1, 2, 3, tile - 6, tile, 0, 2 * tile, 5, 100000, 0, 0, 31]
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    for dt in ("f32", "f64"):
        x = I.uniform(n, dt, seed=8, device=DEV)
        y = I.uniform(n, dt, seed=8, stream=5, device=DEV)
        for op, variant in (("sum", "rigorous"), ("dot", "fast"), ("sum", "plain")):
            before = tf.plan_get(op, True, TD[dt], variant)
            try:
                tf.plan_set(op, True, TD[dt], variant, 256, 2, bps, tile)
                check_csr(op, variant, dt, x, y if op == "dot" else None, off_h)
            finally:
                tf.plan_set(op, True, TD[dt], variant, before["block"], before["unroll"],
                            before["blocks_per_sm"], before["tile"])


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_csr_segment_over_thousands_of_tiles(dt):
    """A segment over 2,501 tiles of 1024 (its pairwise tree of pieces runs
    twelve levels), between segments of 1 to 33 tiles and segments ending on
    tile edges; the variants whose cross-tile pair types differ (binary64,
    the binary128 accumulator), plain and the Kahan chains."""
    tile = 1024
    L = [5, tile - 5, tile * 2500 + 7, tile * 33 - 7, 1, tile * 32, 3, tile + 1]
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    x = I.normal(n, dt, seed=21, device=DEV)
    y = I.normal(n, dt, seed=21, stream=4, device=DEV)
    for op, variant in (("sum", "rigorous"), ("dot", "fast"), ("sum", "wide"), ("sum", "kahan"),
                        ("sum", "plain")):
        before = tf.plan_get(op, True, TD[dt], variant)
        try:
            tf.plan_set(op, True, TD[dt], variant, 256, 1, 2, tile)
            check_csr(op, variant, dt, x, y if op == "dot" else None, off_h)
        finally:
            tf.plan_set(op, True, TD[dt], variant, before["block"], before["unroll"],
                        before["blocks_per_sm"], before["tile"])


@pytest.mark.parametrize("tile", [1024, 4096])
@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("variant", ["fast", "rigorous", "kahan", "wide"])
def test_csr_pieces_at_each_power_of_two(dt, variant, tile):
    """Segments over exactly k tiles for k = 2..5, 8, 9, 16, 17, 31, 32 and 33
    (the merge kernel's butterfly over 2, 4, 8, 16 and 32 lanes on both sides
    of each power of two, and the first count that takes the arrival tree),
    each starting on a tile edge or inside a tile; tiles of 1024 run the
    register kernel, tiles of 4096 the shared-memory ring where it fits."""
    L = []
    for k in (2, 3, 4, 5, 8, 9, 16, 17, 31, 32, 33):
        L += [tile * k, 3, tile * (k - 1) - 3 + 1]     # k tiles from an edge; then k tiles from inside
        L.append(tile - ((sum(L)) % tile) if sum(L) % tile else 0)   # back to a tile edge
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    x = I.normal(n, dt, seed=33, device=DEV)
    y = I.normal(n, dt, seed=33, stream=6, device=DEV)
    for op in ("sum", "dot"):
        before = tf.plan_get(op, True, TD[dt], variant)
        try:
            tf.plan_set(op, True, TD[dt], variant, 128, 1, 2, tile)
            check_csr(op, variant, dt, x, y if op == "dot" else None, off_h)
        finally:
            tf.plan_set(op, True, TD[dt], variant, before["block"], before["unroll"],
                        before["blocks_per_sm"], before["tile"])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_csr_random_layouts(seed):
    """Random mixes of empty, short, about-one-tile and multi-tile segments
    (up to 40 tiles, so both the merge kernel and the arrival tree run), at a
    random tile size and launch shape; every pair bit for bit against the
    replay."""
    rng = np.random.default_rng(100 + seed)
    tile = int(rng.choice([1024, 2048, 4096]))
    kinds = rng.integers(0, 4, size=300)
    L = []
    for k in kinds:
        if k == 0:
            L.append(int(rng.integers(0, 3)))                       # empty or tiny
        elif k == 1:
            L.append(int(rng.integers(1, 200)))                     # short
        elif k == 2:
            L.append(int(tile + rng.integers(-64, 65)))             # about one tile
        else:
            L.append(int(rng.integers(2, 40) * tile + rng.integers(-500, 500)))   # many tiles
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    block = int(rng.choice([128, 256, 512]))
    bps = int(rng.choice([1, 2, 3]))
    for dt in ("f32", "f64"):
        x = I.normal(n, dt, seed=200 + seed, device=DEV)
        y = I.normal(n, dt, seed=200 + seed, stream=7, device=DEV)
        for op, variant in (("sum", "fast"), ("dot", "rigorous")):
            before = tf.plan_get(op, True, TD[dt], variant)
            try:
                tf.plan_set(op, True, TD[dt], variant, block, 1, bps, tile)
                check_csr(op, variant, dt, x, y if op == "dot" else None, off_h)
            finally:
                tf.plan_set(op, True, TD[dt], variant, before["block"], before["unroll"],
                            before["blocks_per_sm"], before["tile"])


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("unroll,block", [(1, 128), (2, 512), (4, 256)])
def test_csr_staged_ring_edges(dt, unroll, block):
    """The shared-memory ring of the batched kernel (16-byte-aligned inputs,
    tile 4096, one block per SM so that the ring fits): totals that end inside
    a 16-byte vector (the tail is read from global memory), totals below one
    vector, empty segments, pieces that start and end inside a chunk, and runs
    of tiles past the ring's depth."""
    tile = 4096
    cases = [[1], [3], [0, 5, 0], [tile * 3 + 3], [2, tile - 1, 7, tile * 2 + 1, 0, 9],
             [tile * 9 + 1, 1, 1], [17] * 700]
    for k, L in enumerate(cases):
        off_h = I.csr_offsets(L)
        n = int(off_h[-1])
        x = I.uniform(max(n, 1), dt, seed=40 + k, device=DEV)[:n]
        y = I.uniform(max(n, 1), dt, seed=40 + k, stream=3, device=DEV)[:n]
        for op, variant in (("sum", "rigorous"), ("dot", "fast"), ("sum", "kahan")):
            before = tf.plan_get(op, True, TD[dt], variant)
            try:
                tf.plan_set(op, True, TD[dt], variant, block, unroll, 1, tile)
                check_csr(op, variant, dt, x, y if op == "dot" else None, off_h)
            finally:
                tf.plan_set(op, True, TD[dt], variant, before["block"], before["unroll"],
                            before["blocks_per_sm"], before["tile"])


def test_workspace_reset_restores_a_scribbled_workspace():
    """A workspace filled with garbage (tickets, counters, flags) is zeroed by
    tf_workspace_reset, after which flat and batched calls on it give the
    replay's bits and no device error."""
    n = 300001
    x = I.normal(n, "f32", seed=44, device=DEV)
    off_h = make_csr(40, 1, 30000, seed=45)
    xs = I.normal(int(off_h[-1]), "f32", seed=46, device=DEV)
    nb = max(tf.workspace_size("sum", False, torch.float32, "rigorous", n),
             tf.workspace_size("sum", True, torch.float32, "rigorous", xs.numel(), 40))
    ws = torch.full((nb,), 0x5A, dtype=torch.uint8, device=DEV)
    tf.workspace_reset(ws)
    assert int(ws.max().item()) == 0
    got = _np(tf.sum(x, "rigorous", ws=ws))
    block, unroll, grid, _ = tf.launch_shape("sum", False, torch.float32, "rigorous", n)
    assert same_bits(got, O.replay_flat("sum", "rigorous", _np(x), block=block, unroll=unroll,
                                        grid=grid))
    off = torch.from_numpy(off_h).to(DEV)
    got = _np(tf.sum_batched(xs, off, "rigorous", ws=ws))
    _, unroll, _, tile = tf.launch_shape("sum", True, torch.float32, "rigorous", xs.numel())
    assert same_bits(got, O.replay_csr("sum", "rigorous", _np(xs), off_h, unroll=unroll, tile=tile))
    assert tf.device_error(ws) == 0


def test_csr_invalid_offsets_flagged_then_recovers():
    x = I.uniform(1000, "f32", seed=1, device=DEV)
    ws = tf.workspace(tf.workspace_size("sum", True, torch.float32, "fast", 1000, 4), DEV)
    tf.device_error(ws)                                     # clear
    bad = torch.tensor([0, 10, 5, 20, 30], dtype=torch.int64, device=DEV)
    out = _np(tf.sum_batched(x, bad, "fast", ws=ws))
    assert np.all(np.isnan(out))
    assert tf.device_error(ws) == 6                         # TF_ERR_OFFSETS
    beyond = torch.tensor([0, 10, 2000], dtype=torch.int64, device=DEV)
    out = _np(tf.sum_batched(x, beyond, "fast", ws=ws))
    assert np.all(np.isnan(out)) and tf.device_error(ws) == 6
    good = torch.tensor([0, 10, 500, 1000], dtype=torch.int64, device=DEV)
    got = _np(tf.sum_batched(x, good, "fast", ws=ws))
    assert tf.device_error(ws) == 0
    _, unroll, _, tile = tf.launch_shape("sum", True, torch.float32, "fast", 1000)
    want = O.replay_csr("sum", "fast", _np(x), _np(good), unroll=unroll, tile=tile)
    assert same_bits(got, want)


def test_csr_no_segments():
    x = I.uniform(10, "f32", seed=1, device=DEV)
    off = torch.zeros(1, dtype=torch.int64, device=DEV)
    assert tf.sum_batched(x, off, "fast").shape == (0, 2)
    allempty = torch.zeros(5, dtype=torch.int64, device=DEV)
    out = _np(tf.sum_batched(x, allempty, "rigorous"))
    assert np.all(out == 0)


# ------------------------------------------------ reproducibility, graphs
def test_concurrent_streams_default_workspaces():
    """Calls in flight on different streams without an explicit workspace get
    one each (a workspace holds the per-call tickets); eight reductions on
    four streams, issued without waiting, match the same calls run one by one."""
    n = (1 << 22) + 5
    xs = [I.normal(n, "f32", seed=30 + k, device=DEV) for k in range(8)]
    want = [_np(tf.sum(x, "rigorous")).copy() for x in xs]
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = []
    torch.cuda.synchronize()
    for k, x in enumerate(xs):
        st = streams[k % 4]
        with torch.cuda.stream(st):
            outs.append(tf.sum(x, "rigorous"))
    torch.cuda.synchronize()
    for o, w in zip(outs, want):
        assert same_bits(_np(o), w)
    wss = set()
    for st in streams:
        with torch.cuda.stream(st):
            wss.add(tf.workspace(0, DEV).data_ptr())
    assert len(wss) == 4


def test_bit_reproducible_runs_streams_and_graph():
    n = (1 << 22) + 7
    x = I.normal(n, "f32", seed=11, device=DEV)
    y = I.normal(n, "f32", seed=11, stream=1, device=DEV)
    ref = _np(tf.dot(x, y, "rigorous"))
    for _ in range(20):
        assert same_bits(_np(tf.dot(x, y, "rigorous")), ref)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ws2 = torch.zeros(tf.workspace_size("dot", False, torch.float32, "rigorous", n),
                          dtype=torch.uint8, device=DEV)
        o2 = tf.dot(x, y, "rigorous", ws=ws2)
    s.synchronize()
    assert same_bits(_np(o2), ref)
    # batched under a CUDA graph, replayed
    off_h = make_csr(2000, 16, 4096, seed=12)
    xs = I.normal(int(off_h[-1]), "f32", seed=13, device=DEV)
    off = torch.from_numpy(off_h).to(DEV)
    ws = torch.zeros(tf.workspace_size("sum", True, torch.float32, "fast", xs.numel(), 2000),
                     dtype=torch.uint8, device=DEV)
    out = torch.empty(2000, 2, device=DEV)
    direct = _np(tf.sum_batched(xs, off, "fast", ws=ws, out=out)).copy()
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gs):
        with torch.cuda.graph(g, stream=gs):
            tf.sum_batched(xs, off, "fast", ws=ws, out=out)
    torch.cuda.synchronize()
    for _ in range(5):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert same_bits(_np(out), direct)


def test_host_buffer_calls_match_device_calls():
    n = 1 << 20
    for dt in ("f32", "f64"):
        x = I.normal(n, dt, seed=14).pin_memory()
        y = I.normal(n, dt, seed=14, stream=1).pin_memory()
        v, e = tf.sum_host(x, "rigorous")
        d = _np(tf.sum(x.to(DEV), "rigorous"))
        assert (v, e) == (d[0], d[1])
        v, e = tf.dot_host(x, y, "fast")
        d = _np(tf.dot(x.to(DEV), y.to(DEV), "fast"))
        assert (v, e) == (d[0], d[1])


def test_host_async_calls_match_device_calls():
    """The asynchronous host-buffer calls, several in flight at once (copies
    on a second stream, or on the compute stream), give the device calls'
    bits once the stream is synchronized."""
    n = (1 << 20) + 3
    cs = torch.cuda.Stream()
    for copy_stream in (cs, None):
        calls = []
        for k, dt in enumerate(("f32", "f64", "f32")):
            x = I.normal(n, dt, seed=50 + k).pin_memory()
            y = I.normal(n, dt, seed=50 + k, stream=1).pin_memory()
            ws = tf.workspace(tf.workspace_size("dot", False, x.dtype, "rigorous", n), DEV)
            xd, yd = torch.empty_like(x, device=DEV), torch.empty_like(y, device=DEV)
            xs = torch.empty_like(x, device=DEV)
            o1 = tf.sum_host_async(x, "rigorous", x_dev=xs, ws=ws, copy_stream=copy_stream)
            o2 = tf.dot_host_async(x, y, "fast", x_dev=xd, y_dev=yd, ws=ws, out_f64=True,
                                   copy_stream=copy_stream)
            calls.append((x, y, o1, o2))
        torch.cuda.synchronize()
        for x, y, o1, o2 in calls:
            d1 = _np(tf.sum(x.to(DEV), "rigorous"))
            d2 = _np(tf.dot(x.to(DEV), y.to(DEV), "fast", out_f64=True))
            assert same_bits(o1.numpy(), d1) and same_bits(o2.numpy(), d2)


@pytest.mark.parametrize("n", [1 << 20, (1 << 22) + 1])
def test_tuner_picks_a_valid_plan_and_stays_exact(n):
    """tf_tune stores its choice in the plan class of n (small or large)."""
    x = I.uniform(n, "f32", seed=15, device=DEV)
    cls = tf.plan_class(n)
    other = tf.PLAN_FLAT if cls == tf.PLAN_FLAT_SMALL else tf.PLAN_FLAT_SMALL
    before = tf.plan_get("sum", cls, torch.float32, "rigorous")
    untouched = tf.plan_get("sum", other, torch.float32, "rigorous")
    try:
        p = tf.tune("sum", "rigorous", x, reps=2)
        assert p == tf.plan_get("sum", cls, torch.float32, "rigorous")
        assert tf.plan_get("sum", other, torch.float32, "rigorous") == untouched
        check_flat("sum", "rigorous", "f32", x, None)
    finally:
        tf.plan_set("sum", cls, torch.float32, "rigorous", before["block"], before["unroll"],
                    before["blocks_per_sm"])


def test_probes_run():
    x = torch.zeros(1 << 24, device=DEV)
    for unroll in (1, 2, 4, 8):
        tf.probe_read(x, unroll=unroll)
        tf.probe_read(x, x, unroll=unroll)
    with pytest.raises(tf.TwofoldError):
        tf.probe_read(x, unroll=3)
    for k in tf.ALU_KINDS:
        tf.probe_alu(k, 100, 152, 256, device=DEV)
    torch.cuda.synchronize()


def test_bounded_barrier_wait_gives_up_and_context_survives():
    """The batched kernel's mbarrier wait on a barrier nothing completes ends
    after its poll limit with a status the host reads; a completed barrier
    passes at once; the context stays usable afterwards."""
    assert tf.probe_wait(False, 2000, device=DEV) is True
    assert tf.probe_wait(True, 2000, device=DEV) is False
    x = I.normal(4099, "f32", seed=9, device=DEV)
    got = _np(tf.sum(x, "rigorous"))
    block, unroll, grid, _ = tf.launch_shape("sum", False, torch.float32, "rigorous", 4099)
    want = O.replay_flat("sum", "rigorous", _np(x), block=block, unroll=unroll, grid=grid)
    assert same_bits(got, want)
