"""GPU parity on data over the whole exponent range, inside the reductions.

The binary64 kernels compute the exact errors of their additions and
products from the integer significands and hand zeros, subnormals, operands
below 2^-969 or at 2^1022 and above, and products outside the normal range to
out-of-line binary64 forms (Theorems 1 and 2, and TwoProduct, written with
the hardware's rounded operations).  binary32 products of tiny operands
underflow, where TwoProduct is no longer error-free.  Here every variant
(plain, fast, rigorous, wide, Kahan and the literal dots), flat and batched,
binary32 and binary64, runs on vectors that mix such items with ordinary ones
and on vectors made of tiny items alone, so that chains pass in and out of
those forms; each result must equal the oracle's replay of the launch order
bit for bit.  Rigorous sums also meet the bound against the exact oracle.
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
# (op, variant, literal product)
CASES = [("sum", "plain", False), ("sum", "fast", False), ("sum", "rigorous", False),
         ("sum", "wide", False), ("sum", "kahan", False), ("dot", "plain", False),
         ("dot", "fast", False), ("dot", "rigorous", False), ("dot", "wide", False),
         ("dot", "kahan", False), ("dot", "fast", True), ("dot", "rigorous", True)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(DEV)
    assert tf.sm_count() > 0, "libtwofold.so does not see an sm_103a device"


def _signed(rng, m, lo_exp, hi_exp, dtype):
    """m values (1 + U[0,1)) * 2^k, k uniform in [lo_exp, hi_exp], random signs,
    rounded once to dtype (gradual underflow below the normal range)."""
    v = np.ldexp(rng.random(m) + 1.0, rng.integers(lo_exp, hi_exp + 1, size=m))
    return (v * rng.choice([-1.0, 1.0], size=m)).astype(dtype)


def mixed_vector(n, dt, seed, for_dot=False):
    """Ordinary N(0,1)-like items mixed with zeros of both signs, subnormals,
    tiny normals below 2^-969 (binary64) and, for sums, two huge items at
    2^1022 .. 1.4*2^1022 and their exact negatives (every partial sum stays
    finite and the exact sum is that of the other items);
    binary32 data mix subnormals and tiny normals the same way."""
    rng = np.random.default_rng(seed)
    dtype = np.float32 if dt == "f32" else np.float64
    x = rng.standard_normal(n).astype(dtype)
    idx = rng.permutation(n)
    k = n // 10
    if dt == "f64":
        x[idx[:k]] = _signed(rng, k, -1074, -1023, dtype)              # subnormals
        x[idx[k:2 * k]] = _signed(rng, k, -1022, -970, dtype)          # normals below 2^-969
        x[idx[2 * k:2 * k + k // 4]] = 0.0
        x[idx[2 * k + k // 4:2 * k + k // 2]] = -0.0
        if not for_dot:
            h = np.ldexp(1.0 + 0.4 * rng.random(2), 1022)
            h = np.array([h[0], -h[0], h[1], -h[1]])
            x[idx[3 * k:3 * k + 4]] = h
    else:
        x[idx[:k]] = _signed(rng, k, -149, -127, dtype)                # subnormals
        x[idx[k:2 * k]] = _signed(rng, k, -126, -100, dtype)           # tiny normals
        x[idx[2 * k:2 * k + k // 4]] = 0.0
        x[idx[2 * k + k // 4:2 * k + k // 2]] = -0.0
    return x


def dot_partner(x, dt, seed):
    """y for a dot with x: many products underflow (operands around the square
    root of the least normal), some are subnormal outright, some leave the
    range of the integer TwoProduct at the top (binary64: two products near
    2^1022 that cancel), the rest ordinary."""
    rng = np.random.default_rng(seed)
    n = x.size
    dtype = x.dtype
    y = rng.standard_normal(n).astype(dtype)
    idx = rng.permutation(n)
    k = n // 8
    if dt == "f64":
        y[idx[:k]] = _signed(rng, k, -560, -500, dtype)        # times ~2^-540 x: underflow
        x[idx[:k]] = _signed(rng, k, -560, -500, dtype)
        y[idx[k:2 * k]] = _signed(rng, k, -1074, -1023, dtype)
        # two products of about 1.5 * 2^1022 that cancel exactly, above the
        # integer TwoProduct's range; every partial sum stays finite
        j = idx[2 * k:2 * k + 2]
        x[j] = np.ldexp(np.array([1.5, -1.5]), 512)
        y[j] = np.ldexp(1.0 + 0.25 * rng.random(), 510)
    else:
        y[idx[:k]] = _signed(rng, k, -75, -60, dtype)          # products ~2^-140: subnormal
        x[idx[:k]] = _signed(rng, k, -75, -60, dtype)
        y[idx[k:2 * k]] = _signed(rng, k, -149, -127, dtype)
    return y


def tiny_vector(n, dt, seed):
    """Tiny items only, so that every chain state stays below 2^-969
    (binary64) or in the binary32 subnormal range."""
    rng = np.random.default_rng(seed)
    if dt == "f64":
        return _signed(rng, n, -1074, -990, np.float64)
    return _signed(rng, n, -149, -120, np.float32)


def _np(t):
    return t.detach().cpu().numpy()


def _oracle_variant(variant, literal):
    return variant + "_literal" if literal else variant


def run_flat_case(op, variant, literal, dt, xh, yh, out_f64=False):
    x = torch.from_numpy(xh).to(DEV)
    y = torch.from_numpy(yh).to(DEV) if op == "dot" else None
    if op == "sum":
        got = _np(tf.sum(x, variant, out_f64=out_f64))
    else:
        got = _np(tf.dot(x, y, variant, out_f64=out_f64, literal=literal))
    block, unroll, grid, _ = tf.launch_shape(op, False, TD[dt], variant, xh.size)
    want = O.replay_flat(op, _oracle_variant(variant, literal), xh, yh if op == "dot" else None,
                         block=block, unroll=unroll, grid=grid, out_f64=out_f64)
    assert same_bits(got, want), (op, variant, literal, dt, xh.size, got, want)
    return got, (block, unroll, grid)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("n", [4099, (1 << 20) + 5])
@pytest.mark.parametrize("op,variant,literal", CASES)
def test_flat_mixed_range_bit_exact(dt, n, op, variant, literal):
    xh = mixed_vector(n, dt, seed=100 + n % 97, for_dot=(op == "dot"))
    yh = dot_partner(xh, dt, seed=200 + n % 89) if op == "dot" else None
    got, (block, unroll, grid) = run_flat_case(op, variant, literal, dt, xh, yh)
    if dt == "f32" and variant not in ("plain",):
        run_flat_case(op, variant, literal, dt, xh, yh, out_f64=True)
    if op == "sum" and variant == "rigorous":
        ex = O.exact(xh, v=float(got[0]), e=float(got[1]))
        u = U32 if dt == "f32" else U64
        D = flat_depth(n, 4 if dt == "f32" else 2, block, unroll, grid)
        assert abs(ex.r) <= twofold_bound(ex.s, ex.sabs, u, D)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("op,variant,literal", CASES)
def test_flat_tiny_only_bit_exact(dt, op, variant, literal):
    n = 300007
    xh = tiny_vector(n, dt, seed=300)
    yh = (np.where(np.random.default_rng(301).random(n) < 0.5, 1.0, -1.0).astype(xh.dtype)
          if op == "dot" else None)
    got, (block, unroll, grid) = run_flat_case(op, variant, literal, dt, xh, yh)
    if variant == "rigorous":
        ex = O.exact(xh, yh, v=float(got[0]), e=float(got[1]))
        # sums and dots by +-1 of tiny items: every transform stays error-free
        u = U32 if dt == "f32" else U64
        D = flat_depth(n, 4 if dt == "f32" else 2, block, unroll, grid)
        assert abs(ex.r) <= twofold_bound(ex.s, ex.sabs, u, D)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_csr_mixed_range_bit_exact(dt):
    L = I.csr_lengths(400, 1, 30000, seed=50)
    L[3] = 0
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    xs = mixed_vector(n, dt, seed=51)
    xd = mixed_vector(n, dt, seed=52, for_dot=True)
    yd = dot_partner(xd, dt, seed=53)
    # one segment of tiny items only
    a, b = int(off_h[10]), int(off_h[11])
    xs[a:b] = tiny_vector(b - a, dt, seed=54)
    xd[a:b] = tiny_vector(b - a, dt, seed=55)
    off = torch.from_numpy(off_h).to(DEV)
    for op, variant, literal in CASES:
        xh, yh = (xs, None) if op == "sum" else (xd, yd)
        x = torch.from_numpy(xh).to(DEV)
        if op == "sum":
            got = _np(tf.sum_batched(x, off, variant))
        else:
            got = _np(tf.dot_batched(x, torch.from_numpy(yh).to(DEV), off, variant, literal=literal))
        _, unroll, _, tile = tf.launch_shape(op, True, TD[dt], variant, n)
        want = O.replay_csr(op, _oracle_variant(variant, literal), xh, off_h, yh, unroll=unroll,
                            tile=tile)
        assert same_bits(got, want), (dt, op, variant, literal)
        if op == "sum" and variant == "rigorous":
            ex = O.exact_batched(xh, off_h, v=got[:, 0].astype(np.float64),
                                 e=got[:, 1].astype(np.float64))
            u = U32 if dt == "f32" else U64
            for s in range(len(L)):
                D = csr_depth(max(int(L[s]), 1), 4 if dt == "f32" else 2, unroll, tile)
                assert abs(ex[s]["r"]) <= twofold_bound(ex[s]["s"], ex[s]["sabs"], u, D), s
