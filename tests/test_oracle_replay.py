"""Pins for the oracle's order replay (CPU only).

The replay is pinned against a second, independent composition of the same
documented order written here in Python: each chain's pair comes from the
paper's sequential loop (Example 1 / Example 3 / the direct and the
double-accumulator loops, or their TwoProduct dot forms) run on the chain's
subsequence, and the tree / butterfly / grid folds are composed from the
oracle's TWO-SUM (Theorem 2).  Special cases then tie the replay to the exact
oracle: integer data, n = 0 and n = 1, sign symmetry, and the error bound of
the rigorous variant with the tree's dependency depth D in place of n - 1.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1401_0248_gb300 import inputs as I

LOOP = {("sum", "plain"): "sum", ("sum", "fast"): "sumtf", ("sum", "rigorous"): "sumt",
        ("sum", "wide"): "sumd", ("dot", "plain"): "dot", ("dot", "fast"): "dottf2",
        ("dot", "rigorous"): "dott2", ("dot", "wide"): "dotd", ("sum", "kahan"): "sumk",
        ("dot", "kahan"): "dotk", ("dot", "fast_literal"): "dottf",
        ("dot", "rigorous_literal"): "dott"}
TWOFOLD = ("fast", "rigorous", "kahan", "fast_literal", "rigorous_literal")


class Arith:
    def __init__(self, f32, twofold):
        self.t = np.float32 if f32 else np.float64
        self.twofold = twofold

    def merge(self, a, b):
        if not self.twofold:
            return (self.t(self.t(a[0]) + self.t(b[0])), self.t(0))
        x, y = O.two_sum(np.array([a[0]], self.t), np.array([b[0]], self.t))
        e = self.t(self.t(self.t(a[1]) + self.t(b[1])) + y[0])
        return (x[0], e)

    def butterfly(self, vals):
        v = list(vals)
        W = len(v)
        o = W // 2
        while o >= 1:
            v = [self.merge(v[i], v[i ^ o]) for i in range(W)]
            o //= 2
        return v[0]

    def tree(self, ch):
        ch = list(ch)
        w = len(ch) // 2
        while w >= 1:
            for c in range(w):
                ch[c] = self.merge(ch[c], ch[c + w])
            w //= 2
        return ch[0]


def chain_pair(op, variant, x, y, idx):
    m = LOOP[(op, variant)]
    if len(idx) == 0:
        return (0.0, 0.0)
    xs = x[idx]
    ys = None if y is None else y[idx]
    v, e = O.loop(m, xs, ys)
    return (v, e)


def out_pair(dt, variant, r, out_f64):
    if dt == np.float64 or out_f64:
        return np.array([r[0], r[1]], dtype=np.float64)
    if variant == "plain":
        return np.array([r[0], r[1]], dtype=np.float32)
    v = np.float32(r[0])
    d = (np.float64(r[0]) - np.float64(v)) + np.float64(r[1])
    return np.array([v, np.float32(d)], dtype=np.float32)


def block_pair(ar, tps, tree):
    """a block's pair from its thread pairs: the tree over the threads, or the
    butterfly of each warp and the butterfly over the warp pairs"""
    if tree:
        return ar.tree(tps)
    wps = [ar.butterfly(tps[w * 32:(w + 1) * 32]) for w in range(len(tps) // 32)]
    return ar.butterfly(wps)


def compose_flat(op, variant, x, y, block, unroll, grid, out_f64=False):
    dt = x.dtype.type
    f32 = dt == np.float32
    V = 4 if f32 else 2
    n = x.size
    nv, tail = n // V, n % V
    P = grid * block
    tw = variant in TWOFOLD
    ab = Arith(f32 and variant != "wide", tw)
    ag = Arith(f32 and variant == "plain", tw)
    tree = (not f32) and tw                    # binary64 twofold: the thread tree
    C = unroll * V
    bps = []
    for b in range(grid):
        tps = []
        for t in range(block):
            g = b * block + t
            lists = [[] for _ in range(C)]
            m = 0
            while g + P * m < nv:
                j = g + P * m
                for l in range(V):
                    lists[(m % unroll) * V + l].append(j * V + l)
                m += 1
            if tail and g == nv % P:
                m = nv // P
                for l in range(tail):
                    lists[(m % unroll) * V + l].append(nv * V + l)
            ch = [chain_pair(op, variant, x, y, np.array(li, dtype=np.int64)) for li in lists]
            tps.append(ab.tree(ch))
        bps.append(block_pair(ab, tps, tree))
    tps = []
    for t in range(block):
        a = (0.0, 0.0)
        if t < grid:
            a = bps[t]
            for i in range(t + block, grid, block):
                a = ag.merge(a, bps[i])
        tps.append(a)
    return out_pair(dt, variant, block_pair(ag, tps, tree), out_f64)


CASES = [
    ("sum", "fast", np.float32, 1000, 32, 1, 2),
    ("sum", "rigorous", np.float32, 4099, 64, 2, 3),
    ("sum", "plain", np.float32, 777, 32, 2, 1),
    ("sum", "wide", np.float32, 1501, 64, 1, 2),
    ("dot", "fast", np.float32, 2003, 32, 2, 2),
    ("dot", "rigorous", np.float64, 1999, 64, 1, 3),
    ("dot", "plain", np.float64, 901, 32, 1, 2),
    ("dot", "wide", np.float32, 1203, 32, 4, 1),
    ("sum", "fast", np.float64, 3001, 32, 4, 5),
    ("sum", "rigorous", np.float64, 2500, 64, 2, 2),
    ("sum", "kahan", np.float32, 2049, 64, 2, 3),
    ("dot", "kahan", np.float64, 1777, 32, 1, 2),
    ("dot", "fast_literal", np.float32, 1500, 32, 2, 2),
    ("dot", "rigorous_literal", np.float64, 1501, 64, 1, 3),
]


@pytest.mark.parametrize("op,variant,dt,n,block,unroll,grid", CASES)
@pytest.mark.parametrize("out_f64", [False, True])
def test_replay_flat_matches_composition(op, variant, dt, n, block, unroll, grid, out_f64):
    s = "f32" if dt == np.float32 else "f64"
    x = I.normal(n, s, seed=n % 4096).numpy()
    y = I.normal(n, s, seed=n % 4096, stream=4).numpy() if op == "dot" else None
    want = compose_flat(op, variant, x, y, block, unroll, grid, out_f64)
    got = O.replay_flat(op, variant, x, y, block=block, unroll=unroll, grid=grid, out_f64=out_f64)
    assert got.dtype == want.dtype
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (got, want)


def test_replay_special_cases():
    for dt in ("f32", "f64"):
        x = I.normal(1, dt, seed=1).numpy()
        for variant in ("plain", "fast", "rigorous"):
            got = O.replay_flat("sum", variant, x, block=256, unroll=4, grid=7)
            assert got[0] == x[0] and got[1] == 0
            got = O.replay_flat("sum", variant, x[:0], block=256, unroll=4, grid=7)
            assert got[0] == 0 and got[1] == 0 and not np.signbit(got[0])
    rng = np.random.default_rng(2)
    xi = rng.integers(-100, 100, size=100003).astype(np.float32)
    S = float(np.sum(xi.astype(np.int64)))
    for variant in ("plain", "fast", "rigorous", "wide"):
        got = O.replay_flat("sum", variant, xi, block=128, unroll=2, grid=9)
        assert float(got[0]) == S and got[1] == 0
    x = I.normal(5001, "f64", seed=3).numpy()
    a = O.replay_flat("sum", "rigorous", x, block=64, unroll=2, grid=4)
    b = O.replay_flat("sum", "rigorous", -x, block=64, unroll=2, grid=4)
    assert a[0] == -b[0] and a[1] == -b[1]


def depth(n, V, block, unroll, grid):
    per_thread = math.ceil(n / (V * grid * block))
    return (per_thread + int(math.log2(unroll * V)) + 5 + int(math.log2(block // 32))
            + math.ceil(math.log2(max(grid, 2))) + 5 + int(math.log2(block // 32)))


@pytest.mark.parametrize("dt,cond", [("f32", 1e4), ("f64", 1e12)])
def test_replay_rigorous_bound_with_tree_depth(dt, cond):
    n = 1 << 17
    ic = I.ill_conditioned(n, dt, cond, seed=21)
    x = ic.x.numpy()
    u = 2.0 ** -24 if dt == "f32" else 2.0 ** -53
    V = 4 if dt == "f32" else 2
    block, unroll, grid = 128, 2, 16
    got = O.replay_flat("sum", "rigorous", x, block=block, unroll=unroll, grid=grid, out_f64=True)
    r = O.exact(x, v=float(got[0]), e=float(got[1]))
    D = depth(n, V, block, unroll, grid)
    g = D * u / (1 - D * u)
    assert abs(r.r) <= u * abs(r.s) + g * g * r.sabs


# ------------------------------------------------------------------- CSR
def compose_csr(op, variant, x, y, off, unroll, tile, out_f64=False):
    dt = x.dtype.type
    f32 = dt == np.float32
    V = 4 if f32 else 2
    tw = variant in TWOFOLD
    ab = Arith(f32 and variant != "wide", tw)
    ag = Arith(f32 and variant == "plain", tw)
    tree = (not f32) and tw                    # binary64 twofold: the thread tree
    C = unroll * V
    outs = []
    for s in range(off.size - 1):
        a, b = int(off[s]), int(off[s + 1])
        if a == b:
            outs.append(out_pair(dt, variant, (0.0, 0.0), out_f64))
            continue
        pcs = []
        for w in range(a // tile, (b - 1) // tile + 1):
            lo, hi = max(a, w * tile), min(b, (w + 1) * tile)
            lists = [[[] for _ in range(C)] for _ in range(32)]
            for i in range(lo, hi):
                r = i - w * tile
                q = r // V
                lists[q % 32][((q // 32) % unroll) * V + r % V].append(i)
            lanes = [ab.tree([chain_pair(op, variant, x, y, np.array(li, dtype=np.int64))
                              for li in lists[l]]) for l in range(32)]
            pcs.append(ab.butterfly(lanes))
        res = piece_merge(ag, pcs, (0.0, 0.0))
        outs.append(out_pair(dt, variant, res, out_f64))
    return np.array(outs)


def piece_merge(ar, pcs, zero):
    """up to 32 pieces: one per lane (zero pairs after them), the butterfly;
    more: the pairwise tree"""
    if len(pcs) == 1:
        return pcs[0]
    if len(pcs) <= 32:
        return ar.butterfly(list(pcs) + [zero] * (32 - len(pcs)))
    return pair_tree(ar, pcs)


def pair_tree(ar, pcs):
    """pieces merged as a complete binary tree over their tile order, written
    top-down: the node over [lo, hi) merges its halves [lo, mid), [mid, hi)
    with mid = lo + the largest power of two below hi - lo"""
    def node(lo, hi):
        if hi - lo == 1:
            return pcs[lo]
        half = 1 << ((hi - lo - 1).bit_length() - 1)
        return ar.merge(node(lo, lo + half), node(lo + half, hi))
    return node(0, len(pcs))


@pytest.mark.parametrize("op,variant,dt,unroll,tile", [
    ("sum", "fast", np.float32, 1, 128), ("sum", "rigorous", np.float64, 2, 128),
    ("dot", "fast", np.float64, 1, 64), ("dot", "rigorous", np.float32, 2, 256),
    ("sum", "plain", np.float32, 1, 128), ("dot", "wide", np.float32, 1, 128),
    ("sum", "kahan", np.float64, 2, 128), ("dot", "rigorous_literal", np.float32, 1, 128),
])
def test_replay_csr_matches_composition(op, variant, dt, unroll, tile):
    s = "f32" if dt == np.float32 else "f64"
    L = I.csr_lengths(24, 1, 700, seed=5)
    L[3] = 0
    L[10] = 0
    off = I.csr_offsets(L)
    n = int(off[-1])
    x = I.normal(n, s, seed=6).numpy()
    y = I.normal(n, s, seed=6, stream=2).numpy() if op == "dot" else None
    want = compose_csr(op, variant, x, y, off, unroll, tile)
    got = O.replay_csr(op, variant, x, off, y, unroll=unroll, tile=tile, nthreads=3)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("op,variant,dt", [("sum", "rigorous", np.float64),
                                           ("dot", "fast", np.float32),
                                           ("sum", "plain", np.float32)])
def test_replay_csr_long_segments_tree(op, variant, dt):
    """segments over more than 32 tiles merge their pieces by the pairwise
    tree (33, 64 and 77 pieces, beside short ones)"""
    tile = 128
    L = [5, 33 * tile - 7, 9, 64 * tile, 77 * tile + 13, 3]
    off = I.csr_offsets(L)
    s = "f32" if dt == np.float32 else "f64"
    x = I.normal(int(off[-1]), s, seed=12).numpy()
    y = I.normal(int(off[-1]), s, seed=12, stream=3).numpy() if op == "dot" else None
    want = compose_csr(op, variant, x, y, off, 1, tile)
    got = O.replay_csr(op, variant, x, off, y, unroll=1, tile=tile, nthreads=2)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def test_replay_csr_segments_independent_and_empty():
    L = I.csr_lengths(50, 1, 5000, seed=7)
    off = I.csr_offsets(L)
    x = I.normal(int(off[-1]), "f32", seed=8).numpy()
    a = O.replay_csr("sum", "rigorous", x, off, unroll=2, tile=1024)
    # insert empty segments everywhere: the non-empty results do not change
    off2 = np.repeat(off, 2)[1:-1]
    off2 = np.concatenate([[0], off2, [off[-1]]])
    b = O.replay_csr("sum", "rigorous", x, off2, unroll=2, tile=1024)
    nonempty = np.diff(off2) > 0
    assert np.array_equal(b[nonempty], a)
    assert np.all(b[~nonempty] == 0)
    # one segment that is the whole vector: the bound holds with tile depth
    ic = I.ill_conditioned(1 << 16, "f64", 1e10, seed=9)
    xx = ic.x.numpy()
    got = O.replay_csr("sum", "rigorous", xx, np.array([0, xx.size]), unroll=2, tile=512)[0]
    r = O.exact(xx, v=float(got[0]), e=float(got[1]))
    u = 2.0 ** -53
    D = 512 // 64 + 2 + 5 + (xx.size // 512) // 32 + 5
    g = D * u / (1 - D * u)
    assert abs(r.r) <= u * abs(r.s) + g * g * r.sabs


# --------------------------------------------- binary128 accumulator ('wide' f64)
def rn113(f):
    """round a Fraction to the nearest binary128 number (ties to even); the
    values here stay far inside binary128's normal range"""
    from fractions import Fraction
    if f == 0:
        return Fraction(0)
    a = abs(f)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scale = Fraction(2) ** (e - 112)
    q, r = divmod(a / scale, 1)
    q = int(q)
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q & 1):
        q += 1
    return (q * scale) if f > 0 else -(q * scale)


class QArith:
    """binary128 accumulation: every add rounds once to 113 bits"""
    def merge(self, a, b):
        return rn113(a + b)

    def butterfly(self, vals):
        return Arith.butterfly(self, vals)

    def tree(self, ch):
        return Arith.tree(self, ch)


def chain_q(x, y, idx):
    from fractions import Fraction
    s = Fraction(0)
    for i in idx:
        t = Fraction(float(x[i])) * (Fraction(float(y[i])) if y is not None else 1)
        s = rn113(s + t)
    return s


def out_q(S):
    from fractions import Fraction
    v = float(S)                       # int/int true division: correctly rounded
    return np.array([v, float(S - Fraction(v))], dtype=np.float64)


def compose_flat_q(x, y, block, unroll, grid):
    """compose_flat's order with binary128 chains and folds"""
    from fractions import Fraction
    V, n, P = 2, x.size, grid * block
    nv, tail = n // V, n % V
    q, C = QArith(), unroll * 2
    bps = []
    for b in range(grid):
        tps = []
        for t in range(block):
            g = b * block + t
            lists = [[] for _ in range(C)]
            m = 0
            while g + P * m < nv:
                for l in range(V):
                    lists[(m % unroll) * V + l].append((g + P * m) * V + l)
                m += 1
            if tail and g == nv % P:
                lists[((nv // P) % unroll) * V].append(nv * V)
            tps.append(q.tree([chain_q(x, y, li) for li in lists]))
        bps.append(block_pair(q, tps, False))
    tps = []
    for t in range(block):
        a = Fraction(0)
        if t < grid:
            a = bps[t]
            for i in range(t + block, grid, block):
                a = q.merge(a, bps[i])
        tps.append(a)
    return out_q(block_pair(q, tps, False))


@pytest.mark.parametrize("op,n,block,unroll,grid", [
    ("sum", 1001, 32, 2, 3), ("dot", 777, 64, 1, 2), ("sum", 2, 32, 4, 1),
    ("dot", 1537, 32, 4, 5)])
@pytest.mark.parametrize("cond", [None, 1e28])
def test_replay_flat_binary128_matches_composition(op, n, block, unroll, grid, cond):
    if cond is not None and n < 3:
        pytest.skip("the ill-conditioned generator needs three elements")
    if cond is None:
        x = I.normal(n, "f64", seed=n + 11).numpy()
        x = x * np.exp2(np.arange(n) % 97 - 48.0)      # wide dynamic range
        y = I.normal(n, "f64", seed=n + 11, stream=5).numpy() if op == "dot" else None
    else:
        # cancellation far beyond 113 bits: the result depends on the order
        ic = I.ill_conditioned(n, "f64", cond, seed=n, dot=op == "dot")
        x, y = ic.x.numpy(), (ic.y.numpy() if op == "dot" else None)
    want = compose_flat_q(x, y, block, unroll, grid)
    got = O.replay_flat(op, "wide", x, y, block=block, unroll=unroll, grid=grid)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (got, want)


def test_replay_binary128_exact_and_bounded():
    """integer data below 2^60 sums exactly in 113 bits; otherwise the pair
    obeys the recursive-summation bound in binary128 plus the output rounding"""
    rng = np.random.default_rng(4)
    xi = rng.integers(-2 ** 52, 2 ** 52, size=50001).astype(np.float64)
    got = O.replay_flat("sum", "wide", xi, block=128, unroll=2, grid=9)
    r = O.exact(xi)
    assert got[0] == r.s and got[1] == r.s_lo
    # 2^60 + 1 - 2^60 is lost by a binary64 sum and kept by binary128
    got = O.replay_flat("sum", "wide", np.array([2.0 ** 60, 1.0, -2.0 ** 60]),
                        block=32, unroll=1, grid=1)
    assert got[0] == 1.0 and got[1] == 0.0
    ic = I.ill_conditioned(1 << 15, "f64", 1e25, seed=5)
    x = ic.x.numpy()
    got = O.replay_flat("sum", "wide", x, block=64, unroll=2, grid=4)
    r = O.exact(x, v=float(got[0]), e=float(got[1]))
    u = 2.0 ** -113
    D = depth(x.size, 2, 64, 2, 4)
    assert abs(r.r) <= 2.0 ** -105 * abs(r.s) + D * u / (1 - D * u) * r.sabs


def test_replay_csr_binary128_matches_composition():
    """compose_csr's tile order with binary128 chains and folds"""
    from fractions import Fraction
    L = I.csr_lengths(12, 3, 400, seed=15)
    L[4] = 0
    L[7] = 40 * 64 + 5                          # a segment over 41 tiles: the tree
    off = I.csr_offsets(L)
    n, unroll, tile = int(off[-1]), 2, 64
    ic = I.ill_conditioned(n, "f64", 1e28, seed=16)
    x = ic.x.numpy()
    q = QArith()
    want = []
    for s in range(off.size - 1):
        a, b = int(off[s]), int(off[s + 1])
        pcs = []
        for w in range(a // tile, (b - 1) // tile + 1) if b > a else []:
            lo, hi = max(a, w * tile), min(b, (w + 1) * tile)
            lists = [[[] for _ in range(unroll * 2)] for _ in range(32)]
            for i in range(lo, hi):
                r = i - w * tile
                lists[(r // 2) % 32][((r // 64) % unroll) * 2 + r % 2].append(i)
            pcs.append(q.butterfly([q.tree([chain_q(x, None, li) for li in lists[l]])
                                    for l in range(32)]))
        res = piece_merge(q, pcs, Fraction(0)) if pcs else Fraction(0)
        want.append(out_q(res))
    got = O.replay_csr("sum", "wide", x, off, unroll=unroll, tile=tile)
    assert np.array_equal(got.view(np.uint8), np.array(want).view(np.uint8))


# ------------------------------------------------------------- rank merge
def test_merge_pairs_pinned_to_two_sum_and_plain_arithmetic():
    """The oracle's rank-order merge of shard pairs, against its definition
    written with the pinned TWO-SUM primitive and numpy's IEEE additions:
    twofold variants (V, q) = TWO-SUM(V, V_g), E = (E + E_g) + q in binary64;
    plain one addition in the data type; the binary32 output rule
    v = RN32(V), e = RN32((V - v) + E); G = 0 and G = 1."""
    rng = np.random.default_rng(70)
    for G in (2, 3, 7):
        pairs = np.stack([rng.standard_normal(G) * 10.0 ** rng.integers(-3, 3, size=G),
                          rng.standard_normal(G) * 1e-17], axis=1)
        V, E = pairs[0]
        for g in range(1, G):
            xs, ys = O.two_sum(np.array([V]), np.array([pairs[g, 0]]))
            E = (E + pairs[g, 1]) + ys[0]
            V = xs[0]
        for variant in ("fast", "rigorous", "kahan", "fast_literal", "rigorous_literal"):
            got = O.merge_pairs(pairs, np.float64, variant)
            assert got[0] == V and got[1] == E, variant
            got64 = O.merge_pairs(pairs, np.float32, variant, out_f64=True)
            assert got64[0] == V and got64[1] == E
            got32 = O.merge_pairs(pairs, np.float32, variant)
            v = np.float32(V)
            assert got32[0] == v and got32[1] == np.float32((V - np.float64(v)) + E)
        p32 = pairs.astype(np.float32).astype(np.float64)
        acc = np.float32(p32[0, 0])
        for g in range(1, G):
            acc = np.float32(acc + np.float32(p32[g, 0]))
        got = O.merge_pairs(p32, np.float32, "plain")
        assert got[0] == acc and got[1] == 0
        acc64 = pairs[0, 0]
        for g in range(1, G):
            acc64 = acc64 + pairs[g, 0]
        assert O.merge_pairs(pairs, np.float64, "plain")[0] == acc64
    z = O.merge_pairs(np.zeros((0, 2)), np.float64, "rigorous")
    assert z[0] == 0 and z[1] == 0 and not np.signbit(z[0])
    one = O.merge_pairs(np.array([[3.0, 1e-20]]), np.float64, "fast")
    assert one[0] == 3.0 and one[1] == 1e-20


def test_merge_pairs_binary128_wide_exact_on_integers():
    """binary64 'wide' pairs merge in binary128: on pairs whose exact sum fits
    113 bits the result is (RN64(S), RN64(S - RN64(S))) of the exact S."""
    from fractions import Fraction
    rng = np.random.default_rng(71)
    for G in (1, 2, 5):
        hi = rng.integers(-2 ** 52, 2 ** 52, size=G).astype(np.float64) * 2.0 ** 40
        lo = rng.integers(-2 ** 30, 2 ** 30, size=G).astype(np.float64)
        S = sum(Fraction(float(a)) + Fraction(float(b)) for a, b in zip(hi, lo))
        got = O.merge_pairs(np.stack([hi, lo], 1), np.float64, "wide")
        assert Fraction(float(got[0])) + Fraction(float(got[1])) == S
        assert got[0] == float(S)


def test_split_reduction_obeys_the_bound():
    """One ill-conditioned vector cut into G contiguous shards, each shard
    replayed in the single-vector launch order (binary64 pair output), the
    pairs merged in rank order: the merged pair meets the twofold bound with
    the shard's depth plus G."""
    import math
    from _helpers import U64, twofold_bound, flat_depth
    n = (1 << 18) + 3
    ic = I.ill_conditioned(n, "f64", 1e14, seed=72)
    x = ic.x.numpy()
    for G in (2, 3, 8):
        m = -(-n // (G * 2)) * 2
        pairs = []
        for g in range(G):
            xs = x[min(g * m, n):min((g + 1) * m, n)]
            pairs.append(O.replay_flat("sum", "rigorous", xs, block=128, unroll=2, grid=7))
        got = O.merge_pairs(np.array(pairs), np.float64, "rigorous")
        r = O.exact(x, v=float(got[0]), e=float(got[1]))
        D = flat_depth(m, 2, 128, 2, 7) + G
        assert abs(r.r) <= twofold_bound(r.s, r.sabs, U64, D)
        assert abs(r.rv) > abs(r.r)
