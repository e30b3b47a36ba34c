"""GPU parity at the benchmark's full sizes, in the launch configurations
bench.py times (the committed GB300 plans).

C1  binary64 sum and TwoProduct dot, N = 2^20, uniform [-1, 1): bit-exact
    against the oracle's replay, rigorous within the bound of the exact sum.
C2  binary32/binary64 twofold sum and dot, N = 2^28, ill-conditioned data
    (cond 1e4, 1e8, 1e16): every (dtype, op, variant, cond) against the
    exactly known sum (bound for rigorous, value + error better than value);
    a sample of them bit-exact against the replay.
C3  binary32 twofold dot, N = 2^30, N(0,1) and signed log-normal(0, 2): bound
    against the exact oracle, beside the binary64-accumulated and plain dots.
C4  16,384 ragged binary32 segments (log-uniform 16 .. 2^18 elements, ~4.4e8
    total), twofold sum and dot in one launch under a CUDA graph: every
    segment bit-exact against the replay.
C5  binary64 twofold dot, N = 2^29, cond 1e8 .. 1e30: rigorous within the
    bound of the known exact dot, the error term tracking value - exact, and
    20 runs bit-identical.
C6  the largest sizes: N = 2^31 + 1234567 elements (past 32-bit indexing),
    flat and batched (segments straddling element 2^31), binary32 and
    binary64, on data in {-1, 0, +1} whose partial sums stay far below 2^24,
    so every order gives the exact integer sum and error +0.
"""
import math
import os
from fractions import Fraction

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
PLANS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_1401_0248_gb300", "plans_gb300.txt")


@pytest.fixture(scope="module", autouse=True)
def _gpu_and_plans():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(DEV)
    if os.path.exists(PLANS):
        tf.plan_load(PLANS)
    yield
    torch.cuda.empty_cache()


def _np(t):
    return t.detach().cpu().numpy()


def run(op, variant, x, y=None, out_f64=False):
    out = tf.sum(x, variant, out_f64=out_f64) if op == "sum" else tf.dot(x, y, variant, out_f64=out_f64)
    return _np(out)


def replay(op, variant, dt, xh, yh, out_f64=False):
    block, unroll, grid, _ = tf.launch_shape(op, False, TD[dt], variant, xh.size)
    return O.replay_flat(op, variant, xh, yh, block=block, unroll=unroll, grid=grid,
                         out_f64=out_f64), (block, unroll, grid)


def test_c1_f64_n2p20_bit_exact_and_bound():
    n = 1 << 20
    x = I.uniform(n, "f64", seed=0, stream=0, device=DEV)
    y = I.uniform(n, "f64", seed=0, stream=1, device=DEV)
    xh, yh = _np(x), _np(y)
    for op in ("sum", "dot"):
        for variant in ("fast", "rigorous", "plain"):
            got = run(op, variant, x, y if op == "dot" else None)
            want, shape = replay(op, variant, "f64", xh, yh if op == "dot" else None)
            assert same_bits(got, want), (op, variant)
            if variant == "rigorous":
                ex = O.exact(xh, yh if op == "dot" else None, v=float(got[0]), e=float(got[1]))
                D = flat_depth(n, 2, *shape)
                assert abs(ex.r) <= twofold_bound(ex.s, ex.sabs, U64, D)


def rel(S, v, e=0.0):
    return float(abs(S - Fraction(float(v)) - Fraction(float(e))) / abs(S))


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_c2_n2p28_ill_conditioned(dt):
    n = 1 << 28
    u = U32 if dt == "f32" else U64
    V = 4 if dt == "f32" else 2
    for cond in (1e4, 1e8, 1e16):
        s = I.ill_conditioned(n, dt, cond, seed=0, device=DEV)
        d = I.ill_conditioned(n, dt, cond, seed=1, device=DEV, dot=True)
        for op, ic in (("sum", s), ("dot", d)):
            plain = run(op, "plain", ic.x, ic.y)
            for variant in ("fast", "rigorous"):
                got = run(op, variant, ic.x, ic.y, out_f64=(dt == "f32"))
                block, unroll, grid, _ = tf.launch_shape(op, False, TD[dt], variant, n)
                D = flat_depth(n, V, block, unroll, grid)
                err = float(abs(ic.S - Fraction(float(got[0])) - Fraction(float(got[1]))))
                if variant == "rigorous":
                    bound = twofold_bound(float(ic.S), ic.sum_abs, u, D)
                    assert err <= bound, (dt, op, cond)
                    # value + error improves on the value alone (up to the bound)
                    assert rel(ic.S, got[0], got[1]) <= rel(ic.S, got[0]) + bound / float(ic.S)
                    if cond <= 1e8:
                        assert rel(ic.S, got[0], got[1]) <= rel(ic.S, plain[0])
        del s, d
        torch.cuda.empty_cache()
    # a sample bit-exact against the replay at full size
    ic = I.ill_conditioned(n, dt, 1e8, seed=0, device=DEV)
    got = run("sum", "fast", ic.x)
    want, _ = replay("sum", "fast", dt, _np(ic.x), None)
    assert same_bits(got, want)
    icd = I.ill_conditioned(n, dt, 1e8, seed=1, device=DEV, dot=True)
    got = run("dot", "rigorous", icd.x, icd.y)
    want, _ = replay("dot", "rigorous", dt, _np(icd.x), _np(icd.y))
    assert same_bits(got, want)


@pytest.mark.parametrize("dist", ["normal", "lognormal"])
def test_c3_f32_dot_n2p30_precision_form(dist):
    n = 1 << 30
    if dist == "normal":
        x = I.normal(n, "f32", seed=0, stream=0, device=DEV)
        y = I.normal(n, "f32", seed=0, stream=10, device=DEV)
    else:
        x = I.signed_lognormal(n, "f32", 2.0, seed=0, stream=0, device=DEV)
        y = I.signed_lognormal(n, "f32", 2.0, seed=0, stream=10, device=DEV)
    tw = run("dot", "rigorous", x, y, out_f64=True)
    fa = run("dot", "fast", x, y, out_f64=True)
    wide = run("dot", "wide", x, y, out_f64=True)
    plain = run("dot", "plain", x, y)
    xh, yh = _np(x), _np(y)
    del x, y
    torch.cuda.empty_cache()
    ex = O.exact(xh, yh, v=float(tw[0]), e=float(tw[1]))
    block, unroll, grid, _ = tf.launch_shape("dot", False, torch.float32, "rigorous", n)
    D = flat_depth(n, 4, block, unroll, grid)
    assert abs(ex.r) <= twofold_bound(ex.s, ex.sabs, U32, D)
    S = Fraction(ex.s) + Fraction(ex.s_lo)
    rt = rel(S, tw[0], tw[1])
    # reported with -s: relative errors of each form against the exact dot
    print("\nC3 %s: cond %.3g  rigorous v+e %.3g  v %.3g  fast v+e %.3g  wide %.3g  plain %.3g"
          % (dist, ex.sabs / abs(ex.s), rt, rel(S, tw[0]), rel(S, fa[0], fa[1]), rel(S, wide[0]),
             rel(S, plain[0])))
    # FP32-arithmetic twofold against binary64 accumulation and plain binary32
    assert rt <= rel(S, plain[0])
    assert rel(S, fa[0], fa[1]) <= rel(S, plain[0])
    assert rel(S, wide[0]) < 1e-6


def test_c4_batched_16384_segments_graph_bit_exact():
    L = I.csr_lengths(16384, 16, 1 << 18, seed=0)
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    assert 3.5e8 < n < 5.5e8
    x = I.uniform(n, "f32", seed=1, device=DEV)
    y = I.uniform(n, "f32", seed=1, stream=1, device=DEV)
    off = torch.from_numpy(off_h).to(DEV)
    for op, variant in (("sum", "fast"), ("dot", "rigorous"), ("sum", "rigorous"), ("dot", "fast")):
        ws = torch.zeros(tf.workspace_size(op, True, torch.float32, variant, n, 16384),
                         dtype=torch.uint8, device=DEV)
        out = torch.empty(16384, 2, device=DEV)
        call = (lambda: tf.sum_batched(x, off, variant, ws=ws, out=out)) if op == "sum" else \
               (lambda: tf.dot_batched(x, y, off, variant, ws=ws, out=out))
        call()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gs):
            with torch.cuda.graph(g, stream=gs):
                call()
        torch.cuda.synchronize()
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = _np(out)
        _, unroll, _, tile = tf.launch_shape(op, True, torch.float32, variant, n)
        want = O.replay_csr(op, variant, _np(x), off_h, _np(y) if op == "dot" else None,
                            unroll=unroll, tile=tile)
        assert same_bits(got, want), (op, variant)
        if op == "dot" and variant == "rigorous":
            ex = O.exact_batched(_np(x), off_h, _np(y), v=got[:, 0].astype(np.float64),
                                 e=got[:, 1].astype(np.float64))
            for s in range(0, 16384, 97):
                D = csr_depth(int(L[s]), 4, unroll, tile)
                assert abs(ex[s]["r"]) <= twofold_bound(ex[s]["s"], ex[s]["sabs"], U32, D)


def test_c5_f64_dot_n2p29_cond_sweep_tracking_and_reproducible():
    n = 1 << 29
    for cond in (1e8, 1e16, 1e24, 1e30):
        ic = I.ill_conditioned(n, "f64", cond, seed=5, device=DEV, dot=True)
        block, unroll, grid, _ = tf.launch_shape("dot", False, torch.float64, "rigorous", n)
        D = flat_depth(n, 2, block, unroll, grid)
        rig = run("dot", "rigorous", ic.x, ic.y)
        fast = run("dot", "fast", ic.x, ic.y)
        S = ic.S
        err = float(abs(S - Fraction(float(rig[0])) - Fraction(float(rig[1]))))
        assert err <= twofold_bound(float(S), ic.sum_abs, U64, D), cond
        # the error term estimates value - exact while gamma_D^2 * cond << 1
        rv = S - Fraction(float(rig[0]))
        rvf = S - Fraction(float(fast[0]))
        print("\nC5 cond %.0e: rigorous |v+e-S|/|S| %.3g, |v-S|/|S| %.3g, e/(S-v) %s; "
              "fast |v+e-S|/|S| %.3g, e/(S-v) %s"
              % (cond, err / abs(float(S)), abs(float(rv)) / abs(float(S)),
                 "%.6f" % float(Fraction(float(rig[1])) / rv) if rv != 0 else "v exact",
                 float(abs(S - Fraction(float(fast[0])) - Fraction(float(fast[1])))) / abs(float(S)),
                 "%.6f" % float(Fraction(float(fast[1])) / rvf) if rvf != 0 else "v exact"))
        if rv != 0 and (D * U64) ** 2 * cond < 0.1:
            rho = float(Fraction(float(rig[1])) / rv)
            assert 0.5 <= rho <= 2.0, (cond, rho)
        if cond == 1e16:
            for _ in range(20):
                assert same_bits(run("dot", "rigorous", ic.x, ic.y), rig)
                assert same_bits(run("dot", "fast", ic.x, ic.y), fast)
        del ic
        torch.cuda.empty_cache()


def test_c6_beyond_2p31_elements_exact_integer_sums():
    n = (1 << 31) + 1234567
    x8 = I.ternary_i8(n, seed=3, stream=0, device=DEV)
    y8 = I.ternary_i8(n, seed=3, stream=1, device=DEV)
    hx, hy = _np(x8), _np(y8)
    off_h = np.array([0, (1 << 30) + 3, (1 << 31) - 5, (1 << 31) + 77, n, n], dtype=np.int64)
    nseg = off_h.size - 1
    S = [int(np.sum(hx[off_h[k]:off_h[k + 1]], dtype=np.int64)) for k in range(nseg)]
    D = [0] * nseg
    for k in range(nseg):
        for a in range(off_h[k], off_h[k + 1], 1 << 26):
            b = min(off_h[k + 1], a + (1 << 26))
            D[k] += int(np.sum(hx[a:b].astype(np.int16) * hy[a:b], dtype=np.int64))
    assert max(abs(v) for v in S + D) < 1 << 20
    off = torch.from_numpy(off_h).to(DEV)
    for dt in ("f32", "f64"):
        x, y = x8.to(TD[dt]), y8.to(TD[dt])
        for variant in ("fast", "rigorous", "plain"):
            got = run("sum", variant, x)
            assert got[0] == sum(S) and got[1] == 0, (dt, variant, got, sum(S))
        got = run("dot", "rigorous", x, y)
        assert got[0] == sum(D) and got[1] == 0, (dt, got, sum(D))
        for op, want in (("sum", S), ("dot", D)):
            out = _np(tf.sum_batched(x, off, "rigorous") if op == "sum"
                      else tf.dot_batched(x, y, off, "rigorous"))
            assert [float(v) for v in out[:, 0]] == [float(v) for v in want], (dt, op)
            assert not out[:, 1].any()
        del x, y
        torch.cuda.empty_cache()
