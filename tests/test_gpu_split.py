"""One vector split into contiguous shards on one GPU, the shard pairs merged
in rank order by tf_merge_pairs: bit for bit against the oracle's replay of
each shard's launch order and its rank-order merge, for every variant, sums
and dots, binary32 and binary64; the merged twofold result meets the bound
against the exact oracle.  (Several GPUs exchange only these pairs; the
gather itself is tested with gloo ranks on the CPU.)"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_0248_gb300 import inputs as I
from paper_1401_0248_gb300 import twofold as tf
from _helpers import U32, U64, flat_depth, same_bits, twofold_bound

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TD = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(DEV)
    assert tf.sm_count() > 0


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("op,variant", [("sum", "plain"), ("sum", "fast"), ("sum", "rigorous"),
                                        ("sum", "wide"), ("sum", "kahan"), ("dot", "fast"),
                                        ("dot", "rigorous"), ("dot", "wide")])
@pytest.mark.parametrize("G", [1, 2, 3, 8])
def test_split_merge_bit_exact(dt, op, variant, G):
    n = (1 << 20) + 11
    ic = I.ill_conditioned(n, dt, 1e10, seed=80 + G, device=DEV, dot=(op == "dot"))
    x, y = ic.x, ic.y
    pairs = torch.empty(G, 2, dtype=torch.float64, device=DEV)
    want_pairs = []
    xh, yh = _np(x), (_np(y) if y is not None else None)
    depth = 0
    for g, (a, b) in enumerate(tf.shard_bounds(n, G, TD[dt])):
        if op == "sum":
            tf.sum(x[a:b], variant, out_f64=True, out=pairs[g])
        else:
            tf.dot(x[a:b], y[a:b], variant, out_f64=True, out=pairs[g])
        block, unroll, grid, _ = tf.launch_shape(op, False, TD[dt], variant, b - a)
        w = O.replay_flat(op, variant, xh[a:b], yh[a:b] if yh is not None else None,
                          block=block, unroll=unroll, grid=grid, out_f64=True)
        want_pairs.append(w.astype(np.float64))
        depth = max(depth, flat_depth(max(b - a, 1), 4 if dt == "f32" else 2, block, unroll, grid))
    want_pairs = np.array(want_pairs)
    assert same_bits(_np(pairs), want_pairs), "shard pairs"
    for out_f64 in ((False, True) if dt == "f32" else (False,)):
        got = _np(tf.merge_pairs(pairs, TD[dt], variant, out_f64=out_f64))
        want = O.merge_pairs(want_pairs, np.float32 if dt == "f32" else np.float64, variant,
                             out_f64=out_f64)
        assert same_bits(got, want), (dt, op, variant, G, out_f64, got, want)
    if variant == "rigorous":
        got = _np(tf.merge_pairs(pairs, TD[dt], variant, out_f64=True))
        err = abs(ic.S - Fraction(float(got[0])) - Fraction(float(got[1])))
        u = U32 if dt == "f32" else U64
        assert float(err) <= twofold_bound(float(ic.S), ic.sum_abs, u, depth + G)


def test_split_into_one_shard_is_the_unsplit_call():
    """G = 1: the merge only converts the one binary64 pair, giving the bits
    of the same call without the split."""
    n = 300007
    for dt in ("f32", "f64"):
        x = I.normal(n, dt, seed=90, device=DEV)
        for variant in ("fast", "rigorous", "plain", "wide", "kahan"):
            p = tf.sum(x, variant, out_f64=True).reshape(1, 2)
            assert same_bits(_np(tf.merge_pairs(p, TD[dt], variant)), _np(tf.sum(x, variant)))


def test_merge_pairs_arguments_and_empty():
    z = torch.zeros(0, 2, dtype=torch.float64, device=DEV)
    got = _np(tf.merge_pairs(z, torch.float64, "rigorous"))
    assert got[0] == 0 and got[1] == 0 and not np.signbit(got[0])
    with pytest.raises(ValueError):
        tf.merge_pairs(torch.zeros(3, 2, dtype=torch.float32, device=DEV), torch.float32, "fast")
    import ctypes as C
    L = tf.lib()
    p = torch.zeros(2, 2, dtype=torch.float64, device=DEV)
    o = torch.zeros(2, dtype=torch.float64, device=DEV)
    assert L.tf_merge_pairs(C.c_void_p(p.data_ptr()), -1, 1, 1, C.c_void_p(o.data_ptr()), 0, None) == 1
    assert L.tf_merge_pairs(C.c_void_p(p.data_ptr() + 4), 2, 1, 1, C.c_void_p(o.data_ptr()), 0,
                            None) == 4
    assert L.tf_merge_pairs(C.c_void_p(p.data_ptr()), 2, 5, 1, C.c_void_p(o.data_ptr()), 0, None) == 2
