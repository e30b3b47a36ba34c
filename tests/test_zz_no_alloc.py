"""tf_sum_noalloc: the single-vector twofold sum for callers that cannot
allocate device memory (their scratch lives in a library-owned device array).

Checked through the C ABI against tf_sum, the entry point with a caller
workspace: same kernel and launch shape, so the pairs must be bit-identical,
on several calls in a row that share the array.  This file is collected last
so that a stopped run has already run every other test; it passes alone in a
fresh process and after the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1401_0248_gb300 import inputs as I
from paper_1401_0248_gb300 import twofold as tf

pytestmark = pytest.mark.gpu


def test_sum_noalloc_matches_tf_sum_on_calls_in_a_row():
    assert torch.cuda.is_available(), "GPU test"
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = tf.lib()
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    # (dtype, variant, n, seed, binary64 output pair for binary32 data); the
    # binary64 'wide' case fills two 16-byte slots per block of the array
    cases = [("f32", "rigorous", (1 << 22) + 3, 41, False), ("f64", "fast", (1 << 21) + 1, 42, False),
             ("f32", "rigorous", (1 << 22) + 3, 41, False), ("f32", "plain", 1000, 43, False),
             ("f64", "wide", (1 << 22) + 5, 44, False), ("f64", "kahan", 300007, 45, False),
             ("f32", "fast", (1 << 21) + 7, 46, True), ("f64", "wide", (1 << 22) + 5, 44, False)]
    for dt, variant, n, seed, out_f64 in cases:
        x = I.normal(n, dt, seed=seed, device=dev)
        want = tf.sum(x, variant, out_f64=out_f64).cpu().numpy()
        out = torch.full((2,), float("nan"), dtype=torch.float64 if out_f64 else x.dtype,
                         device=dev)
        rc = L.tf_sum_noalloc(C.c_void_p(x.data_ptr()), n, tf.DTYPES[x.dtype],
                              tf.VARIANTS[variant], C.c_void_p(out.data_ptr()),
                              1 if out_f64 else 0, stream)
        assert rc == 0, tf.status_string(rc)
        got = out.cpu().numpy()
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (dt, variant, got, want)
    # argument errors come back before any launch
    assert L.tf_sum_noalloc(None, -1, 0, 1, C.c_void_p(out.data_ptr()), 0, stream) == 1


def test_sum_noalloc_rejects_grids_beyond_its_array():
    """binary64 'wide' pairs take 32 bytes, so a launch shape of more than
    1024 blocks does not fit the array: TF_ERR_UNSUPPORTED, nothing launched;
    the same call fits again once the plan is restored."""
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = tf.lib()
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    n = 1 << 22
    x = I.normal(n, "f64", seed=47, device=dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    cls = tf.plan_class(n)
    before = tf.plan_get("sum", cls, torch.float64, "wide")
    try:
        tf.plan_set("sum", cls, torch.float64, "wide", 128, 1, 8)
        grid = tf.launch_shape("sum", False, torch.float64, "wide", n)[2]
        assert grid > 1024
        rc = L.tf_sum_noalloc(C.c_void_p(x.data_ptr()), n, tf.DTYPES[x.dtype], tf.VARIANTS["wide"],
                              C.c_void_p(out.data_ptr()), 0, stream)
        assert rc == 8, tf.status_string(rc)                 # TF_ERR_UNSUPPORTED
        assert bool(torch.isnan(out).all())
    finally:
        tf.plan_set("sum", cls, torch.float64, "wide", before["block"], before["unroll"],
                    before["blocks_per_sm"])
    rc = L.tf_sum_noalloc(C.c_void_p(x.data_ptr()), n, tf.DTYPES[x.dtype], tf.VARIANTS["wide"],
                          C.c_void_p(out.data_ptr()), 0, stream)
    assert rc == 0
    want = tf.sum(x, "wide").cpu().numpy()
    assert np.array_equal(out.cpu().numpy().view(np.uint8), want.view(np.uint8))
