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
    cases = [("f32", "rigorous", (1 << 22) + 3, 41), ("f64", "fast", (1 << 21) + 1, 42),
             ("f32", "rigorous", (1 << 22) + 3, 41), ("f32", "plain", 1000, 43)]
    for dt, variant, n, seed in cases:
        x = I.normal(n, dt, seed=seed, device=dev)
        want = tf.sum(x, variant).cpu().numpy()
        out = torch.full((2,), float("nan"), dtype=x.dtype, device=dev)
        rc = L.tf_sum_noalloc(C.c_void_p(x.data_ptr()), n, tf.DTYPES[x.dtype],
                              tf.VARIANTS[variant], C.c_void_p(out.data_ptr()), 0, stream)
        assert rc == 0, tf.status_string(rc)
        got = out.cpu().numpy()
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (dt, variant, got, want)
    # argument errors come back before any launch
    assert L.tf_sum_noalloc(None, -1, 0, 1, C.c_void_p(out.data_ptr()), 0, stream) == 1
