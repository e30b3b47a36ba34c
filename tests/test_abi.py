"""The C-ABI library builds, loads and exports every symbol of include/twofold.h
(CPU only: no compute calls, only host-side argument checks)."""
import ctypes as C
import os
import re

import pytest

from paper_1401_0248_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "twofold.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tf_sum", "tf_dot", "tf_sum_batched", "tf_dot_batched", "tf_workspace_size",
                 "tf_status_string", "tf_prim", "tf_tune"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1401_0248_gb300 import twofold
    assert set(declared_functions()) == set(twofold.SIGNATURES)
    twofold.lib()      # binds argtypes for all of them


def test_host_side_checks_without_gpu():
    from paper_1401_0248_gb300 import twofold
    L = twofold.lib()
    assert twofold.status_string(0) == "ok"
    assert twofold.status_string(6) == "invalid CSR offsets"
    assert "in flight" in twofold.status_string(9)
    b = C.c_size_t(0)
    assert L.tf_workspace_size(0, 0, 0, 1, 1 << 20, 0, C.byref(b)) == 0 and b.value > 256
    assert L.tf_workspace_size(0, 1, 0, 1, 1 << 20, 100, C.byref(b)) == 0
    big = b.value
    assert L.tf_workspace_size(0, 1, 0, 1, 1 << 24, 100, C.byref(b)) == 0 and b.value > big
    # argument errors come back before any device work
    assert L.tf_sum(None, -1, 0, 1, C.c_void_p(256), C.c_void_p(256), 1 << 20, 0, None) == 1
    assert L.tf_sum(None, 10, 7, 1, C.c_void_p(256), C.c_void_p(256), 1 << 20, 0, None) == 2  # no such dtype
    assert L.tf_sum(C.c_void_p(2), 10, 0, 1, C.c_void_p(256), C.c_void_p(256), 1 << 20, 0, None) == 4
    assert L.tf_sum(C.c_void_p(256), 10, 0, 1, C.c_void_p(256), C.c_void_p(256), 16, 0, None) == 3
    # host-buffer calls check their arguments before enqueuing any copy
    res = (C.c_double * 2)()
    assert L.tf_sum_host(C.c_void_p(16), 10, 0, 9, C.cast(res, C.c_void_p), C.c_void_p(256),
                         C.c_void_p(256), 1 << 20, 0, None) == 1            # no such variant
    assert L.tf_dot_host(C.c_void_p(16), C.c_void_p(16), 10, 0, 1, C.cast(res, C.c_void_p),
                         C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), 16, 0, None) == 3
    p = twofold.Plan(100, 2, 2, 0)
    assert L.tf_plan_set(0, 0, 0, 1, C.byref(p)) == 1          # block must be 128/256/512
    p = twofold.Plan(256, 2, 4, 1000)
    assert L.tf_plan_set(0, 1, 0, 1, C.byref(p)) == 1          # tile not a multiple of 128
    assert L.tf_device_sm_count() >= 0


def test_plan_save_load_roundtrip(tmp_path):
    from paper_1401_0248_gb300 import twofold
    import torch
    before = twofold.plan_get("dot", True, torch.float64, "rigorous")
    twofold.plan_set("dot", True, torch.float64, "rigorous", 128, 4, 8, 8192)
    path = str(tmp_path / "plans.txt")
    twofold.plan_save(path)
    twofold.plan_set("dot", True, torch.float64, "rigorous", before["block"], before["unroll"],
                     before["blocks_per_sm"], before["tile"])
    twofold.plan_load(path)
    assert twofold.plan_get("dot", True, torch.float64, "rigorous") == \
        {"block": 128, "unroll": 4, "blocks_per_sm": 8, "tile": 8192}
    twofold.plan_set("dot", True, torch.float64, "rigorous", before["block"], before["unroll"],
                     before["blocks_per_sm"], before["tile"])
    with open(path, "a") as f:
        f.write("0 0 0 1 100 1 1 0\n")
    with pytest.raises(twofold.TwofoldError):
        twofold.plan_load(path)
    # the small single-vector class keeps its own plans
    small = twofold.plan_get("sum", twofold.PLAN_FLAT_SMALL, torch.float64, "fast")
    twofold.plan_set("sum", twofold.PLAN_FLAT_SMALL, torch.float64, "fast", 128, 1, 4)
    assert twofold.plan_get("sum", twofold.PLAN_FLAT_SMALL, torch.float64, "fast")["block"] == 128
    path2 = str(tmp_path / "plans2.txt")
    twofold.plan_save(path2)
    assert any(line.startswith("0 2 1 1 128 1 4 0") for line in open(path2))
    twofold.plan_set("sum", twofold.PLAN_FLAT_SMALL, torch.float64, "fast", small["block"],
                     small["unroll"], small["blocks_per_sm"])
    assert twofold.plan_class(1 << 22) == 2 and twofold.plan_class((1 << 22) + 1) == 0
    assert twofold.plan_class(5, batched=True) == 1


def test_bad_default_plan_file_raises(tmp_path):
    """A plan file named by TF_PLANS that does not parse makes the first use
    of the library raise TwofoldError (checked in a fresh interpreter)."""
    import subprocess
    import sys
    bad = tmp_path / "bad_plans.txt"
    bad.write_text("0 0 0 1 100 1 1 0\n")
    code = ("from paper_1401_0248_gb300 import twofold as t\n"
            "try:\n    t.lib()\nexcept t.TwofoldError as e:\n    print('raised', e.code)\n")
    env = dict(os.environ, TF_PLANS=str(bad))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "raised 1" in r.stdout


def test_product_path_has_no_cpu_fallback():
    """The binding raises on CPU tensors instead of computing anything."""
    import torch
    from paper_1401_0248_gb300 import twofold
    with pytest.raises(ValueError):
        twofold.sum(torch.zeros(10))
    src = open(os.path.join(ROOT, "paper_1401_0248_gb300", "twofold.py")).read()
    assert "oracle" not in src.replace("oracle is", "")


def test_build_rebuilds_on_every_header():
    """Every header of csrc/ and include/ (the batched kernels' tf_csr.cuh and
    tf_async.cuh included) is a dependency of every object, so an edit to any
    of them rebuilds the library."""
    csrc = os.path.join(ROOT, "paper_1401_0248_gb300", "csrc")
    deps = set(os.path.basename(h) for h in libbuild._headers())
    for f in os.listdir(csrc):
        if f.endswith((".cuh", ".h")):
            assert f in deps, f
    assert {"tf_csr.cuh", "tf_async.cuh", "twofold.h"} <= deps
