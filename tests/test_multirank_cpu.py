"""Multi-rank logic on CPU (no GPU): the benchmark's aggregation over ranks
with a world_size-2 gloo process group, and the shard-and-merge reading of
the method (each rank reduces its own contiguous shard to a pair; the pairs
are all-gathered and merge by TWO-SUM in fixed rank order), with the shard
pairs computed by the oracle and gathered by the benchmark's own gather.

The path shards into independent problems, so bench.py --gpus N runs one
problem per rank with no collective on the data path; the only cross-rank
operations are the timing barrier, the max of the step time and the sum of
the bytes, exercised here.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1401_0248_gb300 import inputs as I
from _helpers import U64, twofold_bound


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), TF_BENCH_BACKEND="gloo")
    import bench
    r, w, _ = bench.dist_setup()
    assert (r, w) == (rank, world)
    step_ms = [12.5, 17.25][rank]
    mx = bench.max_over_ranks(step_ms, w)
    tot = bench.sum_over_ranks(1000.0 * (rank + 1), w)
    bench.barrier(w)
    q.put((rank, mx, tot))
    dist.destroy_process_group()


def test_bench_aggregation_over_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, tot in got:
        assert mx == 17.25          # the slowest rank's step time
        assert tot == 3000.0        # bytes of all ranks


def _split_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), TF_BENCH_BACKEND="gloo")
    import torch
    import bench
    from paper_1401_0248_gb300 import twofold as tf
    r, w, _ = bench.dist_setup()
    out = {}
    for dt, variant in (("f64", "rigorous"), ("f32", "fast"), ("f64", "wide")):
        n = 100003
        x = I.normal(n, dt, seed=60).numpy()
        a, b = tf.shard_bounds(n, w, torch.float32 if dt == "f32" else torch.float64)[r]
        mine = O.replay_flat("sum", variant, x[a:b], block=128, unroll=2, grid=5,
                             out_f64=(dt == "f32")).astype(np.float64)
        allp = bench.gather_pairs(torch.from_numpy(mine), w)
        assert tuple(allp.shape) == (w, 2)
        out[(dt, variant)] = (allp.numpy().copy(),
                              O.merge_pairs(allp.numpy(), np.float32 if dt == "f32" else np.float64,
                                            variant))
    bench.barrier(w)
    q.put((r, out))
    dist.destroy_process_group()


def test_split_gather_and_merge_over_two_gloo_ranks():
    """Each rank's shard pair, gathered with the benchmark's all-gather, lands
    in rank order on both ranks, and both merge to the same pair as one
    process merging the two shard pairs itself."""
    import torch
    from paper_1401_0248_gb300 import twofold as tf
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_split_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    for dt, variant in (("f64", "rigorous"), ("f32", "fast"), ("f64", "wide")):
        n = 100003
        x = I.normal(n, dt, seed=60).numpy()
        td = torch.float32 if dt == "f32" else torch.float64
        want_pairs = np.array([O.replay_flat("sum", variant, x[a:b], block=128, unroll=2, grid=5,
                                             out_f64=(dt == "f32")).astype(np.float64)
                               for a, b in tf.shard_bounds(n, 2, td)])
        want = O.merge_pairs(want_pairs, np.float32 if dt == "f32" else np.float64, variant)
        for r in (0, 1):
            pairs, merged = got[r][(dt, variant)]
            assert np.array_equal(pairs.view(np.uint8), want_pairs.view(np.uint8))
            assert np.array_equal(merged.view(np.uint8), want.view(np.uint8))


def test_shard_bounds():
    import torch
    from paper_1401_0248_gb300 import twofold as tf
    for n in (0, 1, 7, 100003, 1 << 20):
        for G in (1, 2, 3, 8):
            for td, V in ((torch.float32, 4), (torch.float64, 2)):
                sb = tf.shard_bounds(n, G, td)
                assert len(sb) == G and sb[0][0] == 0 and sb[-1][1] == n
                for (a, b), (c, d) in zip(sb, sb[1:]):
                    assert b == c
                for a, b in sb:
                    assert a <= b and (a % V == 0 or a == n)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    args = type("A", (), {"ref_sample": 1024, "steps": 1, "warmup": 3})()
    assert bench.run_reference(args, rank=1, world=2) is None


@pytest.mark.parametrize("shards", [2, 3, 8])
def test_shard_and_merge_emulation(shards):
    """Each shard's pair comes from the paper's rigorous loop (Example 3); the
    shard pairs merge in rank order with TWO-SUM plus one add of the errors.
    The result obeys the twofold bound with depth n/shards + shards + 1."""
    n = 1 << 18
    ic = I.ill_conditioned(n, "f64", 1e12, seed=31)
    x = ic.x.numpy()
    cuts = [n * g // shards for g in range(shards + 1)]
    pairs = [O.loop("sumt", x[cuts[g]:cuts[g + 1]]) for g in range(shards)]
    v, e = pairs[0]
    for v2, e2 in pairs[1:]:
        xs, ys = O.two_sum(np.array([v]), np.array([v2]))
        e = (e + e2) + ys[0]
        v = xs[0]
    r = O.exact(x, v=float(v), e=float(e))
    D = n // shards + shards + 1
    assert abs(r.r) <= twofold_bound(r.s, r.sabs, U64, D)
    # a different sharding changes the bits of the value but not the bound
    assert abs(r.rv) > abs(r.r)


def test_reference_arm_json_line_on_cpu():
    """bench.py --impl reference runs the CPU oracle only and prints one JSON
    line with the contract's keys (here on a tiny sample)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-sample", "4096"], cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3
    assert "workload" in d["config"] and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_bench_refuses_fewer_than_three_warmup_steps():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--warmup", "2"],
                       cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "--warmup must be >= 3" in r.stderr
