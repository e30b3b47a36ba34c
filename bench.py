"""Benchmark: twofold sum / dot on GB300 -- GB/s and relative error vs exact.

Workload (the benchmark's headline configuration): single vectors of
N = 2^28 elements, binary32 and binary64, twofold sum and dot with the fast
(Dekker) and rigorous (Knuth) variants, on ill-conditioned data with target
condition numbers 1e4, 1e8 and 1e16 (half the entries with exponents spread
over 0..E, the rest cancelling them, seeded synthetic data).  One step is one
pass of all 24 twofold reductions (2 dtypes x 2 ops x 2 variants x 3
condition numbers).  Plain binary32/binary64 sums and dots and the wider
accumulators ('wide': binary32 data in binary64, binary64 data in binary128)
run alongside on the same data and are reported per kernel, not in the step.

value    whole-step algorithmic bytes / device time (CUDA events, inputs
         resident in HBM, every input larger than L2).
e2e      the same step through the C ABI's asynchronous host-buffer calls:
         pinned host inputs copied to the device inside the timed region (on
         a copy stream, each reduction ordered behind its copy), the result
         pairs copied back, one host wait per step.
roofline the kernel with the largest share of the step time: its algorithmic
         bytes per launch / its CUDA-event time against the measured HBM copy
         bandwidth; for binary64 kernels, which the binary64 pipe limits,
         also ("alu") its issued binary64 adds against that pipe's measured
         rate.
c3, c5   the two large dot configurations beside the step: binary32 dots of
         N = 2^30 (N(0,1) and signed log-normal(0, 2) data) and binary64 dots
         of N = 2^29 (condition numbers 1e8 .. 1e30), each variant timed, with
         relative errors against the exact dot and the error term's tracking
         of the value's own error; C5 also checks 20 repeated runs for
         identical bits.
cpu_baseline  the CPU oracle's sequential loops (the paper's twofold loops)
         timed on a bounded sample of the same workload on one host core.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--split]
Under torchrun (N > 1) each rank reduces its own copy of the workload (the
path shards into independent problems, no collective on the data path); the
step time is the maximum over ranks and value counts all ranks' bytes.
--split instead cuts every vector into N contiguous shards, one per rank,
gathers the N shard pairs and merges them in rank order on each rank
(strong scaling; one 16-byte all-gather per reduction).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GB/s & rel. error vs exact: twofold vs plain sum/dot, same GB300"
CONDS = (1e4, 1e8, 1e16)
OPS = ("sum", "dot")
TWOFOLD = ("fast", "rigorous")
N_DEFAULT = 1 << 28
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "roofline_traffic.json")
PLANS_PATH = os.path.join(ROOT, "paper_1401_0248_gb300", "plans_gb300.txt")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0

# Binary64-pipe instructions per element that the binary64 kernels issue:
# the twofold steps keep two roundings on the binary64 pipe (t = s + p and
# e = e + y; dots also q + ep) and compute the exact error terms and the
# product on the integer pipe; plain keeps its add (and multiply).  The
# twofold kernels and the plain sum issue their adds as DFMA by 1.0 (the
# faster binary64 instruction on GB300), the plain dot as DADD after its
# multiply; each is held against its own measured rate.
FP64_PIPE_OPS = {("sum", "plain"): 1, ("sum", "fast"): 2, ("sum", "rigorous"): 2,
                 ("dot", "plain"): 2, ("dot", "fast"): 3, ("dot", "rigorous"): 3}
# the paper's operation counts (Examples 1 and 3; dots add TwoProduct and one add)
PAPER_OPS = {("sum", "plain"): 1, ("sum", "fast"): 4, ("sum", "rigorous"): 7,
             ("dot", "plain"): 2, ("dot", "fast"): 7, ("dot", "rigorous"): 10}
FALLBACK_DADD_GOPS = 528.0   # binary64 adds/s of a GB300 (1.67/clk/SM at 2.07 GHz)
FALLBACK_DFMA_GOPS = 626.0   # binary64 fused multiply-adds/s (2/clk/SM at 2.07 GHz)


def kernel_sources_hash(files=("tf_device.cuh", "tf_flat.cu")):
    """Hash of the code a kernel is built from (the single-vector kernel by
    default), comments and blank space left out so that only a change of code
    counts; a recorded ncu traffic figure is used only while it matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1401_0248_gb300", "csrc")
    for f in files:
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(" ".join(line.split()) for line in src.splitlines() if line.strip())
        h.update(f.encode())
        h.update(code.encode())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------- distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = os.environ.get("TF_BENCH_BACKEND", "nccl")
    if backend == "nccl":
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)
    return rank, ws, local


def max_over_ranks(value, world):
    """max of a float over all ranks (identity at world size 1)"""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def gather_pairs(pair, world):
    """Every rank's shard pair in rank order: a (world, 2) tensor on the
    pair's device, from one all-gather of 16 bytes per rank (the only data
    exchange of a vector split over several GPUs)."""
    import torch
    if world <= 1:
        return pair.reshape(1, 2)
    import torch.distributed as dist
    parts = [torch.empty_like(pair) for _ in range(world)]
    dist.all_gather(parts, pair.contiguous())
    return torch.stack(parts)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, enabled=True):
        self.index = index
        self.enabled = enabled
        self.proc = None
        # the raw samples; TF_BENCH_CLOCKS_DIR keeps them somewhere lasting
        base = os.environ.get("TF_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(base, "bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        if not self.enabled:
            return self
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- workload
def build_workload(n, device, seed=0, conds=CONDS):
    import torch
    from paper_1401_0248_gb300 import inputs as I
    data = {}
    for dt in ("f32", "f64"):
        for cond in conds:
            s = I.ill_conditioned(n, dt, cond, seed=seed, device=device)
            d = I.ill_conditioned(n, dt, cond, seed=seed + 1, device=device, dot=True)
            data[(dt, cond)] = {"sum": (s.x, None, s.S, s.cond), "dot": (d.x, d.y, d.S, d.cond)}
    torch.cuda.synchronize()
    return data


def kernel_list(include_baselines, conds=CONDS, only=None):
    """(dtype, cond, op, variant, in_step) of every launch; `only` keeps the
    named kernels ("f64_dot_rigorous", ...) for profiling runs."""
    ks = []
    for dt in ("f32", "f64"):
        for cond in conds:
            for op in OPS:
                for v in TWOFOLD:
                    ks.append((dt, cond, op, v, True))
                if include_baselines:
                    ks.append((dt, cond, op, "plain", False))
                    ks.append((dt, cond, op, "wide", False))
    if only:
        ks = [k for k in ks if "%s_%s_%s" % (k[0], k[2], k[3]) in only]
        ks = [(a, b, c, d, True) for a, b, c, d, _ in ks]
    return ks


def nbytes(dt, op, n):
    return n * (4 if dt == "f32" else 8) * (2 if op == "dot" else 1)


def rel_err(S, v, e=0.0):
    if S == 0:
        return None
    approx = Fraction(float(v)) + Fraction(float(e))
    return float(abs(S - approx) / abs(S))


def run_gpu(args, rank, world, local):
    import torch
    from paper_1401_0248_gb300 import twofold as tf

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if os.path.exists(PLANS_PATH):
        tf.plan_load(PLANS_PATH)
    n = args.n
    data = build_workload(n, dev, seed=rank, conds=args.conds)
    ks_all = kernel_list(True, args.conds, args.only)
    step_ks = [k for k in ks_all if k[4]]
    wsz = max(tf.workspace_size(op, False, torch.float32 if dt == "f32" else torch.float64, v, n)
              for dt, _, op, v, _ in ks_all)
    ws = torch.zeros(wsz, dtype=torch.uint8, device=dev)
    outs = {k: torch.empty(2, dtype=torch.float32 if k[0] == "f32" else torch.float64, device=dev)
            for k in ks_all}
    stream = torch.cuda.current_stream(dev)

    def launch(k):
        dt, cond, op, v, _ = k
        x, y, _, _ = data[(dt, cond)][op]
        if op == "sum":
            tf.sum(x, v, out=outs[k], ws=ws)
        else:
            tf.dot(x, y, v, out=outs[k], ws=ws)

    # warm-up steps (also loads the kernels)
    for _ in range(args.warmup):
        for k in ks_all:
            launch(k)
    torch.cuda.synchronize()

    # timed steps: events around each launch on the launching stream
    ev = {k: [] for k in step_ks}
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local, enabled=not args.no_clocks) as clk:
        t_wait = time.perf_counter() + (0.5 if not args.no_clocks else 0.0)
        while time.perf_counter() < t_wait:          # let the sampler start under load
            launch(step_ks[-1])
            torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            for k in step_ks:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                launch(k)
                b.record(stream)
                ev[k].append((a, b))
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    step_ms_local = t_start.elapsed_time(t_end) / args.steps
    step_ms = max_over_ranks(step_ms_local, world)
    clocks = clk.summary()
    kern_ms = {k: sum(a.elapsed_time(b) for a, b in ev[k]) / len(ev[k]) for k in step_ks}

    # baselines alongside (plain, wide): timed the same way, outside the step
    base_ms = {}
    for k in [k for k in ks_all if not k[4]]:
        for _ in range(2):
            launch(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        reps = max(3, args.steps)
        a.record(stream)
        for _ in range(reps):
            launch(k)
        b.record(stream)
        torch.cuda.synchronize()
        base_ms[k] = a.elapsed_time(b) / reps

    probes = None if args.no_probes else run_probes(data, dev, stream, args.conds[0])

    step_bytes = sum(nbytes(k[0], k[2], n) for k in step_ks)
    total_bytes = sum_over_ranks(step_bytes, world)
    value = total_bytes / (step_ms * 1e-3) / 1e9

    # per-kernel report and accuracy: fractions of the measured copy rate, of
    # the measured read rate of as many arrays (probe: one array for sums,
    # two for dots) and of the nominal 7.9 TB/s
    hbm, peak_kind = load_peaks()
    kernels, accuracy = {}, {}
    for k in ks_all:
        dt, cond, op, v, _ = k
        ms = kern_ms.get(k, base_ms.get(k))
        gbs = nbytes(dt, op, n) / (ms * 1e-3) / 1e9
        read_bw = (probes or {}).get("read2_gbs" if op == "dot" else "read1_gbs")
        name = "%s_%s_%s_c%g" % (dt, op, v, cond)
        kernels[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4),
                         "frac_read": round(gbs / read_bw, 4) if read_bw else None,
                         "frac_nominal": round(gbs / NOMINAL_HBM_GBS, 4),
                         "gelem_s": round(n / (ms * 1e-3) / 1e9, 2)}
        _, _, S, cond_got = data[(dt, cond)][op]
        o = outs[k].cpu().tolist()
        acc = {"cond": float("%.3g" % cond_got), "rel_err_v_plus_e": rel_err(S, o[0], o[1]),
               "rel_err_v": rel_err(S, o[0])}
        if v in TWOFOLD:
            rv = S - Fraction(float(o[0]))
            acc["e_over_residual"] = (float(Fraction(float(o[1])) / rv) if rv != 0 else None)
            # the paper's bound with gamma_{N-1} (finite for binary64 at this N):
            # |S - (v + e)| <= u|S| + gamma_{N-1}^2 sum|x|, sum|x| = cond |S|
            u = 2.0 ** -53 if dt == "f64" else 2.0 ** -24
            if (n - 1) * u < 1 and S != 0:
                g = (n - 1) * u / (1 - (n - 1) * u)
                bound = u * abs(float(S)) + g * g * cond_got * abs(float(S))
                err = abs(S - Fraction(float(o[0])) - Fraction(float(o[1])))
                acc["within_literal_bound"] = bool(float(err) <= bound)
        accuracy[name] = acc

    # how well e estimates the value's own error: rho = e / (S - v) over the
    # step's twofold results
    rhos = [a["e_over_residual"] for a in accuracy.values() if a.get("e_over_residual") is not None]
    nz = [r for r in rhos if r != 0.0]
    zero_ok = [float(Fraction(float(outs[k].cpu()[1]))) == 0.0 for k in step_ks
               if data[(k[0], k[1])][k[2]][2] == Fraction(float(outs[k].cpu()[0]))]
    e_tracking = {
        "n": len(rhos),
        "median_abs_log2_rho": round(statistics.median(abs(math.log2(abs(r))) for r in nz), 6)
        if nz else None,
        "n_e_zero_with_residual": len(rhos) - len(nz),
        "frac_rho_in_half_to_2": round(sum(0.5 <= r <= 2.0 for r in rhos) / len(rhos), 4)
        if rhos else None,
        "e_zero_where_value_exact": (all(zero_ok) if zero_ok else None, len(zero_ok)),
    }

    # roofline of the kernel with the largest share of the step
    dom = max(step_ks, key=lambda k: kern_ms[k])
    dt, cond, op, v, _ = dom
    dom_name = "%s_%s_%s" % (dt, op, v)
    dom_ms = statistics.mean(kern_ms[k] for k in step_ks if k[0] == dt and k[2] == op and k[3] == v)
    traffic = None
    try:
        with open(TRAFFIC_PATH) as f:
            tr = json.load(f)
        ent = tr.get("kernels", {}).get(dom_name)
        if ent and tr.get("sources_hash") == kernel_sources_hash() and ent.get("n") == n:
            traffic = ent["dram_bytes"]
    except Exception:
        pass
    bytes_dom = nbytes(dt, op, n)
    ach = bytes_dom / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": traffic, "kernel": dom_name,
                "bytes_per_launch": bytes_dom, "ms_per_launch": round(dom_ms, 4),
                "peak_source": "%s HBM copy bandwidth (MEASURED_PEAKS.json)" % peak_kind
                if peak_kind == "measured" else "fallback HBM figure (no MEASURED_PEAKS.json)"}
    if dt == "f64":
        # what limits the binary64 kernels: the binary64 pipe (with the exact
        # error terms on the integer pipe); its issued adds against the
        # measured rate of the instruction they use (DFMA by 1.0, except the
        # plain dot's DADD)
        fma_adds = op == "sum" or v != "plain"
        peak_ops = (probes or {}).get("dadd_as_fma_gops" if fma_adds else "dadd_gops") \
            or (FALLBACK_DFMA_GOPS if fma_adds else FALLBACK_DADD_GOPS)
        ops = FP64_PIPE_OPS[(op, v)] * n / (dom_ms * 1e-3) / 1e9
        roofline["alu"] = {
            "achieved": round(ops, 1), "peak": round(peak_ops, 1),
            "unit": "G binary64-pipe ops/s", "frac": round(ops / peak_ops, 4),
            "ops_per_element": FP64_PIPE_OPS[(op, v)],
            "peak_source": ("measured rate of binary64 adds issued as DFMA by a runtime 1.0 "
                            "(probe kind 10) on this GPU" if fma_adds else
                            "measured binary64 add rate (probe kind 1) on this GPU")
            if probes else "fallback (no probes)",
            "paper_ops_per_s_g": round(PAPER_OPS[(op, v)] * n / (dom_ms * 1e-3) / 1e9, 1)}

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded SplitMix64; ill-conditioned, exact sum known by construction)",
        "config": {"workload": "single vectors N=2^28, f32+f64, twofold sum+dot, fast+rigorous, "
                               "cond 1e4/1e8/1e16 (24 reductions per step)",
                   "n": n, "conds": list(args.conds), "l2": "inputs larger than L2 (1-4 GiB each)",
                   "subset": sorted(args.only) or None,
                   "parallelism": "replicas" if world == 1 else "independent problems per rank"},
        "gpu_launches": len(step_ks) * args.steps,
        "clocks": clocks,
        "roofline": roofline,
        "kernels": kernels,
        "accuracy": accuracy,
        "e_tracking": e_tracking,
        "probes": probes,
    }
    return result, data, ws, outs, ks_all, step_ks


def run_split(args, rank, world, local):
    """One vector per reduction cut into `world` contiguous shards: each rank
    reduces its shard (binary64 pair output), the pairs are all-gathered in
    rank order and merged on the device (tf_merge_pairs).  Total work is
    fixed as the rank count grows ("scaling": "strong"); the step time is the
    slowest rank's, gather and merge included."""
    import torch
    from paper_1401_0248_gb300 import twofold as tf

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if os.path.exists(PLANS_PATH):
        tf.plan_load(PLANS_PATH)
    n = args.n
    data = build_workload(n, dev, seed=0, conds=args.conds)     # the same vectors on every rank
    step_ks = kernel_list(False, args.conds, args.only)
    wsz = max(tf.workspace_size(op, False, torch.float32 if dt == "f32" else torch.float64, v, n)
              for dt, _, op, v, _ in step_ks)
    ws = torch.zeros(wsz, dtype=torch.uint8, device=dev)
    pair = {k: torch.empty(2, dtype=torch.float64, device=dev) for k in step_ks}
    outs = {k: torch.empty(2, dtype=torch.float32 if k[0] == "f32" else torch.float64, device=dev)
            for k in step_ks}
    stream = torch.cuda.current_stream(dev)

    def launch(k):
        dt, cond, op, v, _ = k
        x, y, _, _ = data[(dt, cond)][op]
        a, b = tf.shard_bounds(n, world, x.dtype)[rank]
        if op == "sum":
            tf.sum(x[a:b], v, out_f64=True, out=pair[k], ws=ws)
        else:
            tf.dot(x[a:b], y[a:b], v, out_f64=True, out=pair[k], ws=ws)
        tf.merge_pairs(gather_pairs(pair[k], world), x.dtype, v, out=outs[k])

    for _ in range(args.warmup):
        for k in step_ks:
            launch(k)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local, enabled=not args.no_clocks) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            for k in step_ks:
                launch(k)
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    step_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, world)
    total_bytes = sum(nbytes(k[0], k[2], n) for k in step_ks)
    accuracy = {}
    for k in step_ks:
        dt, cond, op, v, _ = k
        S = data[(dt, cond)][op][2]
        o = outs[k].cpu().tolist()
        accuracy["%s_%s_%s_c%g" % (dt, op, v, cond)] = {
            "rel_err_v_plus_e": rel_err(S, o[0], o[1]), "rel_err_v": rel_err(S, o[0])}
    return {
        "metric": METRIC, "value": round(total_bytes / (step_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded SplitMix64; ill-conditioned, exact sum known by construction)",
        "config": {"workload": "single vectors N=2^28 split over the ranks, f32+f64, twofold "
                               "sum+dot, fast+rigorous, cond 1e4/1e8/1e16 (24 reductions per step)",
                   "n": n, "conds": list(args.conds), "l2": "inputs larger than L2",
                   "parallelism": "split: one vector in %d contiguous shards, shard pairs "
                                  "all-gathered and merged in rank order" % world},
        "gpu_launches": 2 * len(step_ks) * args.steps,
        "clocks": clk.summary(),
        "accuracy": accuracy,
    }


def run_probes(data, dev, stream, cond0):
    """Read bandwidth (the paper's read1/read2) and arithmetic rates (its
    p-functions) of this GPU, measured with the library's probe kernels."""
    import torch
    from paper_1401_0248_gb300 import twofold as tf
    sms = tf.sm_count()
    out = {}
    x, y, _, _ = data[("f64", cond0)]["dot"]
    xs = data[("f32", cond0)]["sum"][0]
    # the best of a few launch shapes and of the step's 1 and 2 GiB arrays
    # (the probe's own roofline, as the paper's read1/read2 are the best of
    # its read loops)
    for name, args_ in (("read1_gbs", (x, None)), ("read1_gbs", (xs, None)),
                        ("read2_gbs", (x, y))):
        b = args_[0].numel() * args_[0].element_size() * (2 if args_[1] is not None else 1)
        best = 1e30
        for unroll in (1, 2, 4, 8):
            for bps, threads in ((2, 512), (4, 512), (2, 1024), (8, 256), (4, 256)):
                # launches queued back to back, as the kernels run in the step
                # (a lone launch's event pair would also time its issue gap)
                for _ in range(2):
                    a = torch.cuda.Event(enable_timing=True)
                    e = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    for _ in range(5):
                        tf.probe_read(args_[0], args_[1], blocks=bps * sms, threads=threads,
                                      unroll=unroll)
                    e.record(stream)
                    torch.cuda.synchronize()
                    best = min(best, a.elapsed_time(e) / 5)
        out[name] = max(out.get(name, 0.0), round(b / (best * 1e-3) / 1e9, 1))
    blocks, threads = 4 * sms, 256
    for kind, iters in (("fadd", 20000), ("dadd", 2000), ("dfma", 2000), ("iadd", 20000),
                        ("fast_f32", 5000), ("rigorous_f32", 3000), ("fast_f64", 500),
                        ("rigorous_f64", 300), ("dmul", 2000), ("dadd_as_fma", 2000)):
        tf.probe_alu(kind, iters // 10, blocks, threads, device=dev)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tf.probe_alu(kind, iters, blocks, threads, device=dev)
        e.record(stream)
        torch.cuda.synchronize()
        ops = tf.ALU_OPS_PER_ITER[tf.ALU_KINDS[kind]] * iters * blocks * threads
        out[kind + "_gops"] = round(ops / (a.elapsed_time(e) * 1e-3) / 1e9, 1)
    return out


def _time_calls(call, stream, warmup, reps):
    for _ in range(warmup):
        call()
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        call()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _accuracy_entry(S, sabs, o, twofold):
    acc = {"rel_err_v_plus_e": rel_err(S, o[0], o[1]), "rel_err_v": rel_err(S, o[0])}
    if twofold:
        rv = S - Fraction(float(o[0]))
        acc["e_over_residual"] = float(Fraction(float(o[1])) / rv) if rv != 0 else None
    return acc


def run_c3(args, dev, stream, hbm):
    """Binary32 twofold dots of N = 2^30 per vector (4 GiB each): N(0,1) and
    signed log-normal(0, 2) data; binary32 arithmetic with a binary64 merge
    across blocks, beside the binary64 accumulator ('wide') and the plain
    binary32 dot, each against the exact dot (integer limb sums)."""
    import torch
    from paper_1401_0248_gb300 import inputs as I
    from paper_1401_0248_gb300 import twofold as tf
    n = args.c3_n
    res = {"config": "binary32 dot, N=%d per vector, N(0,1) and signed log-normal(0,2), seed 0" % n,
           "kernels": {}}
    ws = torch.zeros(tf.workspace_size("dot", False, torch.float32, "fast", n), dtype=torch.uint8,
                     device=dev)
    for dist in ("normal", "lognormal"):
        if dist == "normal":
            x = I.normal(n, "f32", seed=0, stream=0, device=dev)
            y = I.normal(n, "f32", seed=0, stream=3, device=dev)
        else:
            x = I.signed_lognormal(n, "f32", seed=0, stream=0, device=dev)
            y = I.signed_lognormal(n, "f32", seed=0, stream=5, device=dev)
        S = I.exact_dot_f32(x, y)
        sabs = 0.0
        for a in range(0, n, 1 << 26):
            sabs += float(torch.sum(torch.abs(x[a:a + (1 << 26)].double() * y[a:a + (1 << 26)].double())))
        ent = {"cond": float("%.3g" % (sabs / abs(float(S)))), "variants": {}}
        out = torch.empty(2, dtype=torch.float32, device=dev)
        for v in ("fast", "rigorous", "wide", "plain"):
            ms = _time_calls(lambda: tf.dot(x, y, v, out=out, ws=ws), stream, args.warmup,
                             max(5, min(args.steps, 10)))
            gbs = nbytes("f32", "dot", n) / (ms * 1e-3) / 1e9
            o = out.cpu().tolist()
            e = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4)}
            e.update(_accuracy_entry(S, sabs, o, v in TWOFOLD))
            ent["variants"][v] = e
        for v in TWOFOLD:
            ent["variants"][v]["vs_plain_time"] = round(ent["variants"][v]["ms"] /
                                                       ent["variants"]["plain"]["ms"], 4)
        res["kernels"][dist] = ent
        del x, y
        torch.cuda.empty_cache()
    return res


def run_c5(args, dev, stream, hbm):
    """Binary64 twofold dots of N = 2^29 per vector (4 GiB each) on
    ill-conditioned data (condition numbers 1e8, 1e16, 1e24, 1e30; exact dot
    known by construction), fast against rigorous beside the plain dot, with
    the error term's tracking of the value's error and 20 repeated runs of
    each twofold variant checked for identical bits."""
    import torch
    from paper_1401_0248_gb300 import inputs as I
    from paper_1401_0248_gb300 import twofold as tf
    n = args.c5_n
    res = {"config": "binary64 dot, N=%d per vector, ill-conditioned, seed 0" % n, "kernels": {}}
    ws = torch.zeros(tf.workspace_size("dot", False, torch.float64, "fast", n), dtype=torch.uint8,
                     device=dev)
    for cond in (1e8, 1e16, 1e24, 1e30):
        ic = I.ill_conditioned(n, "f64", cond, seed=0, device=dev, dot=True)
        ent = {"cond": float("%.3g" % ic.cond), "variants": {}}
        out = torch.empty(2, dtype=torch.float64, device=dev)
        for v in ("fast", "rigorous", "plain"):
            ms = _time_calls(lambda: tf.dot(ic.x, ic.y, v, out=out, ws=ws), stream, args.warmup,
                             max(5, min(args.steps, 10)))
            gbs = nbytes("f64", "dot", n) / (ms * 1e-3) / 1e9
            o = out.cpu().tolist()
            e = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4)}
            e.update(_accuracy_entry(ic.S, ic.sum_abs, o, v in TWOFOLD))
            if v in TWOFOLD:
                ref = out.clone()
                same = True
                for _ in range(20):
                    tf.dot(ic.x, ic.y, v, out=out, ws=ws)
                    same = same and bool(torch.equal(out.view(torch.int64), ref.view(torch.int64)))
                e["bits_identical_20_runs"] = same
            ent["variants"][v] = e
        for v in TWOFOLD:
            ent["variants"][v]["vs_plain_time"] = round(ent["variants"][v]["ms"] /
                                                       ent["variants"]["plain"]["ms"], 4)
        res["kernels"]["c%g" % cond] = ent
        del ic
        torch.cuda.empty_cache()
    return res


def run_misaligned(args, data, dev, stream):
    """The cost of an input that is element-aligned but not 16-byte aligned:
    the kernels then load it with scalar loads in the same order (same bits).
    The step's binary32 fast sum and binary64 fast dot (cond 1e8), timed on
    views that start one element into the arrays, against the aligned views
    of the same n - 1 elements."""
    import torch
    from paper_1401_0248_gb300 import twofold as tf
    cond = 1e8 if 1e8 in args.conds else args.conds[0]
    res = {"config": "views one element into the step's arrays (n - 1 elements)", "kernels": {}}
    reps = max(5, min(args.steps, 10))
    for dt, op in (("f32", "sum"), ("f64", "dot")):
        x, y, _, _ = data[(dt, cond)][op]
        n = x.numel() - 1
        xa, xm = x[:n].clone(), x[1:]
        ya, ym = (y[:n].clone(), y[1:]) if y is not None else (None, None)
        ws = torch.zeros(tf.workspace_size(op, False, x.dtype, "fast", n), dtype=torch.uint8,
                         device=dev)
        out = torch.empty(2, dtype=x.dtype, device=dev)
        ms = {}
        for name, xx, yy in (("aligned", xa, ya), ("misaligned", xm, ym)):
            call = ((lambda xx=xx: tf.sum(xx, "fast", out=out, ws=ws)) if op == "sum" else
                    (lambda xx=xx, yy=yy: tf.dot(xx, yy, "fast", out=out, ws=ws)))
            ms[name] = _time_calls(call, stream, args.warmup, reps)
        res["kernels"]["%s_%s_fast" % (dt, op)] = {
            "aligned_ms": round(ms["aligned"], 4), "misaligned_ms": round(ms["misaligned"], 4),
            "slowdown": round(ms["misaligned"] / ms["aligned"], 3)}
        del xa, ya
        torch.cuda.empty_cache()
    return res


def run_small(dev, stream, reps=20):
    """The L2-resident case: N = 2^20 binary64 (8 MiB per operand), uniform
    [-1, 1).  Launches are replayed from CUDA graphs so that the host's call
    overhead is not timed: hot = `reps` launches back to back; flushed =
    `reps` launches each after writing a 256 MiB buffer (larger than L2),
    minus the same graph without the launches."""
    import torch
    from paper_1401_0248_gb300 import inputs as I
    from paper_1401_0248_gb300 import twofold as tf
    n = 1 << 20
    x = I.uniform(n, "f64", seed=0, stream=0, device=dev)
    y = I.uniform(n, "f64", seed=0, stream=1, device=dev)
    ws = torch.zeros(tf.workspace_size("dot", False, torch.float64, "rigorous", n),
                     dtype=torch.uint8, device=dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(1 << 28, dtype=torch.uint8, device=dev)

    def graph_ms(body, replays=5):
        body()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream(device=dev)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            with torch.cuda.graph(g, stream=gs):
                body()
        torch.cuda.synchronize()
        g.replay()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(replays):
            g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        del g
        return a.elapsed_time(b) / replays

    def flushes():
        for _ in range(reps):
            flush.fill_(1)
    t_flush = graph_ms(flushes)
    res = {"config": "N=2^20 f64, uniform [-1, 1); CUDA-graph replay", "kernels": {}}
    for op in OPS:
        for v in TWOFOLD + ("plain",):
            def call():
                if op == "sum":
                    tf.sum(x, v, out=out, ws=ws)
                else:
                    tf.dot(x, y, v, out=out, ws=ws)

            def hot_body():
                for _ in range(reps):
                    call()

            def cold_body():
                for _ in range(reps):
                    flush.fill_(1)
                    call()
            hot = graph_ms(hot_body) / reps
            cold = max(graph_ms(cold_body) - t_flush, 0.0) / reps
            byts = nbytes("f64", op, n)
            res["kernels"]["f64_%s_%s" % (op, v)] = {
                "hot_us": round(hot * 1e3, 2), "hot_gbs": round(byts / (hot * 1e-3) / 1e9, 1),
                "flushed_us": round(cold * 1e3, 2),
                "flushed_gbs": round(byts / (cold * 1e-3) / 1e9, 1) if cold > 0 else None}
    del flush
    return res


def run_batched(args, dev, stream):
    """The ragged-batch configuration beside the step: 16,384 binary32 CSR
    segments with log-uniform lengths in [16, 2^18] (uniform [-1, 1) data),
    each call an offsets check, one persistent launch and the merge of the
    segments over several tiles, replayed from a CUDA graph; the twofold
    binary64 forms of the same layout beside it."""
    import torch
    from paper_1401_0248_gb300 import inputs as I
    from paper_1401_0248_gb300 import twofold as tf
    nseg = 16384
    L = I.csr_lengths(nseg, 16, 1 << 18, seed=0)
    off_h = I.csr_offsets(L)
    n = int(off_h[-1])
    off = torch.from_numpy(off_h).to(dev)
    hbm, _ = load_peaks()
    res = {"config": "16384 segments, lengths log-uniform [16, 2^18], %d elements; "
                     "binary32 (the configuration) and binary64 (beside it)" % n,
           "graph": True, "kernels": {}}
    for dt, td, variants in (("f32", torch.float32, ("plain", "fast", "rigorous")),
                             ("f64", torch.float64, ("fast", "rigorous"))):
        x = I.uniform(n, dt, seed=1, device=dev)
        y = I.uniform(n, dt, seed=1, stream=1, device=dev)
        _batched_kernels(args, tf, dev, stream, res, dt, td, variants, x, y, off, n, nseg, hbm)
        del x, y
        torch.cuda.empty_cache()
    return res


def _batched_kernels(args, tf, dev, stream, res, dt, td, variants, x, y, off, n, nseg, hbm):
    import torch
    for op in OPS:
        for v in variants:
            ws = torch.zeros(tf.workspace_size(op, True, td, v, n, nseg),
                             dtype=torch.uint8, device=dev)
            out = torch.empty(nseg, 2, dtype=td, device=dev)
            if op == "sum":
                call = (lambda v=v, ws=ws, out=out: tf.sum_batched(x, off, v, ws=ws, out=out))
            else:
                call = (lambda v=v, ws=ws, out=out: tf.dot_batched(x, y, off, v, ws=ws, out=out))
            call()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            gs = torch.cuda.Stream(device=dev)
            gs.wait_stream(stream)
            with torch.cuda.stream(gs):
                with torch.cuda.graph(g, stream=gs):
                    call()
            torch.cuda.synchronize()
            for _ in range(args.warmup):
                g.replay()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            reps = max(5, args.steps)
            a.record(stream)
            for _ in range(reps):
                g.replay()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            byts = nbytes(dt, op, n) + 8 * (nseg + 1) + 2 * (4 if dt == "f32" else 8) * nseg
            gbs = byts / (ms * 1e-3) / 1e9
            ent = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4)}
            if v != "plain":
                # the single-vector kernel on the same concatenated data: what
                # the segments cost beside one long reduction
                fws = torch.zeros(tf.workspace_size(op, False, td, v, n), dtype=torch.uint8,
                                  device=dev)
                fo = torch.empty(2, dtype=td, device=dev)
                fcall = ((lambda v=v: tf.sum(x, v, ws=fws, out=fo)) if op == "sum" else
                         (lambda v=v: tf.dot(x, y, v, ws=fws, out=fo)))
                fms = _time_calls(fcall, stream, args.warmup, max(5, min(args.steps, 10)))
                ent["flat_same_data_ms"] = round(fms, 4)
                ent["batched_over_flat"] = round(ms / fms, 4)
            res["kernels"]["%s_%s_%s" % (dt, op, v)] = ent
            del g


def gpu_numa_cpus(dev):
    """CPUs of the NUMA node the GPU hangs off (host buffers are placed there
    by first touch), or None when the topology is not visible."""
    try:
        import torch
        props = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
        with open("/sys/bus/pci/devices/%s/numa_node" % bus) as f:
            node = int(f.read().strip())
        if node < 0:
            return None
        with open("/sys/devices/system/node/node%d/cpulist" % node) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        return node, cpus
    except Exception:
        return None


def run_e2e(args, data, ws, step_ks, dev):
    """The step through the asynchronous host-buffer C-ABI calls: each
    reduction's pinned inputs are copied to its own device buffers on a copy
    stream, the reduction runs on the compute stream behind its copy (an
    event), its pair comes back to pinned host memory, and the host waits
    once per step."""
    import torch
    from paper_1401_0248_gb300 import twofold as tf
    numa = gpu_numa_cpus(dev)
    old_aff = None
    if numa is not None:
        try:
            old_aff = os.sched_getaffinity(0)
            os.sched_setaffinity(0, numa[1])
        except Exception:
            old_aff = None
    host = {}
    for k in step_ks:
        dt, cond, op, _, _ = k
        if (dt, cond, op) not in host:
            x, y, _, _ = data[(dt, cond)][op]
            xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
            xh.copy_(x)
            yh = None
            if y is not None:
                yh = torch.empty(y.shape, dtype=y.dtype, pin_memory=True)
                yh.copy_(y)
            host[(dt, cond, op)] = (xh, yh)
    # device buffers of their own per reduction, so that no copy refills a
    # buffer an earlier reduction of the same step still reads
    dbuf = {}
    for k in step_ks:
        xh, yh = host[k[:3]]
        dbuf[k] = (torch.empty_like(xh, device=dev),
                   torch.empty_like(yh, device=dev) if yh is not None else None)
    outs = {k: torch.empty(2, dtype=torch.float32 if k[0] == "f32" else torch.float64,
                           pin_memory=True) for k in step_ks}
    copy_stream = torch.cuda.Stream(device=dev)
    reps = max(1, min(args.steps, 3))

    def one_step():
        for k in step_ks:
            dt, cond, op, v, _ = k
            xh, yh = host[k[:3]]
            xd, yd = dbuf[k]
            if op == "sum":
                tf.sum_host_async(xh, v, x_dev=xd, ws=ws, out=outs[k], copy_stream=copy_stream)
            else:
                tf.dot_host_async(xh, yh, v, x_dev=xd, y_dev=yd, ws=ws, out=outs[k],
                                  copy_stream=copy_stream)
        torch.cuda.synchronize(dev)

    def copies_only():
        # the same host-to-device traffic with no reductions: the host link's
        # rate at this moment, the ceiling of the end-to-end figure
        with torch.cuda.stream(copy_stream):
            for k in step_ks:
                xh, yh = host[k[:3]]
                xd, yd = dbuf[k]
                xd.copy_(xh, non_blocking=True)
                if yh is not None:
                    yd.copy_(yh, non_blocking=True)
        torch.cuda.synchronize(dev)

    one_step()        # warm
    t0 = time.perf_counter()
    for _ in range(reps):
        one_step()
    dt_s = (time.perf_counter() - t0) / reps
    copies_only()
    t0 = time.perf_counter()
    for _ in range(reps):
        copies_only()
    dt_copy = (time.perf_counter() - t0) / reps
    if old_aff is not None:
        os.sched_setaffinity(0, old_aff)
    n = args.n
    step_bytes = sum(nbytes(k[0], k[2], n) for k in step_ks)
    bo = sum(16 if k[0] == "f64" else 8 for k in step_ks)
    del dbuf
    torch.cuda.empty_cache()
    return {"value": round(step_bytes / dt_s / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": step_bytes, "d2h_bytes_per_step": bo,
            "ms_per_step": round(dt_s * 1e3, 3), "steps": reps,
            "link_gbs": round(step_bytes / dt_copy / 1e9, 2),
            "e2e_over_link": round(dt_copy / dt_s, 4),
            "calls": "tf_sum_host_async / tf_dot_host_async, copies on a second stream, "
                     "one host wait per step",
            "host_numa_node": None if numa is None else numa[0]}


# ------------------------------------------------------------ CPU oracle
def cpu_oracle_step(data_host, m):
    """The oracle's sequential twofold loops (Examples 1 and 3 and their
    TwoProduct dot forms) over the first m elements of each of the step's
    inputs.  Returns (bytes, seconds)."""
    import oracle as O
    loops = {("sum", "fast"): "sumtf", ("sum", "rigorous"): "sumt",
             ("dot", "fast"): "dottf2", ("dot", "rigorous"): "dott2"}
    t0 = time.perf_counter()
    b = 0
    for (dt, cond, op), (x, y) in data_host.items():
        for v in TWOFOLD:
            O.loop(loops[(op, v)], x[:m], None if y is None else y[:m])
            b += nbytes(dt, op, min(m, x.size))
    return b, time.perf_counter() - t0


def host_sample(data, m):
    out = {}
    for (dt, cond), d in data.items():
        for op in OPS:
            x, y, _, _ = d[op]
            out[(dt, cond, op)] = (x[:m].cpu().numpy(), None if y is None else y[:m].cpu().numpy())
    return out


def run_cpu_baseline(data, m):
    import oracle as O
    hs = host_sample(data, m)
    b, s = cpu_oracle_step(hs, m)
    el = sum(min(m, x.size) for x, _ in hs.values()) * len(TWOFOLD)
    # context: the exact superaccumulator on all host cores, and the paper's
    # binary128 ('d' for double) loop on one core, on the f64 cond-1e8 sample
    x = hs[("f64", 1e8, "sum")][0] if ("f64", 1e8, "sum") in hs else next(iter(hs.values()))[0]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    O.exact(x, nthreads=cores)
    t_ex = time.perf_counter() - t0
    extra = {"exact_superaccumulator_elem_s": round(x.size / t_ex, 1), "exact_cores": cores}
    if x.dtype == np.float64:
        t0 = time.perf_counter()
        O.loop("sumq", x)
        t_q = time.perf_counter() - t0
        extra["sumq_f64_gbs_one_core"] = round(x.nbytes / t_q / 1e9, 4)
    return {"value": round(b / s / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first %d elements of each of the step's 24 inputs, the oracle's "
                      "sequential twofold loops (one host thread, as in the paper)" % m,
            "seconds": round(s, 2), "elem_s": round(el / s, 1), "context": extra}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return None
    import torch
    from paper_1401_0248_gb300 import inputs as I
    m = args.ref_sample
    data = {}
    for dt in ("f32", "f64"):
        for cond in CONDS:
            s = I.ill_conditioned(m, dt, cond, seed=0)
            d = I.ill_conditioned(m, dt, cond, seed=1, dot=True)
            data[(dt, cond, "sum")] = (s.x.numpy(), None)
            data[(dt, cond, "dot")] = (d.x.numpy(), d.y.numpy())
    for _ in range(args.warmup):
        cpu_oracle_step(data, m)
    tot_b = tot_s = 0.0
    for _ in range(args.steps):
        b, s = cpu_oracle_step(data, m)
        tot_b += b
        tot_s += s
    value = tot_b / tot_s / 1e9
    del torch
    return {"metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_s / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded SplitMix64; ill-conditioned)", "impl": "reference",
            "config": {"workload": "single vectors, f32+f64, twofold sum+dot, fast+rigorous, "
                                   "cond 1e4/1e8/1e16 (24 reductions per step)",
                       "n": m, "conds": list(CONDS)},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "N=%d per input (bounded sample of the N=2^28 workload)" % m},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_layouts(args):
    """Batched binary32 fast sum and dot on layouts that separate the costs
    of the batched kernel: one segment per tile, two per tile, segments of two
    tiles, segments offset by half a tile (two cross-tile pieces per tile),
    one segment, and the 16,384-segment configuration, beside the flat kernel
    on the same elements (tile 16,384, CUDA-graph replay, inputs > L2)."""
    import torch
    from paper_1401_0248_gb300 import inputs as I
    from paper_1401_0248_gb300 import twofold as tf
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)
    T, ntile = 16384, 26607
    n = T * ntile
    Lc4 = I.csr_lengths(16384, 16, 1 << 18, seed=0)
    nal = max(n, int(I.csr_offsets(Lc4)[-1]))
    xa = I.uniform(nal, "f32", seed=1, device=dev)
    ya = I.uniform(nal, "f32", seed=1, stream=1, device=dev)
    layouts = {"one_seg_per_tile": [T] * ntile, "two_segs_per_tile": [T // 2] * (2 * ntile),
               "segs_of_two_tiles": [2 * T] * (ntile // 2) + [T] * (ntile % 2),
               "segs_offset_half_tile": [T // 2] + [T] * (ntile - 1) + [T // 2],
               "one_segment": [n], "c4_16384_segments": list(Lc4)}

    def timed(call):
        call()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream(device=dev)
        gs.wait_stream(st)
        with torch.cuda.stream(gs):
            with torch.cuda.graph(g, stream=gs):
                call()
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            g.replay()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.steps):
            g.replay()
        b.record(st)
        torch.cuda.synchronize()
        return round(a.elapsed_time(b) / args.steps, 4)

    res = {"tile": T, "elements": n, "ms": {}}
    for op in ("sum", "dot"):
        x, y = xa[:n], ya[:n]
        ws = torch.zeros(tf.workspace_size(op, False, torch.float32, "fast", n), dtype=torch.uint8,
                         device=dev)
        out = torch.empty(2, device=dev)
        res["ms"]["flat_%s" % op] = timed(
            (lambda: tf.sum(x, "fast", ws=ws, out=out)) if op == "sum" else
            (lambda: tf.dot(x, y, "fast", ws=ws, out=out)))
        p = tf.plan_get(op, True, torch.float32, "fast")
        tf.plan_set(op, True, torch.float32, "fast", p["block"], p["unroll"], p["blocks_per_sm"], T)
        try:
            for name, L in layouts.items():
                oh = I.csr_offsets(L)
                m = int(oh[-1])
                xs, ys = xa[:m], ya[:m]
                off = torch.from_numpy(oh).to(dev)
                wsb = torch.zeros(tf.workspace_size(op, True, torch.float32, "fast", m, len(L)),
                                  dtype=torch.uint8, device=dev)
                outb = torch.empty(len(L), 2, device=dev)
                res["ms"]["%s_%s" % (name, op)] = timed(
                    (lambda: tf.sum_batched(xs, off, "fast", ws=wsb, out=outb)) if op == "sum" else
                    (lambda: tf.dot_batched(xs, ys, off, "fast", ws=wsb, out=outb)))
        finally:
            tf.plan_set(op, True, torch.float32, "fast", p["block"], p["unroll"],
                        p["blocks_per_sm"], p["tile"])
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-sample", type=int, default=1 << 24)
    ap.add_argument("--ref-sample", type=int, default=1 << 22)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probes", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the N=2^30 / 2^29 dot configurations")
    ap.add_argument("--c3-n", type=int, default=1 << 30)
    ap.add_argument("--c5-n", type=int, default=1 << 29)
    ap.add_argument("--no-clocks", action="store_true", help="profiling: no nvidia-smi sampler")
    ap.add_argument("--only", default="", help="profiling: comma list of kernels, e.g. f64_dot_rigorous")
    ap.add_argument("--conds", default="1e4,1e8,1e16", help="profiling: condition numbers")
    ap.add_argument("--split", action="store_true",
                    help="one vector split over the ranks (shard pairs gathered and merged)")
    ap.add_argument("--layouts", action="store_true",
                    help="only the batched layout sweep (one JSON line of its own)")
    args = ap.parse_args(argv)
    args.only = set(k for k in args.only.split(",") if k)
    args.conds = tuple(float(c) for c in args.conds.split(","))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.layouts:
        print(json.dumps({"batched_layouts": run_layouts(args)}))
        return 0
    rank, world, local = dist_setup()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return 0
    import torch
    if args.split:
        res = run_split(args, rank, world, local)
        if rank == 0:
            print(json.dumps(res))
        barrier(world)
        return 0
    res, data, ws, outs, ks_all, step_ks = run_gpu(args, rank, world, local)
    if not args.no_batched:
        res["batched"] = run_batched(args, torch.device("cuda", local),
                                     torch.cuda.current_stream(torch.device("cuda", local)))
        res["small"] = run_small(torch.device("cuda", local),
                                 torch.cuda.current_stream(torch.device("cuda", local)))
    if not args.no_batched:
        d = torch.device("cuda", local)
        res["misaligned"] = run_misaligned(args, data, d, torch.cuda.current_stream(d))
    if not args.no_large:
        d = torch.device("cuda", local)
        hbm, _ = load_peaks()
        res["c3"] = run_c3(args, d, torch.cuda.current_stream(d), hbm)
        res["c5"] = run_c5(args, d, torch.cuda.current_stream(d), hbm)
    if not args.no_e2e:
        e2e = run_e2e(args, data, ws, step_ks, torch.device("cuda", local))
        e2e["value"] = round(sum_over_ranks(e2e["value"], world), 2) if world > 1 else e2e["value"]
        res["e2e"] = e2e
    if rank == 0:
        res["cpu_baseline"] = run_cpu_baseline(data, args.cpu_sample)
        print(json.dumps(res))
    barrier(world)
    return 0


if __name__ == "__main__":
    sys.exit(main())
