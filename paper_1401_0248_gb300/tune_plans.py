"""Tune the launch plans of every (op, batched, dtype, variant) key on this GPU
and write them to a plan file (loaded by tf_plan_load / twofold.plan_load).

Each key is timed with the library's tuner (tf_tune: block, unroll U,
blocks per SM and, for batched keys, the tile) on a representative
problem: single vectors of N elements of uniform data (and of 2^20 elements
for the plans of vectors of at most 2^22 elements), and a ragged batch of
log-uniform segment lengths in [16, 2^18].

    python -m paper_1401_0248_gb300.tune_plans [--out FILE] [--n N] [--nseg S]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans_gb300.txt")


def main(argv=None):
    import torch
    from paper_1401_0248_gb300 import inputs as I
    from paper_1401_0248_gb300 import twofold as tf

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--n", type=int, default=1 << 28)
    ap.add_argument("--small-n", type=int, default=1 << 20,
                    help="size for the plans of single vectors of at most 2^22 elements")
    ap.add_argument("--nseg", type=int, default=16384)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--flat-only", action="store_true")
    ap.add_argument("--batched-only", action="store_true")
    ap.add_argument("--small-only", action="store_true",
                    help="only the plans of single vectors of at most 2^22 elements")
    ap.add_argument("--variants", default="plain,fast,rigorous,wide,kahan",
                    help="comma list of plain, fast, rigorous, wide, kahan")
    ap.add_argument("--dtypes", default="f32,f64", help="comma list of f32, f64")
    ap.add_argument("--load", default=None, help="start from this plan file")
    args = ap.parse_args(argv)

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lengths = I.csr_lengths(args.nseg, 16, 1 << 18, seed=0)
    off = torch.from_numpy(I.csr_offsets(lengths)).to(dev)
    total = int(off[-1].item())
    if args.load:
        tf.plan_load(args.load)
    t0 = time.time()
    variants = args.variants.split(",")
    for dt, td in (("f32", torch.float32), ("f64", torch.float64)):
        if dt not in args.dtypes.split(","):
            continue
        if not args.batched_only:
            sizes = ((args.small_n, "small  "),) if args.small_only else \
                ((args.n, "flat   "), (args.small_n, "small  "))
            for n, label in sizes:
                x = I.uniform(n, dt, seed=0, device=dev)
                y = I.uniform(n, dt, seed=0, stream=1, device=dev)
                for op in ("sum", "dot"):
                    for variant in variants:
                        p = tf.tune(op, variant, x, y if op == "dot" else None,
                                    reps=args.reps if n > tf.SMALL_N else 10 * args.reps)
                        print("%s %s %s %-8s -> %s" % (label, dt, op, variant, p), flush=True)
                del x, y
        if args.flat_only or args.small_only:
            continue
        xs = I.uniform(total, dt, seed=1, device=dev)
        ys = I.uniform(total, dt, seed=1, stream=1, device=dev)
        for op in ("sum", "dot"):
            for variant in variants:
                p = tf.tune(op, variant, xs, ys if op == "dot" else None, offsets=off,
                            reps=args.reps)
                print("batched %s %s %-8s -> %s" % (dt, op, variant, p), flush=True)
        del xs, ys
        torch.cuda.empty_cache()
    tf.plan_save(args.out)
    print("saved %s in %.1f s" % (args.out, time.time() - t0))
    return 0


if __name__ == "__main__":
    sys.exit(main())
