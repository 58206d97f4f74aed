"""Leaf-size autotuner for the Gibbs chain (results cached in tuned.json).

For a workload key (kernel, input recipe, n) it times Gibbs iterations of the
mixed-precision chain and of the FP64 chain for every candidate leaf size B and
stores the per-B times and the B that is fastest for the mixed chain (the
benchmark's headline path; bench.py runs both paths with it).  bench.py and
users read the cached choice, so repeated runs (and profiled runs, whose
timings are distorted) use the same configuration.

Candidates: B in {32, 64, 128}.  B = 256 is out of reach of this library: a
leaf's FP64 Cholesky and triangular solves run in one CTA's shared memory,
which holds at most 227 KB, and a 256 x 256 FP64 leaf alone is 512 KB
(FIFA_LEAF_MAX = 128).  The rank cap only bounds memory (the clustered
workload's ranks stay at or below 7 of 32), and the kernels' tile shapes are
fixed at compile time, so neither is searched.

    python -m paper_2006_06537_gb300.autotune [--n 1048576] [--leaves 32 64 128]
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuned.json")


def workload_key(kind: str, n: int) -> str:
    return f"{kind}_n{n}"


def load(key: str):
    if not os.path.exists(CACHE):
        return None
    return json.load(open(CACHE)).get(key)


def store(key: str, entry: dict):
    data = json.load(open(CACHE)) if os.path.exists(CACHE) else {}
    data[key] = entry
    with open(CACHE, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)


def time_leaf(x, y, leaf, rho0, eps, cap, nugget, iters=5, warmup=3, prec=0, refine_tol=1e-10, overlap=1):
    import torch

    from . import fifa

    stream = torch.cuda.Stream()
    vy = float(np.var(y))
    with torch.cuda.stream(stream):
        ctx = fifa.Context(leaf_size=leaf, aca_tol=eps, rank_cap=cap, prec=prec, refine_max=8, refine_tol=refine_tol,
                           arena_bytes=40 << 30, stream=stream, overlap_proposal=overlap)
        xd = torch.tensor(x, device="cuda")
        yd = torch.tensor(y, device="cuda")
        pr = fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, math.log(rho0), 1.0, 0.2)
        ch = fifa.fifa_chain_create(ctx.h, xd, yd, len(x), fifa.fifa_hyper(0, vy, rho0, 0.5 * vy, nugget), pr, 0, 0)
        fifa.fifa_gibbs_step(ctx.h, ch, warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fifa.fifa_gibbs_step(ctx.h, ch, iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        fifa.fifa_destroy_chain(ctx.h, ch)
        ctx.close()
    return ms


def tune_clustered(n: int, leaves=(32, 64, 128), rho0=0.01, eps=1e-10, cap=32, nugget=1e-6, noise=0.05, overlap=1):
    from .build import build
    from .inputs import clustered

    build()
    x, y = clustered(n, 2, noise=noise)
    mixed = {str(b): time_leaf(x, y, b, rho0, eps, cap, nugget, prec=1, overlap=overlap) for b in leaves}
    fp64 = {str(b): time_leaf(x, y, b, rho0, eps, cap, nugget, prec=0, overlap=overlap) for b in leaves}
    best = int(min(mixed, key=mixed.get))
    entry = {"leaf": best, "ms_per_iter": mixed, "ms_per_iter_fp64": fp64, "rho0": rho0, "eps": eps, "cap": cap,
             "nugget": nugget, "refine_tol": 1e-10, "iters_timed": 5, "warmup": 3, "overlap_proposal": overlap}
    store(workload_key("clustered_se", n), entry)
    return entry


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--leaves", type=int, nargs="+", default=[32, 64, 128])
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="time chains with the proposal overlapped on a second stream (the benchmark's default)")
    a = ap.parse_args()
    print(json.dumps(tune_clustered(a.n, tuple(a.leaves), overlap=a.overlap)))
