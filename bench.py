"""Benchmark: FIFA-GP Gibbs iterations per second on one GB300.

Workload (the headline configuration): n = 2^20 sorted inputs drawn from a
mixture of 8 narrow uniforms (half-width 0.01, centres (2j+1)/16),
y = sin(2 pi x) + N(0, 0.05^2), squared-exponential kernel, rho_0 = 0.01,
ACA tolerance 1e-10, rank cap 32, IG(1,1) priors, random-walk Metropolis on
log rho.  One step = one full Gibbs iteration (M~ factor or its kept factor,
Algorithm 1 draw, sigma2, tau2, proposal assembly + FP64 factor + Metropolis).

paths      = the FP64 chain (M~ factored and solved directly every iteration,
             as Algorithm 1 is written) and the mixed chain (FP64 factor of M~
             kept between iterations and refreshed when rho moves or the
             solves slow down, applied in FP32 as the preconditioner of
             conjugate gradients with FP64 residuals), both from the same
             state and Philox streams, timed with CUDA events over K graph
             replays; `mixed_vs_fp64` compares the two chains step by step.
value      = iterations/s of the fastest valid path (mixed is valid when its
             M~ solves meet a 1e-8 true residual and its draws stay within
             1e-8 of the FP64 chain's).  Inputs and H-matrices exceed the
             129 MB L2 many times over: no flush is needed.
e2e        = the same path through the public API with host buffers: every
             step copies y from pinned host memory into the chain
             (fifa_chain_set_y), runs fifa_gibbs_step(1) with its trace row
             read back, and copies the draw f back to pinned host memory.
roofline   = the dominant operation (the FP64 factorization of C~), timed live
             with CUDA events on the library's stream: algorithmic flops from
             the actual per-node ranks (factor_work) over the FP64 FMA peak
             measured in the same run (fifa_probe_fp64_fma); secondary entries
             for the fused H-matrix product, the FP64 W^-1 sweep and the FP32
             preconditioner solve against the measured HBM bandwidth.
cpu_baseline = the CPU oracle (numpy, FP64) timed on this host on a bounded
             sample of the same workload (one iteration at n = 2^17, scaled).

--impl reference runs the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving leg runs 16 worker streams: with CUDA's default of 8 hardware
# work queues, streams share queues and unrelated kernels wait on each other
# (measured on the 48-request sample: 332 -> 375 iterations/s with 32 queues).
# The setting is read when the process creates its CUDA context.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_2006_06537_gb300.inputs import clustered  # noqa: E402

N_FULL = 1 << 20
RHO0 = 0.01
EPS = 1e-10
CAP = 32
NOISE = 0.05
METRIC = "Gibbs iters/s at n=2^20, mixed vs FP64 at 1e-8 rel err; p50/p99 latency"
UNIT = "iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=10,
                    help="untimed iterations before the timed ones (the chain leaves its start, and the mixed chain's kept M~ factor settles, within the first few)")
    ap.add_argument("--impl", default="fifa", choices=["fifa", "reference"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--leaf", type=int, default=0, help="leaf size (0 = the autotuner's cached choice)")
    ap.add_argument("--nugget", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="requests of the serving stream to run (0 = skip the serving leg)")
    ap.add_argument("--serve-slots", type=int, default=20)
    ap.add_argument("--serve-wide-min", type=int, default=1 << 13,
                    help="requests with n >= this run on the server's wide workers (CTA groups, fused sweeps)")
    ap.add_argument("--serve-wide-workers", type=int, default=4,
                    help="wide workers, each sizing its grouped launches to 1 / this of the GPU")
    ap.add_argument("--paths", default="fp64,mixed", help="chain precisions to time (comma list of fp64, mixed)")
    ap.add_argument("--additive-sweeps", type=int, default=10, help="0 = skip the d-block additive leg")
    ap.add_argument("--arena-gb", type=int, default=40, help="device arena of each chain context (GB)")
    ap.add_argument("--cap", type=int, default=CAP, help="ACA rank cap (profiling runs: a smaller arena)")
    ap.add_argument("--refine-tol", type=float, default=1e-10,
                    help="mixed path: conjugate gradients stop at ||b - M~ x|| <= tol ||b||")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="1: the proposal's assembly and factorization run on a second stream beside the draw "
                         "(fifa_opts.overlap_proposal; same results as 0)")
    ap.add_argument("--no-roofline", action="store_true", help="skip the roofline probe")
    ap.add_argument("--config-table", action="store_true",
                    help="time the other single-chain configurations (n = 2048 sine, FP64; n = 131072 Matern-5/2, "
                         "FP64 and mixed) and print one JSON object, instead of the bench line")
    ap.add_argument("--profile-factor", action="store_true",
                    help="only assemble C~(rho0) of the workload and factor it once (a target for ncu), then exit")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, world, device):
    """Element-wise max of per-rank timings over the process group (the
    slowest replica bounds the job); the values themselves when world == 1."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_rates(per_step_ms, e2e_s_per_step, world):
    """Whole-job iterations/s of `world` replicas, one chain each, from the
    slowest rank's device time per step (ms) and end-to-end time per step (s)."""
    return world * 1e3 / per_step_ms, world / e2e_s_per_step


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                    if out.returncode == 0 and out.stdout.strip():
                        self.rows.append([c.strip() for c in out.stdout.strip().split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)

        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------
REF_SAMPLE_N = 1 << 17  # oracle sample size: one iteration takes seconds on the host cores


def threads_used():
    try:
        from threadpoolctl import threadpool_info

        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and its core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                name = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform

    return {"model": name or platform.processor() or "unknown", "arch": platform.machine(), "cpus": os.cpu_count()}


def oracle_chain(n_sample: int, leaf: int, nugget: float, warmup: int, steps: int):
    """The oracle's Gibbs chain on the clustered recipe at n_sample points:
    set-up (assembly + factorization of C~(rho0)) untimed, `warmup` untimed
    iterations, then `steps` timed ones.  Returns (seconds per iteration, threads)."""
    from oracle import sampler

    x, y = clustered(n_sample, 2, noise=NOISE)
    opts = sampler.Opts(B=leaf, eps=EPS, cap=CAP, kind=0, nugget=nugget)
    prior = sampler.Prior(logrho_mu=math.log(RHO0))
    st = sampler.init_state(x, y, RHO0, opts)
    for _ in range(warmup):
        sampler.gibbs_step(st, x, y, prior, opts, seed=0, chain=0)
    t0 = time.perf_counter()
    for _ in range(steps):
        sampler.gibbs_step(st, x, y, prior, opts, seed=0, chain=0)
    return (time.perf_counter() - t0) / max(1, steps), threads_used()


def nlog2(n):
    return n * math.log2(n) ** 2


def cpu_baseline(n_full: int, leaf: int, nugget: float):
    """Oracle per-iteration time at a sample size, scaled to n_full by n log^2 n
    (the method's factorization cost, Sec. 4.1.1)."""
    n_s = min(n_full, REF_SAMPLE_N)
    dt, thr = oracle_chain(n_s, leaf, nugget, 0, 1)
    scale = nlog2(n_full) / nlog2(n_s)
    return {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": thr, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"1 oracle Gibbs iteration at n={n_s} of the same clustered recipe ({dt:.2f} s), "
                      f"scaled to n={n_full} by n log2(n)^2 (x{scale:.2f})"}


def reference_arm(args):
    """The oracle as the reference arm: every step one oracle Gibbs iteration on
    the clustered recipe at n = 2^17 (a bounded sample of the 2^20 workload),
    measured; the line's n is the sample's, and the n log^2 n extrapolation to
    the workload size is reported in its own field."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from paper_2006_06537_gb300 import autotune

    entry = autotune.load(autotune.workload_key("clustered_se", args.n))
    leaf = args.leaf or (entry["leaf"] if entry else 32)
    n_s = min(args.n, REF_SAMPLE_N)
    per, thr = oracle_chain(n_s, leaf, args.nugget, args.warmup, args.steps)
    v = 1.0 / per
    scale = nlog2(args.n) / nlog2(n_s)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"clustered SE n={n_s} (sample of the n={args.n} workload), 8 clusters, "
                                   f"rho0={RHO0}, sigma={NOISE}", "n": n_s, "workload_n": args.n,
                       "leaf": leaf, "aca_tol": EPS, "rank_cap": CAP, "nugget": args.nugget, "precision": "fp64"},
            "extrapolated_to_workload_n": {"n": args.n, "value": v / scale, "unit": UNIT,
                                           "scaling": "n log2(n)^2 (the factorization's cost)", "factor": scale},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{args.steps} oracle Gibbs iterations at n={n_s} after {args.warmup} "
                                       f"untimed ones (measured, not scaled)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def gpu_arm(args):
    import torch

    from paper_2006_06537_gb300 import build
    from paper_2006_06537_gb300 import fifa

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    build.build()
    n = args.n
    x, y = clustered(n, 2 + rank, noise=NOISE)  # replicas: each rank its own chain and data
    stream = torch.cuda.Stream()
    if args.profile_factor:
        profile_factor(args, fifa, torch, stream, x)
        return
    if args.config_table:
        config_table(args, fifa, torch, stream)
        return
    prior_mu = math.log(RHO0)
    vy = float(np.var(y))

    def make(prec, leaf, refine_max=8, arena_gb=args.arena_gb):
        with torch.cuda.stream(stream):
            ctx = fifa.Context(leaf_size=leaf, aca_tol=EPS, rank_cap=args.cap, prec=prec, refine_max=refine_max,
                               refine_tol=args.refine_tol, arena_bytes=int(arena_gb) << 30, stream=stream,
                               overlap_proposal=args.overlap)
            xd = torch.tensor(x, device="cuda")
            yd = torch.tensor(y, device="cuda")
            pr = fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, prior_mu, 1.0, 0.2)
            ch = fifa.fifa_chain_create(ctx.h, xd, yd, n, fifa.fifa_hyper(0, vy, RHO0, 0.5 * vy, args.nugget), pr,
                                        0, rank)
        return ctx, ch

    def time_chain(ctx, ch, steps, warmup):
        wtr = np.zeros((max(warmup, 1), fifa.FIFA_TRACE_FIELDS))
        fifa.fifa_gibbs_step(ctx.h, ch, warmup, wtr[:warmup] if warmup else None)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        trace = np.zeros((steps, fifa.FIFA_TRACE_FIELDS))
        fifa.fifa_gibbs_step(ctx.h, ch, steps, trace)
        e1.record(stream)
        torch.cuda.synchronize()
        f = torch.empty(n, dtype=torch.float64, device="cuda")
        mean = torch.empty_like(f)
        fifa.fifa_chain_get(ctx.h, ch, f, mean)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), np.vstack([wtr[:warmup], trace]), f.cpu().numpy(), mean.cpu().numpy()

    def close(ctx, ch):
        fifa.fifa_destroy_chain(ctx.h, ch)
        ctx.close()
        torch.cuda.synchronize()

    # leaf size: the autotuner's cached choice for this workload (tuned.json),
    # measured by `python -m paper_2006_06537_gb300.autotune`; tuned here (and
    # cached) only if no entry exists yet
    from paper_2006_06537_gb300 import autotune

    if args.leaf:
        leaf, tune = args.leaf, {}
    else:
        entry = autotune.load(autotune.workload_key("clustered_se", n))
        if entry is None and rank == 0:
            entry = autotune.tune_clustered(n, nugget=args.nugget)
        leaf, tune = (entry["leaf"], entry["ms_per_iter"]) if entry else (32, {})

    results = {}
    wanted = [p.strip() for p in args.paths.split(",") if p.strip()]
    for name, prec in (("fp64", fifa.FIFA_FP64), ("mixed", fifa.FIFA_MIXED)):
        if name not in wanted:
            continue
        ctx, ch = make(prec, leaf)
        try:
            clocks = ClockSampler(local)
            clocks.start()
            ms, trace, f_end, m_end = time_chain(ctx, ch, args.steps, args.warmup)
            clk = clocks.stop()
            ok, why = True, ""
        except fifa.FifaError as exc:
            ms, trace, f_end, m_end, clk, ok, why = float("nan"), None, None, None, None, False, str(exc)
        timed = trace[args.warmup:] if trace is not None else None
        res = float(np.nanmax(timed[:, 9])) if timed is not None else float("nan")
        if ok and prec == fifa.FIFA_MIXED and not (res <= 1e-8):
            ok, why = False, f"M~ solve residual {res:.2e} above 1e-8"
        results[name] = dict(ms=ms / args.steps if ok else float("nan"), ok=ok, why=why, clocks=clk, trace=trace,
                             kernels=fifa.fifa_chain_kernel_nodes(ch), refine_res=res, f=f_end, mean=m_end)
        close(ctx, ch)
    # the mixed chain against the FP64 chain (same state, data and Philox streams)
    cmp = None
    if "fp64" in results and "mixed" in results and results["fp64"]["ok"] and results["mixed"]["ok"]:
        t6, tm = results["fp64"]["trace"], results["mixed"]["trace"]
        same = bool(np.array_equal(t6[:, 4], tm[:, 4]))

        def rmax(a, b):
            return float(np.max(np.abs(a - b) / np.abs(b)))

        rf = float(np.linalg.norm(results["mixed"]["f"] - results["fp64"]["f"]) / np.linalg.norm(results["fp64"]["f"]))
        rm = float(np.linalg.norm(results["mixed"]["mean"] - results["fp64"]["mean"]) /
                   np.linalg.norm(results["fp64"]["mean"]))
        fin = np.isfinite(t6[:, 5]) & np.isfinite(tm[:, 5])
        cmp = {"steps_compared": int(len(t6)), "accept_decisions_equal": same,
               "sigma2_max_rel": rmax(tm[:, 1], t6[:, 1]), "tau2_max_rel": rmax(tm[:, 2], t6[:, 2]),
               "log_alpha_max_abs": float(np.max(np.abs(tm[fin, 5] - t6[fin, 5]))) if fin.any() else None,
               "f_final_rel": rf, "mean_final_rel": rm,
               "mixed_refactor_fraction": float(tm[args.warmup:, 11].mean()),
               "mixed_cg_iters_mean": float(tm[args.warmup:, 12].mean()),
               "mixed_cg_iters_max": int(tm[args.warmup:, 12].max())}
        if same and not (rf <= 1e-8 and rm <= 1e-8):
            results["mixed"]["ok"] = False
            results["mixed"]["why"] = f"draw / mean differ from the FP64 chain by {rf:.1e} / {rm:.1e} (> 1e-8)"
    valid = [k for k in results if results[k]["ok"]]
    head = min(valid, key=lambda k: results[k]["ms"])
    per_head = results[head]["ms"]
    hprec = fifa.FIFA_FP64 if head == "fp64" else fifa.FIFA_MIXED

    # end-to-end through the public API with pinned host buffers: each step
    # streams y into the chain, runs one iteration, reads f and the trace row back
    ctx, ch = make(hprec, leaf)
    yh = torch.tensor(y).pin_memory()
    fh = torch.empty(n, dtype=torch.float64).pin_memory()
    fd = torch.empty(n, dtype=torch.float64, device="cuda")
    row = np.zeros((1, fifa.FIFA_TRACE_FIELDS))
    fifa.fifa_gibbs_step(ctx.h, ch, args.warmup, None)
    e2e_steps = args.steps  # the same iterations of the chain as the device-timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            fifa.fifa_chain_set_y(ctx.h, ch, yh)
            fifa.fifa_gibbs_step(ctx.h, ch, 1, row)
            fifa.fifa_chain_get(ctx.h, ch, fd, None)
            fh.copy_(fd, non_blocking=True)
        stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    close(ctx, ch)
    roof = None
    if not args.no_roofline:
        with torch.cuda.stream(stream):
            pctx = fifa.Context(leaf_size=leaf, aca_tol=EPS, rank_cap=CAP, prec=fifa.FIFA_FP64,
                                arena_bytes=min(24, args.arena_gb) << 30, stream=stream)
            mctx = fifa.Context(leaf_size=leaf, aca_tol=EPS, rank_cap=CAP, prec=fifa.FIFA_MIXED, refine_max=8,
                                refine_tol=1e-12, arena_bytes=min(24, args.arena_gb) << 30, stream=stream)
            xd = torch.tensor(x, device="cuda")
        roof = roofline_probe(pctx, mctx, fifa, torch, stream, xd, n, leaf, args.nugget)
        pctx.close()
        mctx.close()

    # serving (continuous batching, p50/p99) and the d-block additive model:
    # measured after the headline, outside its timed region
    serving = additive = None
    if rank == 0 and args.serve_requests > 0:
        serving = serving_leg(fifa, args.serve_requests, args.serve_slots, fifa.FIFA_MIXED, 32,
                              wide_min_n=args.serve_wide_min, wide_workers=args.serve_wide_workers,
                              overlap=args.overlap)
    if rank == 0 and args.additive_sweeps > 0:
        additive = additive_leg(fifa, torch, args.additive_sweeps, 32)

    per_head, e2e_s = max_over_ranks([per_head, e2e_s], world, "cuda")
    value, e2e_value = job_rates(per_head, e2e_s, world)
    if rank != 0:
        return
    try:
        kl = kl_report(fifa, torch, leaf, args.nugget)
    except Exception as exc:  # a report, not part of the timed path
        kl = {"kl": None, "note": f"failed: {exc}"}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_baseline(n, leaf, args.nugget)
        except Exception as exc:  # the baseline must not hide the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}
    tr = results[head]["trace"][args.warmup:]
    paths = {k: {"value": (1e3 / v["ms"]) if v["ok"] else None, "ms_per_step": v["ms"] if v["ok"] else None,
                 "valid": v["ok"], "note": v["why"], "refine_residual": v["refine_res"],
                 "kernels_per_step": v["kernels"]} for k, v in results.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_head, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": f"clustered SE n={n}, 8 clusters, rho0={RHO0}, sigma={NOISE}", "n": n, "leaf": leaf,
                   "leaf_autotune_ms": tune, "aca_tol": EPS, "rank_cap": CAP, "nugget": args.nugget,
                   "precision": head, "l2": "inputs and H-matrices (>> 129 MB L2) resident; no flush needed",
                   "overlap_proposal": args.overlap, "parallelism": f"replicas x{world}"},
        "paths": paths,
        "mixed_vs_fp64": cmp,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n + 8 * fifa.FIFA_TRACE_FIELDS,
                "step": "y pinned host -> chain (fifa_chain_set_y), fifa_gibbs_step(1) + trace row, f -> pinned host"},
        "chain": {"rho": float(tr[-1, 3]), "sigma2": float(tr[-1, 1]), "tau2": float(tr[-1, 2]),
                  "accept_rate": float(tr[:, 4].mean())},
        "roofline": roof,
        "kl": kl,
        "serving": serving,
        "additive": additive,
        "cpu_baseline": cpu,
        "gpu_launches": int(results[head]["kernels"]) * args.steps,
        "clocks": results[head]["clocks"],
    }
    print(json.dumps(line))


def profile_factor(args, fifa, torch, stream, x):
    """One assembly and one FP64 factorization of C~(rho0) of the workload, with
    the leaf size the bench uses; nothing else runs (the ncu traffic capture of
    the factorization kernels)."""
    from paper_2006_06537_gb300 import autotune

    entry = autotune.load(autotune.workload_key("clustered_se", args.n))
    leaf = args.leaf or (entry["leaf"] if entry else 32)
    with torch.cuda.stream(stream):
        ctx = fifa.Context(leaf_size=leaf, aca_tol=EPS, rank_cap=args.cap, arena_bytes=int(args.arena_gb) << 30,
                           stream=stream)
        xd = torch.tensor(x, device="cuda")
        H = fifa.fifa_assemble(ctx.h, xd, args.n, fifa.fifa_hyper(0, 1.0, RHO0, 1.0, args.nugget))
        F = fifa.fifa_factor(ctx.h, H)
        ld, code = fifa.fifa_logdet(ctx.h, F)
    torch.cuda.synchronize()
    print(json.dumps({"profile_factor": {"n": args.n, "leaf": leaf, "logdet": ld, "status": int(code)}}))
    fifa.fifa_destroy_fact(ctx.h, F)
    fifa.fifa_destroy_hmat(ctx.h, H)
    ctx.close()


def config_table(args, fifa, torch, stream):
    """Iterations/s of the single-chain configurations other than the headline:
    n = 2048 uniform inputs, y = sin(2 pi x) + N(0, 0.1^2), SE, leaf 64, ACA
    tolerance 1e-12, FP64, 200 iterations; n = 131072 uniform inputs, y a
    Matern-5/2 draw (rho = 0.05) + N(0, 0.2^2), Matern-5/2 kernel, leaf 128,
    tolerance 1e-10, FP64 and mixed, `args.steps` iterations.  CUDA events
    around the iterations after `args.warmup` untimed ones."""
    from paper_2006_06537_gb300.inputs import matern_draw, uniform_sine

    def run(x, y, kind, rho, leaf, eps, prec, steps):
        n = len(x)
        vy = float(np.var(y))
        with torch.cuda.stream(stream):
            ctx = fifa.Context(leaf_size=leaf, aca_tol=eps, rank_cap=CAP, prec=prec, refine_max=8,
                               refine_tol=args.refine_tol, arena_bytes=8 << 30, stream=stream,
                               overlap_proposal=args.overlap)
            ch = fifa.fifa_chain_create(ctx.h, torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"), n,
                                        fifa.fifa_hyper(kind, vy, rho, 0.5 * vy, 1e-6),
                                        fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, math.log(rho), 1.0, 0.2), 0, 0)
            if args.warmup:
                fifa.fifa_gibbs_step(ctx.h, ch, args.warmup, None)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            tr = np.zeros((steps, fifa.FIFA_TRACE_FIELDS))
            fifa.fifa_gibbs_step(ctx.h, ch, steps, tr)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        fifa.fifa_destroy_chain(ctx.h, ch)
        ctx.close()
        return {"ms_per_iter": ms, "iters_per_s": 1e3 / ms, "iters_timed": steps,
                "accept_rate": float(tr[:, 4].mean())}

    out = {}
    x, y = uniform_sine(2048, 0)
    out["sine_se_n2048_leaf64_fp64"] = run(x, y, 0, 0.1, 64, 1e-12, fifa.FIFA_FP64, 200)
    x, y, _ = matern_draw(131072, 1, rho=0.05, var=1.0, noise=0.2)
    for name, prec in (("fp64", fifa.FIFA_FP64), ("mixed", fifa.FIFA_MIXED)):
        out[f"matern52_n131072_leaf128_{name}"] = run(x, y, 1, 0.05, 128, 1e-10, prec, args.steps)
    print(json.dumps({"config_table": out}))


def dense_ctilde(ex, n):
    """C~ written out densely from fifa_hmat_export (leaves column-major,
    level-l bases: U on the left child's rows, V on the right child's)."""
    L = ex["L"]
    nodes = [(0, n)]
    Ct = np.zeros((n, n))
    for lvl in range(L):
        for i, (s, e) in enumerate(nodes):
            h = s + (e - s) // 2
            r = int(ex["ranks"][(1 << lvl) - 1 + i])
            U = ex["bases"][lvl, :r, s:h].T
            V = ex["bases"][lvl, :r, h:e].T
            Ct[s:h, h:e] = U @ V.T
            Ct[h:e, s:h] = V @ U.T
        nodes = [b for s, e in nodes for b in ((s, s + (e - s) // 2), (s + (e - s) // 2, e))]
    for i, (s, e) in enumerate(nodes):
        Ct[s:e, s:e] = ex["leaves"][i, :e - s, :e - s].T
    return Ct


def kl_report(fifa, torch, leaf, nugget, n_kl=2048):
    """KL(P || Q) of Sec. 4.1.3 (Theorem 4.1) for the library's C~ on the
    workload's recipe at n_kl points: P the exact posterior of f for
    K = tau2 (C + nugget I), Q the law Algorithm 1 samples for K~ = tau2 C~
    (covariance K~ M~^-1, M~ = K~ / sigma2 + I, mean that covariance times
    y / sigma2).  C~ is assembled on the GPU and exported; both Gaussians are
    formed densely in FP64 here."""
    x, y = clustered(n_kl, 2, noise=NOISE)
    tau2, sigma2 = float(np.var(y)), NOISE * NOISE
    ctx = fifa.Context(leaf_size=leaf, aca_tol=EPS, rank_cap=CAP, arena_bytes=1 << 28)
    H = fifa.fifa_assemble(ctx.h, torch.tensor(x, device="cuda"), n_kl, fifa.fifa_hyper(0, 1.0, RHO0, 1.0, nugget))
    ex = fifa.fifa_hmat_export(ctx.h, H)
    ctx.close()
    out = kl_terms(x, y, dense_ctilde(ex, n_kl), tau2, sigma2, RHO0, nugget)
    out.update({"n": n_kl, "leaf": leaf, "aca_tol": EPS,
                "workload": f"clustered SE n={n_kl}, 8 clusters, rho={RHO0}, tau2=var(y), sigma2={sigma2:g}, "
                            f"nugget={nugget:g}",
                "ranks_max": int(np.max(ex["ranks"])),
                "note": "C~ from fifa_assemble + fifa_hmat_export; P and Q formed densely in numpy FP64"})
    return out


def kl_terms(x, y, Ct, tau2, sigma2, rho, nugget):
    """KL(P || Q) and its parts for the SE kernel: P the exact posterior for
    K = tau2 (C + nugget I), Q the one for K~ = tau2 C~ (Ct dense)."""
    n = len(x)
    dx = x[:, None] - x[None, :]
    eye = np.eye(n)
    K = tau2 * (np.exp(-dx * dx / (2 * rho * rho)) + nugget * eye)
    Kt = tau2 * Ct

    def post(Km):
        S = Km @ np.linalg.inv(Km / sigma2 + eye)
        S = 0.5 * (S + S.T)
        return S @ y / sigma2, S

    mp, Sp = post(K)
    mq, Sq = post(Kt)
    ldq, ldp = np.linalg.slogdet(Sq)[1], np.linalg.slogdet(Sp)[1]
    tr = float(np.trace(np.linalg.solve(Sq, Sp))) - n
    dm = mq - mp
    quad = float(dm @ np.linalg.solve(Sq, dm))
    return {"kl": 0.5 * (ldq - ldp + tr + quad),
            "parts": {"logdet": 0.5 * (ldq - ldp), "trace": 0.5 * tr, "quad": 0.5 * quad},
            "e_max": float(np.abs(Kt - K).max())}


def serving_leg(fifa, count, slots, prec, leaf, iters=100, ndraws=20, rate=200.0, budget=120 << 30,
                wide_min_n=1 << 14, wide_workers=4, overlap=0):
    """The serving workload: the first `count` requests of a Poisson stream at
    `rate` req/s, n log-uniform in [2^10, 2^18], SE or Matern-5/2 per request,
    each `iters` Gibbs iterations returning the posterior mean and `ndraws`
    draws, admitted under an HBM budget.  Requests are submitted at their
    arrival times; latency = completion - submission on the server's clock."""
    from paper_2006_06537_gb300.inputs import request_data, serving_requests

    reqs = serving_requests(count, rate)
    data = [request_data(r) for r in reqs]
    opts = fifa.fifa_opts(leaf, EPS, CAP, prec, 1e-12, 8, 1, 0, 0, overlap)
    srv = fifa.fifa_server_create(opts, budget, slots, wide_min_n, wide_workers)
    ids = [None] * count
    res = [None] * count
    done = threading.Event()

    def waiter():
        for i in range(count):
            while ids[i] is None:
                time.sleep(0.0002)
            if ids[i] < 0:  # submission failed: nothing to wait for
                res[i] = (-1, 0.0, 0.0, 0.0)
                continue
            n = reqs[i]["n"]
            mean, draws = np.empty(n), np.empty((ndraws, n))
            st, r = fifa.fifa_server_wait(srv, ids[i], mean, draws, allow=tuple(range(16)))
            res[i] = (st, r.t_submit, r.t_start, r.t_done)
        done.set()

    th = threading.Thread(target=waiter)
    th.start()
    pr = fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, math.log(0.1), 1.0, 0.2)
    t0 = time.perf_counter()
    try:
        for i, r in enumerate(reqs):
            wait = r["t"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            x, y = data[i]
            vy = float(np.var(y))
            try:
                ids[i] = fifa.fifa_server_submit(srv, x, y, fifa.fifa_hyper(r["kind"], vy, 0.1, 0.5 * vy, 1e-6), pr,
                                                 0, r["id"], iters, iters // 2, ndraws)
            except fifa.FifaError:
                ids[i] = -1
    finally:
        for i in range(count):
            if ids[i] is None:
                ids[i] = -1
        th.join()
    stats = fifa.fifa_server_stats(srv)
    fifa.fifa_server_destroy(srv)
    ok = [r for r in res if r[0] == 0]
    if not ok:
        return {"requests": count, "completed": 0, "statuses": sorted({int(r[0]) for r in res})}
    lat = np.array([r[3] - r[1] for r in ok])
    span = max(r[3] for r in ok) - min(r[1] for r in ok)
    sizes = np.array([r["n"] for r in reqs])
    return {
        "workload": f"first {count} requests of a Poisson stream at {rate:g} req/s, n log-uniform in [2^10, 2^18], "
                    f"SE or Matern-5/2, {iters} iterations + posterior mean + {ndraws} draws each",
        "requests": count, "completed": len(ok), "offered_req_per_s": rate, "slots": slots,
        "wide_min_n": wide_min_n, "wide_workers": wide_workers, "overlap_proposal": overlap,
        "hbm_budget_gb": budget / 2**30, "precision": "fp64" if prec == fifa.FIFA_FP64 else "mixed",
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(lat.mean()), "iters_per_s": len(ok) * iters / span,
        "points_iters_per_s": float(sizes[[r[0] == 0 for r in res]].sum()) * iters / span,
        "served_req_per_s": len(ok) / span, "span_s": span, "peak_in_flight": stats.peak_in_flight,
        "peak_hbm_gb": stats.peak_bytes / 2**30,
    }


def additive_leg(fifa, torch, sweeps, leaf, n=65536, d=4):
    """The d-block additive workload: n points uniform in [0,1]^d,
    y = sum_k sin(2 pi (k+1) x_k) + N(0, 0.1^2), one SE block per coordinate;
    block-Gibbs sweeps per second on each precision (mixed valid only if every
    M~ solve refined to 1e-8)."""
    from paper_2006_06537_gb300.inputs import additive4

    X, y = additive4(n)
    vy = float(np.var(y))
    out = {"workload": f"additive d={d}, n={n}, SE blocks, sigma=0.1", "n": n, "d": d, "leaf": leaf}
    for name, prec in (("fp64", fifa.FIFA_FP64), ("mixed", fifa.FIFA_MIXED)):
        stream = torch.cuda.Stream()
        ctx = fifa.Context(leaf_size=leaf, aca_tol=EPS, rank_cap=CAP, prec=prec, refine_max=8, refine_tol=1e-12,
                           arena_bytes=8 << 30, stream=stream)
        Xd = torch.tensor(np.ascontiguousarray(X[:, :d].T), device="cuda")
        yd = torch.tensor(y, device="cuda")
        torch.cuda.synchronize()
        pr = fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, math.log(0.1), 1.0, 0.2)
        m = fifa.fifa_additive_create(ctx.h, Xd, yd, n, d, fifa.fifa_hyper(0, vy / d, 0.1, 0.5 * vy, 1e-6), pr, 0)
        tr = np.zeros((sweeps, fifa.fifa_additive_trace_fields(d)))
        st = fifa.fifa_additive_sweep(ctx.h, m, 3, None, allow=tuple(range(16)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        if st == 0:
            st = fifa.fifa_additive_sweep(ctx.h, m, sweeps, tr, allow=tuple(range(16)))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / sweeps
        res = float(tr[:, 4].max())
        ok = st == 0 and (prec == fifa.FIFA_FP64 or res <= 1e-8)
        out[name] = {"sweeps_per_s": 1e3 / ms if ok else None, "ms_per_sweep": ms if ok else None, "valid": ok,
                     "refine_residual": res, "status": int(st), "kernels_per_sweep": fifa.fifa_additive_kernel_nodes(m),
                     "sigma2": float(tr[-1, 1]), "rho": [float(v) for v in tr[-1, 5 + d:5 + 2 * d]]}
        fifa.fifa_destroy_additive(ctx.h, m)
        ctx.close()
    return out


def factor_work(n, leaf, ranks):
    """Algorithmic FP64 flops of one HODLR factorization (per level too), from
    the per-node ranks (heap order): leaf m^3/3 + m^2 C_anc, levels 4 r^2 m
    (CholeskyQR2) + 4 r C_anc m (ancestor update)."""
    L = 0
    while (n + (1 << L) - 1) >> L > leaf:
        L += 1
    b = [[0, n]]
    for _ in range(L):
        nxt = []
        for s_, e_ in b:
            h_ = s_ + (e_ - s_) // 2
            nxt += [[s_, h_], [h_, e_]]
        b = nxt if nxt else b
    leaves_m = np.array([e_ - s_ for s_, e_ in b], dtype=np.float64)
    nl = len(leaves_m)
    canc_leaf = np.zeros(nl)
    for l in range(L):
        r_l = ranks[(1 << l) - 1:(1 << (l + 1)) - 1]
        canc_leaf += np.repeat(r_l, nl >> l)
    flops = float(np.sum(leaves_m ** 3) / 3.0 + np.sum(leaves_m ** 2 * canc_leaf))
    per_level = [flops]  # leaves first, then levels L-1 .. 0
    lv = []
    for l in range(L):
        r_l = ranks[(1 << l) - 1:(1 << (l + 1)) - 1].astype(np.float64)
        m = n / (1 << l)
        canc = np.zeros_like(r_l)
        for j in range(l):
            canc += np.repeat(ranks[(1 << j) - 1:(1 << (j + 1)) - 1], 1 << (l - j))
        f = float(np.sum(4.0 * r_l * r_l * m + 4.0 * r_l * canc * m))
        lv.append(f)
        flops += f
    per_level += lv[::-1]
    return flops, L, per_level, leaves_m


def apply_work(n, leaves_m, ranks, L, nrhs=2):
    """Algorithmic bytes of the application kernels for nrhs right-hand sides:
    rank_rows = sum over levels of the level's mean rank times n (basis entries
    one pass reads).
      FP64 W^-1 sweep: the leaf factors' lower triangles and the bases once
        (8 bytes), v read and written once.
      FP32 preconditioner solve W32^-T W32^-1: both triangles of the leaf
        factors and the bases twice (4 bytes), v read and written once (FP64).
      FP64 H-matrix product: the dense leaves and the bases once (8 bytes), x
        read and y written once; flops 2 (m + 2 rank_rows / n) n nrhs."""
    rank_rows = n * float(sum(ranks[(1 << l) - 1:(1 << (l + 1)) - 1].mean() for l in range(L)))
    vec = 2 * 8.0 * n * nrhs
    sweep = 8.0 * (np.sum(leaves_m ** 2) / 2.0 + rank_rows) + vec
    precond = 4.0 * (np.sum(leaves_m ** 2) + 2 * rank_rows) + vec
    mv_bytes = 8.0 * (np.sum(leaves_m ** 2) + rank_rows) + vec
    mv_flops = 2.0 * (np.sum(leaves_m ** 2) + 2 * rank_rows) * nrhs
    return float(sweep), float(precond), float(mv_bytes), float(mv_flops)


def sweep_flops(n, leaves_m, ranks, L, nrhs=2):
    """FP64 flops of one W^-1 sweep: the leaf triangular solves (m^2 each) and
    per level the projection and the update (2 r flops per row each)."""
    rank_rows = n * float(sum(ranks[(1 << l) - 1:(1 << (l + 1)) - 1].mean() for l in range(L)))
    return float((np.sum(leaves_m ** 2) + 4 * rank_rows) * nrhs)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, summed over the 44
# launches of one FP64 factorization of C~(rho0) of this workload at n = 2^20,
# leaf 32: 6.44 GB read + 4.07 GB written) from one ncu capture of
# `bench.py --profile-factor` on the current factorization kernels.
FACTOR_TRAFFIC_BYTES = 10.51e9
FACTOR_TRAFFIC_CONFIG = (1 << 20, 32)  # (n, leaf) it was captured at


def roofline_probe(ctx, mctx, fifa, torch, stream, xd, n, leaf, nugget):
    """The FP64 factorization of C~(rho0) of this workload (the dominant
    operation) and the application kernels, each timed alone with CUDA events
    on the library stream (ctx an FP64 context; mctx a mixed-precision one for
    the preconditioner and the mixed solve); peaks: the FP64 FMA probe of this
    run and the measured HBM copy bandwidth."""
    hbm, src = peaks()
    peak_fp64, probe_ms = fifa.fifa_probe_fp64_fma(ctx.h, 20000)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()  # warm-up
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        H = fifa.fifa_assemble(ctx.h, xd, n, fifa.fifa_hyper(0, 1.0, RHO0, 1.0, nugget))
        ranks = fifa.fifa_hmat_export(ctx.h, H, bases=False, leaves=False)["ranks"].astype(np.float64)
        ms = 0.0
        F = fifa.fifa_factor(ctx.h, H)  # warm-up
        torch.cuda.synchronize()
        fifa.fifa_destroy_fact(ctx.h, F)
        reps = 3
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record(stream)
            F = fifa.fifa_factor(ctx.h, H)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1) / reps
            fifa.fifa_destroy_fact(ctx.h, F)
        F = fifa.fifa_factor(ctx.h, H)
        v = torch.randn(2, n, dtype=torch.float64, device="cuda")
        w = torch.empty_like(v)
        ms_sw = timed(lambda: fifa.fifa_apply_W(ctx.h, F, 0, 1, v, v, 2), 5)
        ms_mv = timed(lambda: fifa.fifa_matvec(ctx.h, H, v, w, 2), 5)
        fifa.fifa_destroy_fact(ctx.h, F)
        fifa.fifa_destroy_hmat(ctx.h, H)
        # the mixed context: M~ = s C~ + I at the chain's s (tau2 / sigma2 ~
        # 0.5 / 0.05^2) with its kept factor: the FP32 preconditioner solve and
        # a whole mixed solve
        Hm = fifa.fifa_assemble(mctx.h, xd, n, fifa.fifa_hyper(0, 1.0, RHO0, 1.0, nugget))
        M = fifa.fifa_shift_scale(mctx.h, Hm, 200.0)
        FM = fifa.fifa_factor(mctx.h, M)
        ms_pc = timed(lambda: fifa.fifa_apply_precond(mctx.h, FM, v, w, 2), 5)
        ms_solve = timed(lambda: fifa.fifa_solve(mctx.h, FM, v, w, 2), 3)
        fifa.fifa_destroy_fact(mctx.h, FM)
        fifa.fifa_destroy_hmat(mctx.h, M)
        fifa.fifa_destroy_hmat(mctx.h, Hm)
    flops, L, per_level, leaves_m = factor_work(n, leaf, ranks)
    sweep_b, pc_b, mv_b, mv_f = apply_work(n, leaves_m, ranks, L)
    achieved = flops / (ms * 1e-3) / 1e12

    def hbm_entry(op, ms_, bytes_):
        a = bytes_ / (ms_ * 1e-3) / 1e9
        return {"bound": "hbm", "op": op, "ms": ms_, "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                "bytes": bytes_, "peak_source": src}

    sw = hbm_entry("fused W^-1 sweep, FP64, 2 right-hand sides", ms_sw, sweep_b)
    sw_f = sweep_flops(n, leaves_m, ranks, L)
    sw["fp64"] = {"flops": sw_f, "achieved": sw_f / (ms_sw * 1e-3) / 1e12, "peak": peak_fp64, "unit": "TFLOP/s",
                  "frac": sw_f / (ms_sw * 1e-3) / 1e12 / peak_fp64}
    mv = hbm_entry("fused H-matrix product C~ x, FP64, 2 right-hand sides", ms_mv, mv_b)
    mv["fp64"] = {"flops": mv_f, "achieved": mv_f / (ms_mv * 1e-3) / 1e12, "peak": peak_fp64, "unit": "TFLOP/s",
                  "frac": mv_f / (ms_mv * 1e-3) / 1e12 / peak_fp64}
    return {"bound": "alu", "op": "FP64 HODLR factorization of C~ (leaf Cholesky + TRSM, per-level CholeskyQR2, "
                                  "capacitance, ancestor update)",
            "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s", "frac": achieved / peak_fp64,
            "traffic": FACTOR_TRAFFIC_BYTES if (n, leaf) == FACTOR_TRAFFIC_CONFIG else None, "ms": ms, "flops": flops, "rank_mean": float(ranks.mean()), "levels": L,
            "gflops_leaves_then_levels_deep_to_top": [round(f / 1e9, 4) for f in per_level],
            "rank_mean_per_level": [round(float(ranks[(1 << l) - 1:(1 << (l + 1)) - 1].mean()), 2) for l in range(L)],
            "peak_source": f"FP64 FMA throughput measured in this run (fifa_probe_fp64_fma, {probe_ms:.1f} ms)",
            "sweep": sw,
            "matvec": mv,
            "precond_fp32": hbm_entry("FP32 preconditioner solve W32^-T W32^-1 (one fused launch), 2 right-hand sides",
                                      ms_pc, pc_b),
            "mixed_solve_ms": ms_solve}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
