"""Benchmark: FP64 recursive Householder QR (QR-EG with TSQR base case) on
one GB300, reported as TFLOP/s at the algorithmic count 2mn^2 - 2n^3/3.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--layout panel|full] [--impl gbqr|reference]

A step is one full factorization of the workload's matrix (every step of the
path: non-finite scan, TSQR base cases, update and T-assembly GEMMs, the
right-looking top-level updates).  Each step first restores A from a pristine
device copy (included in the step; it is < 0.1 % of it).  The inputs are
larger than L2, so no flush is needed between steps.  Under torchrun every
rank factors its own matrix (independent replicas, no collective on the data
path); the reported value is the flops of all ranks over the slowest rank's
time.

The timed region runs with launch tracing off.  The roofline of the dominant
kernel (the FP64 GEMM family) comes from a separate traced pass of the same
factorization with the look-ahead off, so that every launch runs alone and
its event-bracketed duration is its own (with look-ahead the side stream's
panel shares the SMs and stretches the GEMMs it overlaps).

--impl reference times the CPU oracle (unblocked Householder QR, the build
whose column loops run on every host core) on a bounded, stratified sample
of the same workload: in each of 8 equal ranges of the n Householder steps a
few steps are timed on the trailing matrix of the range's midpoint, and the
full factorization's time is estimated as the sum over ranges of the
range's flops at that range's measured rate.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

FP64_NOMINAL_TFLOPS = 1.25          # GB300 FP64 (CUDA and tensor cores), nominal
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# Derived FP64 peak: 152 SMs x 4 FP64 flop/clk/SM (2 FMA) x 2.070 GHz.
FP64_FLOP_PER_CLK_PER_SM = 4.0
FP64_PEAK_TFLOPS = SM_COUNT * FP64_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
# DRAM bytes (read + write) of dgemm launches over their algorithmic bytes
# 8 (MK + KN + 2MN), from an ncu capture of every dgemm launch of the
# quarter-size graded 4096 x 4096 factorization with the same panel width,
# cutoff and engine (one-pass metrics); the roofline's traffic is that ratio
# times the measured pass's algorithmic bytes per launch, null for any other
# configuration.
DGEMM_TRAFFIC_RATIO = {
    # (workload, panel_nb, cutoff_b, engine): ratio
    ("graded_8192x8192", 128, 16, "dfma"): 0.780,
    ("graded_4096x4096", 128, 16, "dfma"): 0.780,
}
DGEMM_TRAFFIC_SOURCE = "ncu: all dgemm launches of graded 4096x4096 (nb 128, b 16, DFMA), dram read+write / algorithmic"
METRIC = "QR TFLOP/s (2mn^2-2n^3/3) vs peak; LS solves/s, p99 ms: mixed vs FP64"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default=workloads.SQUARE_8192.name, choices=sorted(workloads.WORKLOADS))
    p.add_argument("--layout", default="panel", choices=["panel", "full"])
    p.add_argument("--impl", default="gbqr", choices=["gbqr", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget per oracle build")
    p.add_argument("--roofline-steps", type=int, default=2,
                   help="traced factorizations (look-ahead off) for the GEMM family's roofline")
    p.add_argument("--sub-configs", default="gaussian_1024x128,graded_32768x2048",
                   help="other workloads timed beside the headline one (library defaults)")
    p.add_argument("--sub-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                   help="skip the backward-error / orthogonality check after the timed region")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cutoff", type=int, default=0)
    p.add_argument("--fp64-gemm", choices=["dmma", "dfma"], default="dfma",
                   help="engine of the 64 x 64 FP64 GEMM tiles")
    p.add_argument("--autotune-ms", type=float, default=40000.0,
                   help="wall-clock budget of gbqr_autotune before the timed region (0: library defaults)")
    p.add_argument("--batched-autotune-ms", type=float, default=20000.0,
                   help="budget of gbqr_autotune_batched for the batched measurement (0: defaults)")
    p.add_argument("--panel", type=int, default=0)
    p.add_argument("--lookahead", choices=["on", "off"], default=None,
                   help="look-ahead of the PANEL top level (default: on, or the tuner's choice)")
    p.add_argument("--leaf", type=int, default=0)
    p.add_argument("--fanout", type=int, default=0)
    p.add_argument("--ls-solves", type=int, default=3, help="timed least-squares solves per grid point and precision (0: skip)")
    p.add_argument("--ls-decades", default="2,6,10", help="column-grading decades (kappa ~ 10^d x kappa(Gaussian))")
    p.add_argument("--ls-shapes", default="32768x2048,8192x8192")
    p.add_argument("--ls-precisions", default="fp64,mixed", help="which LS paths to time (fp64, mixed)")
    p.add_argument("--ls-oracle-shapes", default="32768x2048",
                   help="LS shapes whose results are also compared with the CPU oracle's solution")
    p.add_argument("--no-ls-kappa", action="store_true", help="skip the condition estimate (torch.linalg)")
    p.add_argument("--ls-autotune-ms", type=float, default=0.0,
                   help="gbqr_autotune budget per LS shape and precision before timing (0: defaults; the "
                        "tuner's objective is the factorization, and it measured slower for the solve)")
    p.add_argument("--batched", type=int, default=2000, help="matrices in the batched measurement (0: skip)")
    p.add_argument("--batched-steps", type=int, default=3)
    p.add_argument("--batched-streams", type=int, default=0)
    p.add_argument("--batched-cutoff", type=int, default=0)
    p.add_argument("--batched-cutoff32", type=int, default=0, help="cutoff b of the FP32 batch (0: default 16)")
    p.add_argument("--serving", type=int, default=200, help="requests per serving run (0: skip)")
    p.add_argument("--serving-rates", default="100,400,1600,5000")
    p.add_argument("--serving-workers", type=int, default=16)
    return p.parse_args()


def accuracy_of(gb, ctx, A, T, A0, layout, nb, m, n, dev):
    """||A - QR||_F / ||A||_F, ||Q^T Q - I||_F and ||Q^T Q - I||_2 of a
    factorization (measurement only: torch on the device; Q from gbqr_form_q)."""
    import torch
    Q = gb.colmajor(m, n, f"cuda:{dev}")
    ctx.form_q(A, T, Q, layout, nb)
    torch.cuda.synchronize()
    R = torch.triu(A[:n, :])
    bwd = float(torch.linalg.matrix_norm(A0 - Q @ R) / torch.linalg.matrix_norm(A0))
    E = Q.T @ Q
    E.diagonal().sub_(1.0)
    fro = float(torch.linalg.matrix_norm(E))
    two = float(torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max())
    del Q, R, E
    return {"backward_err_fro": bwd, "orthogonality_fro": fro, "orthogonality_2": two}


def measure_config(gb, dev, w, args):
    """One other workload with the library defaults (PANEL layout): ms per
    factorization over args.sub_steps timed steps (CUDA events, after 3
    warm-ups, A restored from a device copy inside each step), TFLOP/s at
    2mn^2 - 2n^3/3, and the accuracy of the last step."""
    import torch
    a = w.matrix()
    A0 = gb.to_colmajor(a, f"cuda:{dev}")
    A = gb.colmajor(w.m, w.n, f"cuda:{dev}")
    nb = gb.default_panel_nb(w.m, w.n)
    T = gb.colmajor(min(nb, w.n), w.n, f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    ctx = gb.Context(dev, stream)

    def step():
        A.copy_(A0)
        ctx.factor(A, T, gb.GBQR_T_PANEL)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.sub_steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.sub_steps
    st, _ = ctx.sync()
    acc = accuracy_of(gb, ctx, A, T, A0, gb.GBQR_T_PANEL, nb, w.m, w.n, dev)
    ctx.close()
    tf = w.flops / (ms * 1e-3) / 1e12
    return {"m": w.m, "n": w.n, "graded": w.graded, "seed": w.seed, "ms_per_step": ms, "tflops": tf,
            "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS, "steps": args.sub_steps, "status": int(st), **acc}


def measure_serving(gb, dev, args):
    """Least-squares serving: Poisson arrivals at each rate, requests from
    workloads.serving_specs, served by gbqr_server_* (continuous batching,
    HBM admission cap 120 GB) with FP64 only vs GBQR_PREC_AUTO (mixed first,
    FP64 when refinement stalls).  Reports solves/s (requests / makespan) and
    p50 / p99 latency (submit to done) per rate and mode."""
    import torch
    specs = workloads.serving_specs(args.serving)
    probs = [workloads.serving_device_problem(m, n, d, workloads.SERVING_SEED * 1000 + i, f"cuda:{dev}")
             for i, (m, n, d) in enumerate(specs)]
    xs = [torch.zeros(n, dtype=torch.float64, device=f"cuda:{dev}") for (m, n, d) in specs]
    torch.cuda.synchronize()
    rates = [float(r) for r in args.serving_rates.split(",") if r]
    rng = np.random.default_rng(workloads.SERVING_SEED + 1)
    gaps = rng.exponential(1.0, size=len(specs))
    out = {"workload": f"{len(specs)} LS requests, m log-U[512,65536], n log-U[32,1024], kappa log-U[1e1,1e8], "
                       f"one RHS, seed {workloads.SERVING_SEED}", "workers": args.serving_workers,
           "cap_bytes": 120 << 30, "mean_flops_per_request": float(np.mean([2.0 * m * n * n for (m, n, d) in specs]))}
    for mode, prec in [("fp64", gb.GBQR_FP64), ("mixed_auto", gb.GBQR_PREC_AUTO)]:
        ctx = gb.Context(dev)
        ctx.serve(args.serving_workers, 120 << 30)
        # warm-up: one request of each size class through the server
        for i in range(min(4, len(specs))):
            ctx.poll(ctx.submit(probs[i][0], probs[i][2], xs[i], prec), wait=True)
        res_mode = {}
        for rate in rates:
            arrivals = np.cumsum(gaps / rate)
            t0 = time.perf_counter()
            ids = []
            for i, (a, xt, b) in enumerate(probs):
                now = time.perf_counter() - t0
                if arrivals[i] > now:
                    time.sleep(arrivals[i] - now)
                ids.append(ctx.submit(a, b, xs[i], prec, tag=i))
            results = [ctx.poll(r, wait=True) for r in ids]
            makespan = max(r.latency_ms / 1e3 + arrivals[i] for i, r in enumerate(results))
            lat = sorted(r.latency_ms for r in results)
            bad = sum(1 for r in results if r.status != gb.GBQR_OK)
            ran_mixed = sum(1 for r in results if r.prec_used != gb.GBQR_FP64)
            res_mode[str(int(rate))] = {"solves_per_s": len(results) / makespan,
                                        "p50_ms": lat[len(lat) // 2],
                                        "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                                        "failed": bad, "ran_mixed": ran_mixed,
                                        "ran_fp64": len(results) - ran_mixed,
                                        "fell_back_to_fp64": sum(1 for r in results if r.fell_back)}
        if mode == "fp64":
            x_fp64 = [x.clone() for x in xs]
        else:
            # the AUTO result against the FP64 result of the same request,
            # scaled by the conditioning bound kappa u (kappa = 10^d graded)
            d = [float(torch.linalg.norm(x - x0) / torch.linalg.norm(x0)) for x, x0 in zip(xs, x_fp64)]
            res_mode["max_rel_diff_vs_fp64"] = max(d)
            res_mode["max_rel_diff_over_kappa_u"] = max(v / (10.0 ** sp[2] * 2.0 ** -53) for v, sp in zip(d, specs))
            res_mode["max_rel_diff_vs_fp64_kappa_le_1e2"] = max([v for v, sp in zip(d, specs) if sp[2] <= 2.0] or [0.0])
        ctx.stop_serving()
        ctx.close()
        out[mode] = res_mode
    return out


def _time_batch_graph(gb, ctx, stream, buf, pristine, As, Ts, o, steps):
    """Capture gbqr_factor_batched(As, Ts) into one graph; time `steps`
    replays (inputs restored by one device copy before each, untimed)."""
    import torch
    with torch.cuda.stream(stream):
        ctx.factor_batched(As, Ts, o)                   # warm-up: lanes, workspace
        torch.cuda.synchronize()
        graph = ctx.capture(lambda: ctx.factor_batched(As, Ts, o))
        times = []
        for _ in range(max(1, steps)):
            buf.copy_(pristine)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.launch()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    graph.close()
    return sorted(times)[len(times) // 2]


def measure_batched(gb, dev, args):
    """The batched tall-skinny workload: args.batched matrices, m log-uniform
    in [256, 16384], n uniform in [16, 256], factored by gbqr_factor_batched
    (FP64: one persistent kernel launch for the whole batch, captured in a
    graph with its table upload), then the same matrices rounded to FP32 by
    gbqr_factor_batched_f32.  Each timed step restores the inputs with one
    device copy (untimed), then launches the graph."""
    import torch
    shapes = workloads.batched_shapes(args.batched, workloads.BATCHED_SEED)
    buf, offs = workloads.batched_device_buffer(shapes, workloads.BATCHED_SEED, f"cuda:{dev}")
    pristine = buf.clone()
    As = [buf[o:o + m * n].view(n, m).T for (m, n), o in zip(shapes, offs)]
    Ts = [torch.empty((n, min(128, n)), dtype=torch.float64, device=f"cuda:{dev}").T for (m, n) in shapes]
    stream = torch.cuda.Stream(dev)
    ctx = gb.Context(dev, stream)
    flops = sum(workloads.qr_flops(m, n) for (m, n) in shapes)
    o = gb.opts(batch_streams=args.batched_streams, cutoff_b=args.batched_cutoff)
    tuned, tune_ms = None, None
    if args.batched_autotune_ms > 0 and not (args.batched_streams or args.batched_cutoff):
        with torch.cuda.stream(stream):
            o, tune_ms = ctx.autotune_batched(shapes, gb.GBQR_FP64, args.batched_autotune_ms)
        tuned = gb.opts_dict(o)
    ms = _time_batch_graph(gb, ctx, stream, buf, pristine, As, Ts, o, args.batched_steps)
    st, _ = ctx.sync()
    out = {"workload": f"{len(shapes)} matrices, m log-uniform [256, 16384], n uniform [16, 256], "
                       f"iid N(0,1), seed {workloads.BATCHED_SEED}",
           "total_flops": flops, "ms_per_batch": ms, "tflops": flops / (ms * 1e-3) / 1e12,
           "frac_of_fp64_peak": flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
           "matrices_per_s": len(shapes) / (ms * 1e-3), "graph_launches_per_batch": 1, "status": int(st),
           "engine": "one persistent kernel launch (panel and update tasks, list-scheduled), captured in a graph",
           "kernel_launches_per_batch": 1, "cutoff_b": o.cutoff_b or 16,
           "tuned": tuned, "tuned_ms": tune_ms, "dtype": "f64"}
    del As, Ts, buf, pristine
    # FP32: the same matrices rounded to float32, FP32 arithmetic throughout
    buf32, _ = workloads.batched_device_buffer(shapes, workloads.BATCHED_SEED, f"cuda:{dev}")
    buf32 = buf32.float()
    pristine32 = buf32.clone()
    As32 = [buf32[o_:o_ + m * n].view(n, m).T for (m, n), o_ in zip(shapes, offs)]
    Ts32 = [torch.empty((n, min(128, n)), dtype=torch.float32, device=f"cuda:{dev}").T for (m, n) in shapes]
    o32 = gb.opts(cutoff_b=args.batched_cutoff32, batch_streams=args.batched_streams)
    ms32 = _time_batch_graph(gb, ctx, stream, buf32, pristine32, As32, Ts32, o32, args.batched_steps)
    st32, _ = ctx.sync()
    out["fp32"] = {"ms_per_batch": ms32, "tflops": flops / (ms32 * 1e-3) / 1e12,
                   "matrices_per_s": len(shapes) / (ms32 * 1e-3), "status": int(st32), "dtype": "f32",
                   "cutoff_b": args.batched_cutoff32 or 16, "kernel_launches_per_batch": 1}
    ctx.close()
    return out


def kappa_estimate(R, iters: int = 40) -> float:
    """sigma_max / sigma_min of the n x n upper triangular R (= kappa_2(A)),
    by power iteration on R^T R and inverse power iteration with two
    triangular solves per step (measurement only: torch on the device)."""
    import torch
    g = torch.Generator(device=R.device)
    g.manual_seed(0)
    v = torch.randn(R.shape[0], 1, dtype=torch.float64, device=R.device, generator=g)
    u = v.clone()
    smax2 = smin2_inv = 0.0
    for _ in range(iters):
        v = R.T @ (R @ v)
        smax2 = float(torch.linalg.norm(v))
        v /= smax2
        y = torch.linalg.solve_triangular(R.T, u, upper=False)
        u = torch.linalg.solve_triangular(R, y, upper=True)
        smin2_inv = float(torch.linalg.norm(u))
        u /= smin2_inv
    return math.sqrt(smax2 * smin2_inv)


def measure_ls(gb, ctx, dev, args):
    """Least squares on the graded workloads (32768 x 2048 and 8192 x 8192,
    column j scaled by 10^(-d j / n) for d in args.ls_decades, x_true iid
    N(0,1), b = A x_true + 1e-8 N(0,1)), FP64 path vs mixed path (tensor-core
    split-BF16 updates + FP64 refinement).  Each solve is timed alone with
    CUDA events; solves/s = count / summed time; p50 / p99 over the solves.
    Accuracy per result: error vs x_true, the mixed result vs the FP64
    result, and the normwise backward error
    ||A^T r|| / (||A||_F ||r|| + ||A||_F^2 ||x||) with r = b - A x, all in FP64.
    kappa_2(A) is estimated from the FP64 R factor."""
    import torch
    devs = f"cuda:{dev}"
    stream = torch.cuda.current_stream(dev)
    ctx = gb.Context(dev, stream)        # its own, library-grown workspace
    shapes = [tuple(int(v) for v in s.split("x")) for s in args.ls_shapes.split(",") if s]
    decades = [float(d) for d in str(args.ls_decades).split(",") if d]
    oracle_shapes = set(x for x in args.ls_oracle_shapes.split(",") if x)
    grid = []
    for (m, n) in shapes:
        for d in decades:
            seed = 11 + int(d)
            A, xt, b = workloads.serving_device_problem(m, n, d, seed, devs)
            af = float(torch.linalg.matrix_norm(A))
            Af = A.clone()
            Tf = gb.colmajor(min(gb.default_panel_nb(m, n), n), n, devs)
            ctx.factor(Af, Tf, gb.GBQR_T_PANEL)
            torch.cuda.synchronize()
            kappa = None if args.no_ls_kappa else kappa_estimate(torch.triu(Af[:n, :n]))
            del Af, Tf
            row = {"m": m, "n": n, "decades": d, "kappa_est": kappa, "seed": seed}
            xs = {}
            for prec, name in [(gb.GBQR_FP64, "fp64"), (gb.GBQR_MIXED_SPLITBF16, "mixed_splitbf16")]:
                if name.split("_")[0] not in args.ls_precisions.split(","):
                    continue
                # the tuner's choice for this shape class and precision (cached in ctx,
                # picked up by gbqr_ls_solve); once per shape
                if args.ls_autotune_ms > 0 and ctx.tuned(gb.GBQR_TUNE_FACTOR, m, n, gb.GBQR_T_PANEL, prec) is None:
                    best, _ = ctx.autotune(m, n, gb.GBQR_T_PANEL, prec, args.ls_autotune_ms)
                    row.setdefault("tuned", {})[name] = gb.opts_dict(best)
                x = torch.zeros(n, dtype=torch.float64, device=devs)
                st, info = ctx.ls_solve(A, b, x, prec)          # warm-up
                times = []
                for _ in range(args.ls_solves):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st, info = ctx.ls_solve(A, b, x, prec)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                times.sort()
                xs[name] = x.clone()
                r = b - A @ x
                bwd = float(torch.linalg.norm(A.T @ r)) / (af * float(torch.linalg.norm(r)) + af * af * float(torch.linalg.norm(x)))
                row[name] = {"status": int(st), "solves_per_s": len(times) / (sum(times) * 1e-3),
                             "p50_ms": times[len(times) // 2],
                             "p99_ms": times[min(len(times) - 1, int(0.99 * len(times)))],
                             "refine_iters": int(info.refine_iters), "refine_last": float(info.refine_last),
                             "gmres_steps": int(info.gmres_steps), "lib_backward_err": float(info.backward_err),
                             "rel_err_vs_xtrue": float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt)),
                             "backward_err": bwd}
            if len(xs) < 2:
                grid.append(row)
                del A, b, xt
                torch.cuda.empty_cache()
                continue
            row["mixed_vs_fp64_rel_diff"] = float(torch.linalg.norm(xs["mixed_splitbf16"] - xs["fp64"]) /
                                                  torch.linalg.norm(xs["fp64"]))
            if f"{m}x{n}" in oracle_shapes:
                # both results against the FP64 oracle's solution of the same
                # problem (all-cores build on the host; bytes copied from the device)
                import oracle
                t0 = time.perf_counter()
                x_orc, _ = oracle.all_cores().ls_solve(gb.to_numpy(A), b.cpu().numpy())
                xo = torch.from_numpy(x_orc).to(devs)
                for name in ("fp64", "mixed_splitbf16"):
                    row[name]["rel_err_vs_oracle"] = float(torch.linalg.norm(xs[name] - xo) / torch.linalg.norm(xo))
                row["oracle_seconds"] = time.perf_counter() - t0
                row["kappa_u"] = (kappa or 0.0) * 2.0 ** -53
            row["speedup_mixed"] = row["mixed_splitbf16"]["solves_per_s"] / row["fp64"]["solves_per_s"]
            grid.append(row)
            del A, b, xt
            torch.cuda.empty_cache()
    ctx.close()
    return {"workload": "ls graded m x n, column j scaled 10^(-d j/n), x_true N(0,1), b = A x_true + 1e-8 N(0,1), "
                        "seeded torch generator (seed 11 + d)", "solves_per_point": args.ls_solves, "grid": grid}


# ------------------------------------------------------------- multi-rank
def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank factors its own matrix (independent replicas)."""
    return base_seed + rank


def max_over_ranks(value: float, dist, device="cpu") -> float:
    """The slowest rank's time: all-reduce MAX (the only collective; it is on
    the timing path, never on the data path)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank: float, world: int, ms_per_step: float) -> float:
    return flops_per_rank * world / (ms_per_step * 1e-3) / 1e12


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU baseline
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_steps_seconds(orc, block: np.ndarray, k: int) -> float:
    """Seconds of the oracle's C call for the first k Householder steps of a
    fresh copy of block (the copy is made outside the timed call)."""
    import ctypes
    work = np.array(block, dtype=np.float64, order="F", copy=True)
    mm, nn = work.shape
    tau = np.zeros(max(1, min(mm, nn)))
    P = ctypes.POINTER(ctypes.c_double)
    t0 = time.perf_counter()
    rc = orc.lib.orc_house_qr(mm, nn, work.ctypes.data_as(P), max(1, mm), tau.ctypes.data_as(P), k)
    dt = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError(f"oracle house_qr returned {rc}")
    return dt


def oracle_rate(orc, a: np.ndarray, budget_s: float, strata: int = 8):
    """Stratified estimate of the oracle's rate on the full QR of a.  The n
    Householder steps are cut into `strata` equal ranges; in each, k steps
    (sized to budget_s / strata seconds) are timed on the trailing matrix at
    the range's middle, and the range's time is its flops at that rate.
    Returns (TFLOP/s of the whole factorization, estimated seconds for it,
    sampled steps, seconds spent in the sampled calls)."""
    m, n = a.shape
    kmax = min(m, n)
    bounds = [round(s * kmax / strata) for s in range(strata + 1)]
    per = budget_s / strata
    est, steps, spent = 0.0, 0, 0.0
    for s in range(strata):
        j0, j1 = bounds[s], bounds[s + 1]
        if j1 <= j0:
            continue
        mid = (j0 + j1) // 2
        t1 = _oracle_steps_seconds(orc, a[mid:, mid:], 1)
        k = int(max(1, min(j1 - j0, per / max(t1, 1e-9))))
        start = max(j0, min(mid - k // 2, j1 - k))
        tk = _oracle_steps_seconds(orc, a[start:, start:], k)
        rate = workloads.qr_flops_partial(m - start, n - start, k) / max(tk, 1e-12)
        est += workloads.qr_flops_partial(m - j0, n - j0, j1 - j0) / rate
        steps += k
        spent += t1 + tk
    return workloads.qr_flops(m, n) / est / 1e12, est, steps, spent


def cpu_baseline(a: np.ndarray, budget_s: float) -> dict:
    """The oracle on this host: the all-cores build (reported value) and the
    one-thread build, each a stratified sample of budget_s seconds."""
    import oracle
    par, ser = oracle.all_cores(), oracle.default()
    tf, est, steps, spent = oracle_rate(par, a, budget_s)
    tf1, est1, steps1, spent1 = oracle_rate(ser, a, budget_s)
    m, n = a.shape
    return {"value": tf, "unit": "TFLOP/s", "cores": par.threads, "kind": "oracle",
            "sample": f"stratified: {steps} of {min(m, n)} Householder steps of the same {m}x{n} matrix, "
                      f"8 step ranges, each timed at its midpoint ({spent:.1f} s); full QR estimated at {est:.1f} s",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(), "build": "oracle/house.c -fopenmp (all cores)",
            "single_thread": {"value": tf1, "unit": "TFLOP/s", "cores": 1, "estimated_full_qr_s": est1,
                              "sample": f"{steps1} steps ({spent1:.1f} s), same strata"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workloads.WORKLOADS[args.workload]
    a = w.matrix()
    # each step: one stratified sample of the workload, sized so that the
    # whole run ends within a few minutes
    per_step_budget = max(0.8, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    import oracle
    orc = oracle.all_cores()
    for _ in range(args.warmup):
        oracle_rate(orc, a, per_step_budget)
    ests, spent, steps = [], 0.0, 0
    for _ in range(args.steps):
        _, est, k, sp = oracle_rate(orc, a, per_step_budget)
        ests.append(est)
        spent += sp
        steps += k
    est_mean = sum(ests) / len(ests)
    value = w.flops / est_mean / 1e12
    sample = (f"per step: a stratified sample of the {w.m}x{w.n} factorization (8 step ranges, a few steps timed "
              f"at each range's midpoint; {steps} steps, {spent:.1f} s over {args.steps} steps), the full "
              f"factorization's time estimated from it; oracle built with OpenMP on {orc.threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * est_mean,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "graded": w.graded, "seed": w.seed},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": orc.threads, "kind": "oracle",
                         "sample": sample, "nproc": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gbqr(args):
    import ctypes

    import torch

    import paper_1805_05278_gb300 as gb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)

    gb.build()
    w = workloads.WORKLOADS[args.workload]
    layout = gb.GBQR_T_PANEL if args.layout == "panel" else gb.GBQR_T_FULL
    o = gb.opts(cutoff_b=args.cutoff, panel_nb=args.panel, leaf_rows=args.leaf, fanout=args.fanout,
                lookahead={None: 0, "on": 1, "off": -1}[args.lookahead],
                fp64_gemm=gb.GBQR_GEMM_DMMA if args.fp64_gemm == "dmma" else gb.GBQR_GEMM_DFMA)
    stream = torch.cuda.current_stream(dev)
    ctx = gb.Context(dev, stream)
    # the tuner picks (b, k, leaf, nb, look-ahead, GEMM engine) unless any is given
    tuned, tune_ms = None, None
    explicit = (args.cutoff or args.panel or args.leaf or args.fanout or args.fp64_gemm != "dfma"
                or args.lookahead is not None)
    if args.autotune_ms > 0 and not explicit:
        o, tune_ms = ctx.autotune(w.m, w.n, layout, gb.GBQR_FP64, args.autotune_ms)
        tuned = gb.opts_dict(o)
    nb = o.panel_nb or gb.default_panel_nb(w.m, w.n)
    trows = w.n if layout == gb.GBQR_T_FULL else min(nb, w.n)

    seed = replica_seed(w.seed, rank)
    a_host = workloads.graded(w.m, w.n, seed) if w.graded else workloads.gaussian(w.m, w.n, seed)
    A0 = gb.to_colmajor(a_host, f"cuda:{dev}")
    A = gb.colmajor(w.m, w.n, f"cuda:{dev}")
    T = gb.colmajor(trows, w.n, f"cuda:{dev}")
    ws = torch.empty(gb.workspace_bytes(w.m, w.n, layout, o), dtype=torch.uint8, device=f"cuda:{dev}")
    ctx.set_workspace(ws)

    def step():
        A.copy_(A0)
        ctx.factor(A, T, layout, o)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st, _ = ctx.sync()
    if st != gb.GBQR_OK:
        raise RuntimeError(f"warm-up reported status {st}")

    # timed region: K steps, launch tracing off, clocks sampled alongside
    launches0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    clocks = clk.summary()
    ms_step = max_over_ranks(ms_total / args.steps, dist, f"cuda:{dev}")
    value = whole_job_tflops(w.flops, world, ms_step)

    # roofline pass (after the timed region): the same factorization with the
    # look-ahead off, traced, so that each launch runs alone on the GPU and
    # its event-bracketed duration is its own; the GEMM family's summed time
    # then cannot exceed the step's
    o_serial = gb.opts(**{**gb.opts_dict(o), "lookahead": -1})
    ctx.trace(True)
    ctx.trace_read()
    es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    es0.record(stream)
    for _ in range(args.roofline_steps):
        A.copy_(A0)
        ctx.factor(A, T, layout, o_serial)
    es1.record(stream)
    torch.cuda.synchronize()
    serial_ms = es0.elapsed_time(es1)
    trace = ctx.trace_read()
    ctx.trace(False)

    # end to end through the C ABI with host buffers (pinned), copies inside
    a_pin = torch.from_numpy(np.ascontiguousarray(a_host.T)).pin_memory()   # (n, m) row-major = A column-major
    t_pin = torch.empty((w.n, trows), dtype=torch.float64).pin_memory()
    e2e_times = []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        a_pin.copy_(torch.from_numpy(np.ascontiguousarray(a_host.T)))
        t0 = time.perf_counter()
        gb.check(gb.gbqr_factor(ctx.handle, w.m, w.n, ctypes.c_void_p(a_pin.data_ptr()), w.m,
                                ctypes.c_void_p(t_pin.data_ptr()), trows, layout, ctypes.byref(o)), "gbqr_factor(host)")
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_times.append(dt)
    e2e_value = w.flops * world / statistics.median(e2e_times) / 1e12 if e2e_times else None

    # accuracy of the last timed factorization (measurement only: torch on
    # the device): Q from gbqr_form_q, backward error and orthogonality (F-norm)
    accuracy = None
    if args.accuracy and w.m >= w.n:
        try:
            step()                      # one more factorization in the timed configuration
            torch.cuda.synchronize()
            accuracy = accuracy_of(gb, ctx, A, T, A0, layout, nb, w.m, w.n, dev)
            accuracy["note"] = "||A - QR||_F / ||A||_F, ||Q^T Q - I||_F and _2 of a step in the timed configuration, FP64"
        except (gb.GbqrError, RuntimeError) as exc:
            accuracy = {"error": str(exc)}

    st, info = ctx.sync()
    ls = measure_ls(gb, None, dev, args) if (args.ls_solves > 0 and rank == 0) else None
    batched = measure_batched(gb, dev, args) if (args.batched > 0 and rank == 0) else None
    serving = measure_serving(gb, dev, args) if (args.serving > 0 and rank == 0) else None

    gemm = trace.get("gemm", {})
    achieved = gemm["flops"] / (gemm["ms"] * 1e-3) / 1e12 if gemm.get("ms") else None
    share = (gemm.get("ms", 0.0) / serial_ms) if serial_ms else None
    if share is not None and share > 1.0:
        raise RuntimeError(f"GEMM family time exceeds the step in the serial pass (share {share:.3f})")
    alg_bytes = (gemm["bytes"] / gemm["launches"]) if gemm.get("launches") else None
    ratio = DGEMM_TRAFFIC_RATIO.get(
        (w.name, nb if layout == gb.GBQR_T_PANEL else 0, o.cutoff_b or 16, "dmma" if o.fp64_gemm == gb.GBQR_GEMM_DMMA else "dfma"))
    roofline = {
        "bound": "alu", "kernel": "dgemm_kernel (update / T-assembly products)",
        "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
        "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.070 GHz (nominal 1.25 TFLOP/s FP64); "
                       "measured DFMA probe 1.06, DMMA probe 1.10, largest update launch 1.22 TFLOP/s",
        "how": f"algorithmic flops / summed CUDA-event durations of every GEMM launch in {args.roofline_steps} "
               f"traced factorizations with the look-ahead off (launches run alone)",
        "traffic": (ratio * alg_bytes) if (ratio and alg_bytes) else None,
        "traffic_unit": "bytes per launch (dram read + write): ncu ratio to algorithmic bytes x this pass's "
                        "algorithmic bytes per launch",
        "traffic_ratio_ncu": ratio,
        "traffic_source": DGEMM_TRAFFIC_SOURCE if ratio else None,
        "algorithmic_bytes_per_launch": alg_bytes,
        "launches": gemm.get("launches"), "share_of_step": share,
        "serial_ms_per_step": serial_ms / max(1, args.roofline_steps),
        "step_frac": value / world / FP64_PEAK_TFLOPS,
    }
    fams = {k: {"launches": v["launches"] / max(1, args.roofline_steps),
                "ms_per_step": v["ms"] / max(1, args.roofline_steps),
                "algorithmic_bytes_per_step": v["bytes"] / max(1, args.roofline_steps),
                "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] else None} for k, v in trace.items()}

    subs = {}
    if rank == 0 and args.sub_configs:
        for name in [n_ for n_ in args.sub_configs.split(",") if n_]:
            subs[name] = measure_config(gb, dev, workloads.WORKLOADS[name], args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(a_host, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "m": w.m, "n": w.n, "graded": w.graded, "seed": w.seed,
                       "t_layout": args.layout, "panel_nb": nb if layout == gb.GBQR_T_PANEL else None,
                       "cutoff_b": o.cutoff_b or 16, "fanout": o.fanout or "adaptive", "leaf_rows": o.leaf_rows,
                       "lookahead": o.lookahead, "fp64_gemm": "dmma" if o.fp64_gemm == gb.GBQR_GEMM_DMMA else "dfma",
                       "autotuned": tuned is not None, "autotune_ms": tune_ms, "parallelism": f"replicas x{world}",
                       "l2": "inputs (%.0f MB) larger than L2, no flush" % (w.m * w.n * 8 / 1e6),
                       "step": "restore A from a device copy + gbqr_factor"},
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": w.m * w.n * 8,
                    "d2h_bytes_per_step": w.m * w.n * 8 + trows * w.n * 8,
                    "how": "gbqr_factor on pinned host buffers (H2D, factor, D2H inside the call)"},
            "gpu_launches": launches,
            "roofline": roofline,
            "families_serial_pass": fams,
            "configs": subs,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "ls": ls,
            "batched": batched,
            "serving": serving,
            "accuracy": accuracy,
            "status_after": int(st),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gbqr(args)


if __name__ == "__main__":
    sys.exit(main())
