"""Benchmark: decomposed ADMM (Algorithm 1) on the banded SDP workload
(n=2000, half-bandwidth 10, m=500; 1990 cliques of order 11) on one GB300.

A step is one full solve to eps = 1e-4 from a cold start (every step of the
iteration: scatter, affine projection with the cached inverse, clique gather,
batched PSD projection, multiplier update, stopping reductions), with the
adaptive penalty of Section 7.1.2 applied every iteration (mu = 2, nu = 10,
rho starting at 1).

  value     ADMM iterations/s of the FP32-projection form (launch schedule from
            the library autotuner, chosen before timing), whole solve as one
            CUDA graph (device-side while loop), inputs resident in HBM,
            L2 flushed (256 MiB write) before every timed step
  e2e       the same metric through the public API from host arrays:
            host preprocessing, one H2D upload, solve, D2H of X, y, Z
  fp64_plain  FP64 everywhere, cold Jacobi, one launch per phase, no graph
  fixed_rho   both forms again with rho = 1 throughout
  batched   256 independent uneven block-arrow SDPs (cliques of order
            20..60) solved as one direct sum, each stopping on its own test
  roofline  the batched projection kernel (FP32 ALU bound), launch durations
            from CUDA events in a profiled solve on the solve's stream
  cpu_baseline  the FP64 oracle on a bounded sample (host cores, 1 thread)

--impl reference runs the FP64 oracle (the CPU reference of this build) on the
same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM iters/s & time-to-1e-4 (FP32 batched vs FP64 plain, 1 GB300); clique-proj GFLOP/s"
WORKLOAD = "banded_n2000_w10_m500"
SM_COUNT = 152
# DRAM bytes of one launch of the dominant kernel (k_project_primal<float,12> on the
# banded workload, x formed by its own kernel) from the ncu capture summarised
# under profiles/ (3.359488 MB read, 0 written); to be re-taken whenever that
# kernel changes.
KERNEL_TRAFFIC_BYTES = 3359488
FP32_LANES_PER_SM = 128


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _clock_sampler(dev_index):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                                 "-i", str(dev_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1])); smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_baseline(iters, timeout=600):
    """Time the FP64 oracle (as it stands) on `iters` iterations of the
    workload in a fresh single-threaded process; returns (iters/s, seconds)."""
    code = (
        "import os,sys,time,json\n"
        f"sys.path.insert(0,{ROOT!r})\n"
        "from oracle import admm\n"
        "from paper_1707_05058_gb300 import workloads as W\n"
        "dp=admm.decompose(W.workload(1))\n"
        "t=time.perf_counter()\n"
        f"r=admm.primal_admm(dp,eps=0.0,max_iter={iters},adapt_every=1)\n"
        "dt=time.perf_counter()-t\n"
        "print(json.dumps({'iters':r.iters,'sec':dt}))\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["iters"] / d["sec"], d["sec"], d["iters"]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    iters = 10
    vals, secs = [], []
    for s in range(args.warmup + args.steps):
        v, sec, _ = _cpu_baseline(iters)
        if s >= args.warmup:
            vals.append(v); secs.append(sec)
    value = sum(iters for _ in vals) / sum(secs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "primal", "rho": "adaptive every iteration",
                       "sample": f"{iters} ADMM iterations per step"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{iters} iterations of the FP64 oracle (Algorithm 1) on {WORKLOAD} per step, 1 thread"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_over_ranks(torch, dist, world, total_ms, total_iters, device):
    """Whole-job rate of N replicas: iterations summed over ranks divided by the
    slowest rank's device time (max), as every rank's timed region is bracketed
    by the same barriers.  Returns (value, max_ms, summed_iters)."""
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(total_iters)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return n.item() / (t.item() / 1e3), t.item(), n.item()


def batch_shard(problems, rank, world):
    """The independent SDPs of the batched workload that rank `rank` solves:
    every world-th one (a partition of the batch; no data-path exchange)."""
    return problems[rank::world]


def _batched(cdsdp, workloads, torch, flush, stream, rank=0, world=1):
    """256 uneven block-arrow SDPs (l in [10,100], d in [10,40], h in [10,20],
    m in [50,400]; A_i with 5% density on the pattern) as one direct sum, each
    component stopping and freezing on its own test; FP32 graph with the
    adaptive penalty to eps = 1e-4, then per-iteration times of the first 50
    iterations (every component active) for the FP32 graph form, the profiled
    projection launches, and the plain FP64 form."""
    import numpy as np
    t0 = time.perf_counter()
    prob = workloads.direct_sum(batch_shard(workloads.workload(2), rank, world))
    t1 = time.perf_counter()
    P = cdsdp.Problem(prob)
    t2 = time.perf_counter()
    P.bind(max_iter=10000)
    info = P.info

    def timed(**kw):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = P.solve("primal", outputs=False, **kw)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    tuned, cand_ms = P.autotune("primal", iters=20, precision="fp32", adaptive_rho=1)
    kw = dict(eps=1e-4, max_iter=10000, precision="fp32", use_graph=1, adaptive_rho=1, **tuned)
    P.solve("primal", outputs=False, **kw)  # warm-up (graph build)
    ms, out = timed(**kw)
    it, st, _ = P.component_results()
    ms50, _ = timed(eps=0.0, max_iter=50, precision="fp32", use_graph=1, adaptive_rho=1, **tuned)
    P.solve("primal", outputs=False, eps=0.0, max_iter=20, precision="fp32", profile=1, adaptive_rho=1, **tuned)
    proj_ms, launches, iter_ms = P.profile()
    ms64, _ = timed(eps=0.0, max_iter=10, precision="fp64", use_graph=0, check_every=10, warm_start=0, adaptive_rho=1)
    sizes = np.diff(P.cliques()[0]).astype(np.float64)
    flops = float(np.sum(10.0 * sizes ** 3))
    gflops = flops / (proj_ms / launches / 1e3) / 1e9
    return {"workload": "256 block-arrow SDPs, direct sum", "n": int(info["n"]), "m": int(info["m"]),
            "cliques": int(info["p"]), "clique_order_max": int(info["max_clique"]), "components": int(info["ncomp"]),
            "nnz_A": int(info["nnz_A"]), "generate_s": t1 - t0, "setup_s": t2 - t1,
            "time_to_eps_ms": ms, "status": int(out["status"]), "iters_to_eps_max": int(out["iters"]),
            "component_iters": {"min": int(it.min()), "median": int(np.median(it)), "max": int(it.max()),
                                "sum": int(it.sum())},
            "components_solved": int(np.sum(st == 0)),
            "fp32_graph_ms_per_iter_all_active": ms50 / 50,
            "fp64_plain_ms_per_iter_all_active": ms64 / 10,
            "per_iter_speedup_fp32_graph_vs_fp64_plain": (ms64 / 10) / (ms50 / 50),
            "schedule": tuned, "autotune_ms_per_iter": cand_ms,
            "clique_proj_gflops": gflops, "proj_ms_per_iter": proj_ms / launches,
            "proj_flops_per_iter_nominal": flops}


def _grad_batch(cdsdp, workloads, torch, stream):
    """Differentiation workload: 64 banded SDPs (n=500, w=8, m=200) as one
    direct sum; 500 unrolled iterations of Algorithm 1 in the FP32-projection
    form with checkpoints every 50, then the reverse pass for the gradient of
    <g, x> with respect to c and b (g random).  Device times of both passes."""
    import numpy as np
    prob = workloads.direct_sum(workloads.workload(4))
    P = cdsdp.Problem(prob).bind(max_iter=64)
    c, b = P.problem_data()
    g = torch.tensor(np.random.default_rng(0).standard_normal(int(P.info["nnz_pattern"])), device="cuda")
    times = []
    for rep in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, gws = P.unrolled_forward(c, b, 500, 50, "fp32", 1.0)
        e1.record(stream)
        cbar, bbar = P.unrolled_backward(c, b, g, 500, 50, gws, "fp32", 1.0)
        e2.record(stream)
        e2.synchronize()
        times.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    fwd, bwd = times[-1]
    return {"workload": "64 banded SDPs n=500 w=8 m=200, direct sum", "n": int(P.info["n"]), "m": int(P.info["m"]),
            "cliques": int(P.info["p"]), "iterations": 500, "checkpoint_every": 50, "precision": "fp32 projection",
            "forward_ms": fwd, "backward_ms": bwd, "grad_finite": bool(torch.isfinite(cbar).all().item())}


def _completion(cdsdp, workloads, torch, stream):
    """Maximum-determinant completion (Section 7.1.1) of a positive definite
    partial matrix on the pattern of (a) the banded n=2000 workload and (b)
    the 64-SDP direct sum (n=500 each): factor only (t_k, s_k, log det) and
    with the dense blocks.  Device time over the whole call (the call waits
    once on the stream for its positive-definiteness flag)."""
    import numpy as np
    res = {}
    for key, prob in (("banded_n2000", workloads.workload(1)),
                      ("direct_sum_64x_n500", workloads.direct_sum(workloads.workload(4)))):
        P = cdsdp.Problem(prob)
        r, c = P.pattern()
        X = torch.tensor(workloads.pd_on_pattern(prob.n, r, c, 5), device="cuda")
        sb, we, _ = P.completion_sizes()
        scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
        Wd = torch.empty(we, dtype=torch.float64, device="cuda")
        out = {}
        for dense in (False, True):
            ms = []
            for rep in range(4):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.complete(X, dense=dense, stream=stream, scratch=scratch, out=Wd)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            out["dense_ms" if dense else "factor_ms"] = statistics.median(ms[1:])
        vc, _ = P.components()
        sizes = np.bincount(vc)
        out.update({"n": int(prob.n), "components": int(P.info["ncomp"]), "dense_doubles": int(we),
                    "step_launches": int(sizes.max()) - 1})
        res[key] = out
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-SDP batched workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1707_05058_gb300 import cdsdp, workloads

    prob = workloads.workload(1)
    t0 = time.perf_counter()
    P = cdsdp.Problem(prob)
    setup_s = time.perf_counter() - t0
    max_iter = 40000
    P.bind(max_iter=max_iter)
    info = P.info
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_solves(nsteps, warm, **opts):
        for _ in range(warm):
            P.solve("primal", outputs=False, eps=1e-4, max_iter=max_iter, **opts)
        ms, its = [], []
        for _ in range(nsteps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = P.solve("primal", outputs=False, eps=1e-4, max_iter=max_iter, **opts)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(out["iters"])
            assert out["status"] == 0, out
        return ms, its

    ADAPT = dict(adaptive_rho=1)
    # launch schedule of the FP32 form chosen by the library's autotuner (before timing)
    TUNED, tune_ms = P.autotune("primal", iters=30, precision="fp32", adaptive_rho=1)
    # ---- FP32-projection form, graph (the headline value)
    barrier()
    clk = _clock_sampler(torch.cuda.current_device()) if rank == 0 else None
    ms32, it32 = timed_solves(args.steps, args.warmup, precision="fp32", use_graph=1, **ADAPT, **TUNED)
    barrier()
    clocks = _clock_summary(clk) if rank == 0 else None
    value, _, _ = aggregate_over_ranks(torch, dist, world, sum(ms32), sum(it32), "cuda")
    time_to_eps_ms = statistics.median(ms32)

    # ---- plain FP64 form (FP64 everywhere, one launch per phase, no graph)
    ms64, it64 = timed_solves(1, 0, precision="fp64", use_graph=0, check_every=10, warm_start=0, **ADAPT)
    # ---- both forms with the penalty fixed at rho = 1
    ms32f, it32f = timed_solves(1, 1, precision="fp32", use_graph=1, **TUNED)
    ms64f, it64f = timed_solves(1, 0, precision="fp64", use_graph=0, check_every=10, warm_start=0)

    # ---- profiled FP32 solve: per-launch projection time from CUDA events
    P.solve("primal", outputs=False, eps=1e-4, max_iter=max_iter, precision="fp32", profile=1, check_every=50, **ADAPT,
            **TUNED)
    proj_ms, proj_launches, iter_ms = P.profile()
    sizes = np.diff(P.cliques()[0])
    flops_per_launch = float(np.sum(10.0 * sizes.astype(np.float64) ** 3))   # nominal 10 s^3 per clique
    proj_s_per_launch = proj_ms / 1e3 / max(proj_launches, 1)
    gflops = flops_per_launch / proj_s_per_launch / 1e9
    sm_mhz = (clocks or {}).get("sm_mhz") or 1440.0
    peak_fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s at the sampled clock

    # ---- end to end through the public API from host arrays
    e2e_ms, e2e_it = [], []
    e2e_parts = {"setup": [], "bind_upload": [], "solve_download": []}
    h2d = d2h = 0
    for s in range(6):
        torch.cuda.synchronize()
        t = time.perf_counter()
        Q = cdsdp.Problem(prob)
        t1 = time.perf_counter()
        Q.bind(max_iter=max_iter)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out = Q.solve("primal", eps=1e-4, max_iter=max_iter, precision="fp32", use_graph=1, **ADAPT, **TUNED)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        dt = t3 - t
        if s > 0:  # the first call also loads the library's kernels
            e2e_ms.append(dt * 1e3)
            e2e_it.append(out["iters"])
            e2e_parts["setup"].append((t1 - t) * 1e3)
            e2e_parts["bind_upload"].append((t2 - t1) * 1e3)
            e2e_parts["solve_download"].append((t3 - t2) * 1e3)
        nz = int(info["nnz_pattern"])
        h2d = int(Q.info["upload_bytes"])
        d2h = (2 * nz + int(info["m"])) * 8 + out["iters"] * 8 * 8
        del Q
    e2e_med = statistics.median(e2e_ms)
    e2e_value = statistics.median(e2e_it) / (e2e_med / 1e3)
    del P

    batched = None if args.no_batched else _batched(cdsdp, workloads, torch, flush, stream, rank, world)
    grad = None if args.no_batched else _grad_batch(cdsdp, workloads, torch, stream)
    compl = None if args.no_batched else _completion(cdsdp, workloads, torch, stream)
    if batched is not None and world > 1:  # each rank solved its share of the 256 SDPs
        _, tmax, _ = aggregate_over_ranks(torch, dist, world, batched["time_to_eps_ms"], 0, "cuda")
        batched["time_to_eps_ms"] = tmax
        batched["workload"] += f", {world} shards (every {world}th SDP per rank), time = slowest rank"

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            try:
                v, sec, n_it = _cpu_baseline(30)
                cpu = {"value": v, "unit": "iters/s", "cores": 1, "kind": "oracle",
                       "sample": f"{n_it} iterations of the FP64 oracle (Algorithm 1) on {WORKLOAD}, 1 thread, {sec:.1f} s"}
            except Exception as exc:  # report, do not hide
                cpu = {"value": None, "unit": "iters/s", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}
        launches_per_iter = 4  # scatter, A W t, cached-inverse GEMV, projection (+ x update, stopping test)
        gpu_launches = sum(it32) * launches_per_iter + len(it32)
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms32), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "primal", "eps": 1e-4, "cliques": int(info["p"]),
                       "clique_order": int(info["max_clique"]), "m": int(info["m"]),
                       "precision": "fp32 projection, fp64 affine step and reductions",
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_eps_ms": time_to_eps_ms, "iters_to_eps": int(statistics.median(it32)),
            "fp64_plain": {"iters_per_s": sum(it64) / (sum(ms64) / 1e3), "time_to_eps_ms": statistics.median(ms64),
                           "iters_to_eps": int(statistics.median(it64)),
                           "form": "float64 everywhere, cold Jacobi every iteration, one launch per phase, no graph"},
            "speedup_time_to_eps_fp32_graph_vs_fp64_plain": statistics.median(ms64) / time_to_eps_ms,
            "rho": "adaptive (Section 7.1.2), every iteration, mu 2, nu 10, from rho = 1",
            "schedule": TUNED, "autotune_ms_per_iter": tune_ms,
            "fixed_rho": {"rho": 1.0,
                          "fp32_graph": {"time_to_eps_ms": ms32f[0], "iters_to_eps": it32f[0],
                                         "iters_per_s": it32f[0] / (ms32f[0] / 1e3)},
                          "fp64_plain": {"time_to_eps_ms": ms64f[0], "iters_to_eps": it64f[0],
                                         "iters_per_s": it64f[0] / (ms64f[0] / 1e3)},
                          "speedup_time_to_eps": ms64f[0] / ms32f[0]},
            "batched": batched,
            "grad": grad,
            "completion": compl,
            "clique_proj_gflops": gflops,
            "setup_ms": setup_s * 1e3,
            "roofline": {"bound": "alu", "achieved": gflops / 1e3, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": gflops / 1e3 / peak_fp32, "traffic": KERNEL_TRAFFIC_BYTES,
                         "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one warm-started launch, "
                                           "ncu full capture (cold caches), profiles/k_project_primal_banded_n2000_fp32.md",
                         "kernel": "k_project_primal<float,12>",
                         "peak_note": f"FP32 FMA peak derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x sampled SM clock",
                         "flops_per_launch": flops_per_launch, "launch_ms": proj_s_per_launch * 1e3},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_med, "steps": len(e2e_ms), "statistic": "median",
                    "breakdown_ms": {k: statistics.median(v) for k, v in e2e_parts.items()},
                    "setup_ms": setup_s * 1e3},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
