"""Benchmark: the decomposed ADMM of arXiv 1707.05058 (Algorithm 1) on the
batched block-arrow workload on one GB300: 256 independent block-arrow SDPs of
uneven size (l in [10, 100], d in [10, 40], h in [10, 20], m in [50, 400];
A_i with 5% density on the pattern), solved as one direct sum in one CUDA
graph, each SDP stopping on its own test at eps = 1e-4 (adaptive penalty of
Section 7.1.2 every iteration).  n = 362,087, m = 58,337, 14,371 cliques of
order 20..60.

A step is one solve of the whole batch to eps = 1e-4 from a cold start (every
step of the iteration: scatter, affine projection with the cached inverse,
clique gather, batched PSD projection, multiplier update, stopping
reductions).

  value     SDP-iterations/s of the FP32-projection form: the iterations run by
            the 256 SDPs (each its own count until it stops) per second of
            device time (CUDA events on the solve's stream); launch schedule
            from the library autotuner, chosen before timing; the workspace
            (5.8 GB) is larger than L2, and L2 is also flushed (256 MiB write)
            before every timed step
  e2e       the same metric through the public API from host arrays:
            cdsdp_setup_batch (host preprocessing), one H2D upload of the
            workspace, solve, D2H of X, y, Z and the history
  per_iteration  ms per iteration with every SDP active, for the FP32 graph,
            FP32 plain launches, FP64 plain (cold Jacobi), FP64 plain (warm
            Jacobi) and FP64 graph (warm) forms: precision, warm start and
            graph separated
  parity    objective gap of the timed solve's SDPs against stored oracle
            solves of three summands (tests/golden/batch_oracle.json)
  roofline  the projection size class with the largest device time (FP32 ALU
            bound): nominal 10 s^3 flops per clique / its mean launch duration
            from CUDA events over a profiled 200-iteration solve from the cold
            start (every SDP active, size classes launched one after the other
            so that each launch is timed alone), against the FMA peak measured
            by cdsdp_fma_peak on this GPU
  hsde      Algorithm 3 on the batch, each SDP scaled alone and embedded
            alone: time to 1e-4 of one FP32 graph solve, and parity of three
            summands against stored oracle solves
  affine_sweep  affine-projection cost against m (block-arrow l=100, d=10,
            h=20, m = 200 and 1000) per form, cached inverse and 5 CG steps
  dense_sample  eight SDPs of the batch with A_i dense on the pattern (1.1e8
            nonzeros): ms per iteration, the non-projection part's GB/s
            against the measured HBM peak, time to 1e-4
  banded    the banded workload (n=2000, w=10, m=500; 1990 cliques of order
            11): time to 1e-4 in the FP32 graph and plain FP64 forms
  maxcut    the MaxCut workload (n = 10^4, G(n, 6/(n-1)), merged cliques up to
            order 3560): clique histogram, per-iteration split, the tensor-core
            sign iteration against the TF32 peak, FP32 solve to 1e-4 (capped)
  cpu_baseline  the FP64 oracle on a bounded sample of the same batch: 8 of its
            SDPs, 4 iterations each, on 1 host thread and on one process per
            SDP

--impl reference runs the FP64 oracle (the CPU reference implementation) on
the same workload and metric (bounded samples; see run_reference).
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
WORKLOAD = "batch256_block_arrow_l10-100_d10-40_h10-20_m50-400_density0.05"
BANDED = "banded_n2000_w10_m500"
# SDPs of the batch in the CPU-baseline sample (every 32nd) and oracle iterations per SDP
CPU_SAMPLE = list(range(0, 256, 32))
# iterations of the profiled solve behind the per-class launch times
PROFILE_ITERS = 200
CPU_ITERS = 4
# DRAM bytes of one launch of the roofline's kernel (padded order 52, 1667
# cliques): the ncu capture summarised in profiles/k_project_cta52_batched128_fp32.md
# read 44.18 MB for 812 cliques of the class (the clique state, the gathered x
# and the eigenvector cache; no re-reads), scaled by the clique count.  Set to
# None when the kernel changes until it is captured again.
KERNEL_TRAFFIC_BYTES = 44.18e6 * 1667 / 812


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


# ---- CPU baseline: the oracle as it stands -----------------------------------

def _oracle_member(args):
    """Oracle (Algorithm 1, FP64, adaptive penalty every iteration) on SDP
    `member` of the batch for `iters` iterations in this process; returns
    (iterations, seconds of the iteration loop)."""
    member, iters = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import admm
    from paper_1707_05058_gb300 import workloads as W
    dp = admm.decompose(W.workload_batch_member(2, member))
    t = time.perf_counter()
    r = admm.primal_admm(dp, eps=0.0, max_iter=iters, adapt_every=1)
    return r.iters, time.perf_counter() - t


def _oracle_sample(members, iters, processes):
    """The oracle on `members` of the batch, `iters` iterations each, in a
    spawned pool of `processes` single-threaded processes (1: one after the
    other).  Returns (SDP-iterations/s over the wall time of the iteration
    loops, seconds, iterations)."""
    import multiprocessing as mp
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(processes) as pool:
            if processes == 1:
                res = [pool.apply(_oracle_member, ((m, iters),)) for m in members]
                secs = sum(r[1] for r in res)
            else:
                res = pool.map(_oracle_member, [(m, iters) for m in members])
                secs = max(r[1] for r in res)  # the loops run side by side
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    its = sum(r[0] for r in res)
    return its / secs, secs, its


def _cpu_baseline_block():
    cores = min(len(CPU_SAMPLE), os.cpu_count() or 1)
    v1, s1, n1 = _oracle_sample(CPU_SAMPLE, CPU_ITERS, 1)
    vn, sn, nn = _oracle_sample(CPU_SAMPLE, CPU_ITERS, cores)
    sample = (f"SDPs {CPU_SAMPLE[0]}, {CPU_SAMPLE[1]}, ..., {CPU_SAMPLE[-1]} of the batch (every 32nd), "
              f"{CPU_ITERS} iterations of the FP64 oracle (Algorithm 1, adaptive rho) each; setup excluded")
    return {"value": vn, "unit": "SDP-iters/s", "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": sn, "single_thread": {"value": v1, "cores": 1, "seconds": s1},
            "host_cores": os.cpu_count()}


def run_reference(args):
    """--impl reference: the FP64 oracle on the machine's host cores, each step one
    bounded sample of the batch (8 of its SDPs, 4 iterations each, one
    process per SDP); same metric and unit as the GPU arm."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = min(len(CPU_SAMPLE), os.cpu_count() or 1)
    vals, secs, its = [], [], []
    for s in range(args.warmup + args.steps):
        v, sec, n = _oracle_sample(CPU_SAMPLE, CPU_ITERS, cores)
        if s >= args.warmup:
            vals.append(v); secs.append(sec); its.append(n)
    value = sum(its) / sum(secs)
    sample = (f"SDPs {CPU_SAMPLE[0]}, {CPU_SAMPLE[1]}, ..., {CPU_SAMPLE[-1]} of the batch, {CPU_ITERS} iterations "
              f"of the FP64 oracle each per step, {cores} processes")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "SDP-iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "primal", "rho": "adaptive every iteration", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "SDP-iters/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "SDP-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- multi-rank helpers ----------------------------------------------------------

def aggregate_over_ranks(torch, dist, world, total_ms, total_iters, device):
    """Whole-job rate of N ranks: iterations summed over ranks divided by the
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


# ---- sub-blocks ----------------------------------------------------------------

def _event_ms(torch, stream, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def _parity_vs_oracle(P, parts, members):
    """Objective of each stored oracle summand in the last solve against the
    oracle's objective at the same iteration (tests/golden/batch_oracle.json)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "batch_oracle.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = [g for g in json.load(f)["results"] if g["form"] == "primal"]
    X, _, _ = P.results()
    r, c = P.pattern()
    it, st, res = P.component_results()
    index = {}
    vo = np.concatenate([[0], np.cumsum([q.n for q in parts])])
    out = []
    for g in gold:
        j = g["summand"]
        if j not in members:
            continue
        k = members.index(j)
        q = parts[k]
        mask = (c >= vo[k]) & (c < vo[k + 1])
        rr, cc = r[mask] - vo[k], c[mask] - vo[k]
        index = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(rr, cc))}
        cvec = np.zeros(len(rr))
        for a, b, v in zip(q.C_row, q.C_col, q.C_val):
            cvec[index[(int(a), int(b))]] += v
        obj = float(np.sum(np.where(rr == cc, 1.0, 2.0) * cvec * X[mask]))
        want = g["objective"][min(int(it[k]), len(g["objective"])) - 1]
        out.append({"summand": j, "iters": int(it[k]), "oracle_iters": g["iters"],
                    "rel_objective_gap": abs(obj - want) / abs(want), "residuals": [float(res[k, 0]), float(res[k, 1])]})
    return out


def _hsde_batch(cdsdp, parts, members, torch, flush, stream):
    """Algorithm 3 on the batch, each SDP scaled alone (Section 7.1.3, 4
    equilibration passes) and embedded alone: one FP32 graph solve to
    eps = 1e-4 from the cold start (every SDP stops on its own test), CUDA
    events; parity of three summands against stored oracle solves of each
    summand scaled alone (tests/golden/batch_hsde_scaled_oracle.json)."""
    import numpy as np
    t0 = time.perf_counter()
    Q = cdsdp.Problem.batch(parts, scale_passes=4)
    setup_s = time.perf_counter() - t0
    Q.bind(max_iter=40000)
    flush.fill_(1)
    ms, out = _event_ms(torch, stream, lambda: Q.solve("hsde", outputs=True, eps=1e-4, max_iter=40000,
                                                       precision="fp32", use_graph=1))
    it, st, res = Q.component_results()
    block = {"workload": "the batch, each SDP scaled alone (4 passes), one embedding per SDP", "setup_s": setup_s,
             "time_to_eps_ms": ms, "iters_to_eps_max": int(out["iters"]), "sdp_iters": int(it.sum()),
             "sdp_iters_per_s": float(it.sum()) / (ms / 1e3), "all_solved": bool(np.all(st == 0)),
             "ms_per_iteration_mean": ms / max(1, int(out["iters"]))}
    path = os.path.join(ROOT, "tests", "golden", "batch_hsde_scaled_oracle.json")
    if os.path.exists(path):
        with open(path) as f:
            gold = json.load(f)["results"]
        r, c = Q.pattern()
        vo = np.concatenate([[0], np.cumsum([q.n for q in parts])])
        par = []
        for g in gold:
            j = g["summand"]
            if j not in members:
                continue
            k = members.index(j)
            q = parts[k]
            mask = (c >= vo[k]) & (c < vo[k + 1])
            rr, cc = r[mask] - vo[k], c[mask] - vo[k]
            index = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(rr, cc))}
            cvec = np.zeros(len(rr))
            for a, b, v in zip(q.C_row, q.C_col, q.C_val):
                cvec[index[(int(a), int(b))]] += v
            obj = float(np.sum(np.where(rr == cc, 1.0, 2.0) * cvec * out["X"][mask]))
            par.append({"summand": j, "iters": int(it[k]), "oracle_iters": g["iters"],
                        "rel_objective_gap": abs(obj - g["objective"]) / abs(g["objective"]),
                        "residuals": [float(res[k, 0]), float(res[k, 1])]})
        block["parity_vs_oracle"] = par
    del Q
    return block


def _affine_sweep():
    """The affine projection against m (block-arrow l=100, d=10, h=20, A_i
    dense on the pattern, the smallest and largest m of the paper's
    affine-projection table): affine and projection ms per iteration of a
    profiled 50-iteration solve per form with the cached inverse, and of
    Algorithms 1-2 with 5 conjugate-gradient steps per iteration instead."""
    from paper_1707_05058_gb300 import affine_sweep
    rows = affine_sweep.sweep_rows([200, 1000], 50)
    cg = affine_sweep.sweep_rows([200, 1000], 50, forms=("primal", "dual"), cg=True, cg_steps=5)
    out = []
    for r, c in zip(rows, cg):
        out.append({"m": r["m"], "nnz_A": r["nnz_A"], "cliques": r["cliques"],
                    "affine_ms_per_iter": {f: r[f]["affine_ms_per_iter"] for f in ("primal", "dual", "hsde")},
                    "proj_ms_per_iter": r["primal"]["proj_ms_per_iter"],
                    "hsde_over_primal_affine": r["hsde_over_primal_affine"],
                    "cg5_affine_ms_per_iter": {f: c[f]["affine_ms_per_iter"] for f in ("primal", "dual")}})
    return out


def _dense_sample(cdsdp, workloads, torch, flush, stream):
    """Eight SDPs of the batch (every 32nd) with every A_i dense on the
    block-arrow pattern (the batch's shapes at full density; the whole batch
    at that density would hold 2.2e9 nonzeros).  FP32 graph ms per
    iteration with every SDP active; a profiled 50-iteration solve splits it
    into the projection and the rest (scatter, A W t, cached inverse, x
    update, stopping tests), whose algorithmic bytes (A W and A^T streamed
    once each, 12 B a nonzero, and the cached inverse blocks once, 8 B an
    entry) give its GB/s; one solve to eps = 1e-4 from the cold start."""
    members = list(range(0, 256, 32))
    t0 = time.perf_counter()
    parts = [workloads.block_arrow_batch_member(256, 3707, j, density=None) for j in members]
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    Q = cdsdp.Problem.batch(parts)
    setup_s = time.perf_counter() - t0
    Q.bind(max_iter=10000)
    info = Q.info
    KWD = dict(precision="fp32", adaptive_rho=1)
    tuned, _ = Q.autotune("primal", iters=20, **KWD)
    flush.fill_(1)
    ms, out = _event_ms(torch, stream, lambda: Q.solve("primal", outputs=False, eps=0.0, max_iter=50, use_graph=1,
                                                       **KWD, **tuned))
    Q.solve("primal", outputs=False, eps=0.0, max_iter=50, profile=1, check_every=50, **KWD,
            **{**tuned, "proj_streams": 1})
    proj_ms, launches, iter_ms = Q.profile()
    affine_ms = (iter_ms - proj_ms) / launches
    nnz, m = int(info["nnz_A"]), int(info["m"])
    inv_doubles = sum(int(q.m) ** 2 for q in parts)
    bytes_affine = 2 * nnz * 12 + inv_doubles * 8
    flush.fill_(1)
    tms, tout = _event_ms(torch, stream, lambda: Q.solve("primal", outputs=False, eps=1e-4, max_iter=10000,
                                                         use_graph=1, **KWD, **tuned))
    it, st, _ = Q.component_results()
    hbm = _peaks().get("hbm_gbs")
    block = {"workload": "SDPs 0, 32, ..., 224 of the batch with A_i dense on the pattern", "sdps": len(parts),
             "n": int(info["n"]), "m": m, "nnz_A": nnz, "generate_s": gen_s, "setup_s": setup_s,
             "upload_bytes": int(info["upload_bytes"]), "schedule": tuned,
             "fp32_graph_ms_per_iter": ms / out["iters"],
             "profiled": {"proj_ms_per_iter": proj_ms / launches, "rest_ms_per_iter": affine_ms,
                          "rest_algorithmic_bytes": bytes_affine,
                          "rest_gbs": bytes_affine / (affine_ms / 1e3) / 1e9,
                          "rest_frac_of_hbm": (bytes_affine / (affine_ms / 1e3) / 1e9) / hbm if hbm else None},
             "time_to_eps_ms": tms, "iters_to_eps_max": int(tout["iters"]), "sdp_iters": int(it.sum()),
             "all_solved": bool((st == 0).all())}
    del Q
    return block


def _banded(cdsdp, workloads, torch, flush, stream):
    """Banded n=2000, w=10, m=500: time to eps = 1e-4 (adaptive penalty every
    iteration) in the FP32 graph form (autotuned schedule) and the plain FP64
    form, and ADMM iterations/s of both."""
    prob = workloads.workload(1)
    P = cdsdp.Problem(prob).bind(max_iter=40000)
    tuned, _ = P.autotune("primal", iters=30, precision="fp32", adaptive_rho=1)

    def run(n, **kw):
        ms, its = [], []
        for _ in range(n):
            flush.fill_(1)
            t, out = _event_ms(torch, stream, lambda: P.solve("primal", outputs=False, eps=1e-4, max_iter=40000,
                                                              adaptive_rho=1, **kw))
            assert out["status"] == 0, out
            ms.append(t); its.append(out["iters"])
        return ms, its
    run(2, precision="fp32", use_graph=1, **tuned)
    ms32, it32 = run(5, precision="fp32", use_graph=1, **tuned)
    ms64, it64 = run(1, precision="fp64", use_graph=0, check_every=10, warm_start=0)
    P.solve("primal", outputs=False, eps=1e-4, max_iter=40000, precision="fp32", profile=1, check_every=50,
            adaptive_rho=1, **tuned)
    cls = P.profile_orders()
    top = max(cls, key=lambda c: c["ms"])
    return {"workload": BANDED, "cliques": int(P.info["p"]), "clique_order": int(P.info["max_clique"]),
            "fp32_graph": {"time_to_eps_ms": statistics.median(ms32), "iters": int(statistics.median(it32)),
                           "iters_per_s": sum(it32) / (sum(ms32) / 1e3)},
            "fp64_plain": {"time_to_eps_ms": ms64[0], "iters": it64[0], "iters_per_s": it64[0] / (ms64[0] / 1e3),
                           "form": "float64 everywhere, cold Jacobi, one launch per phase, no graph"},
            "speedup_time_to_eps": ms64[0] / statistics.median(ms32), "schedule": tuned,
            "projection": {"order": top["order"], "ms_per_launch": top["ms"] / top["launches"],
                           "nominal_gflops": top["nominal_flops"] / (top["ms"] / top["launches"] / 1e3) / 1e9}}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _maxcut(cdsdp, workloads, torch, flush, stream, max_iter=2500):
    """MaxCut relaxation on G(n, 6/(n-1)), n = 10^4 (weights U(0,1), C = -L/4,
    diag(X) = 1): minimum-degree extension, cliques merged
    (CDSDP_SETUP_MERGE_CLIQUES).  Clique-order histogram; a profiled run of 10
    iterations (the step of the cliques above order 128 on the tensor cores
    against the rest); Algorithm 1 in the FP32 form with the adaptive penalty
    to eps = 1e-4 within max_iter iterations."""
    import numpy as np
    prob = workloads.workload(3)
    t0 = time.perf_counter()
    P = cdsdp.Problem(prob, merge_cliques=True)
    setup_s = time.perf_counter() - t0
    P.bind(max_iter=max_iter)
    sizes = np.diff(P.cliques()[0])
    edges = [1, 17, 33, 65, 129, 513, 2049, 1 << 20]
    hist = {f"{lo}-{hi - 1}": int(np.sum((sizes >= lo) & (sizes < hi))) for lo, hi in zip(edges[:-1], edges[1:])}
    P.solve("primal", outputs=False, eps=0.0, max_iter=10, precision="fp32", profile=1, check_every=10, adaptive_rho=1)
    proj_ms, launches, iter_ms = P.profile()
    lg = P.profile_large()
    lg_ms = lg["ms"] / max(1, lg["launches"])
    tensor_tflops = lg["tensor_flops"] / (lg_ms / 1e3) / 1e12
    pk = _peaks()
    tf32_peak = pk.get("bf16_tflops", 1910.0) * (1.1 / 2.25)  # nominal tf32 / bf16 dense ratio
    flush.fill_(1)
    ms, out = _event_ms(torch, stream, lambda: P.solve("primal", outputs=False, eps=1e-4, max_iter=max_iter,
                                                       precision="fp32", adaptive_rho=1))
    return {"workload": "maxcut_gnp_n10000_deg6, cliques merged", "n": int(P.info["n"]), "m": int(P.info["m"]),
            "cliques": int(P.info["p"]), "clique_order_max": int(P.info["max_clique"]), "clique_histogram": hist,
            "n_d_lower": int(P.info["n_d_lower"]), "components": int(P.info["ncomp"]), "setup_s": setup_s,
            "ms_per_iter": iter_ms / launches, "proj_ms_per_iter": proj_ms / launches,
            "large_cliques": lg["cliques"], "large_step_ms_per_iter": lg_ms,
            "tensor_roofline": {"bound": "tensor", "achieved": tensor_tflops, "peak": tf32_peak, "unit": "TFLOP/s",
                                "frac": tensor_tflops / tf32_peak,
                                "peak_source": "measured bf16 burst (MEASURED_PEAKS.json) x nominal tf32/bf16 ratio",
                                "work": "59 products x 3 TF32 MMAs over the lower 128x128 tiles per step"},
            "fp32_primal": {"status": int(out["status"]), "iters": int(out["iters"]), "ms": ms, "max_iter": max_iter}}


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
                t, _ = _event_ms(torch, stream, lambda: P.complete(X, dense=dense, stream=stream, scratch=scratch,
                                                                   out=Wd))
                ms.append(t)
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
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the banded, MaxCut, gradient and completion blocks")
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

    t0 = time.perf_counter()
    allparts = workloads.workload(2)
    members = batch_shard(list(range(len(allparts))), rank, world)
    parts = [allparts[j] for j in members]
    prob = workloads.direct_sum(parts)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    P = cdsdp.Problem(prob)
    setup_s = time.perf_counter() - t0
    max_iter = 10000
    P.bind(max_iter=max_iter)
    info = P.info
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peak32 = cdsdp.fma_peak("fp32")
    peak64 = cdsdp.fma_peak("fp64")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ADAPT = dict(adaptive_rho=1)
    TUNED, tune_ms = P.autotune("primal", iters=20, precision="fp32", **ADAPT)
    KW = dict(eps=1e-4, max_iter=max_iter, precision="fp32", use_graph=1, **ADAPT, **TUNED)

    def solve_step():
        flush.fill_(1)
        ms, out = _event_ms(torch, stream, lambda: P.solve("primal", outputs=False, **KW))
        it, st, _ = P.component_results()
        assert out["status"] == 0 and np.all(st == 0), (out, int(np.sum(st != 0)))
        return ms, int(it.sum()), int(out["iters"])

    # ---- FP32-projection form, one graph per solve (the headline value)
    for _ in range(args.warmup):
        solve_step()
    barrier()
    clk = _clock_sampler(torch.cuda.current_device()) if rank == 0 else None
    steps = [solve_step() for _ in range(args.steps)]
    barrier()
    clocks = _clock_summary(clk) if rank == 0 else None
    ms_steps = [s[0] for s in steps]
    sdp_iters = [s[1] for s in steps]
    value, _, _ = aggregate_over_ranks(torch, dist, world, sum(ms_steps), sum(sdp_iters), "cuda")
    parity = _parity_vs_oracle(P, parts, members)

    # ---- ms per iteration with every SDP active: precision, warm start and graph apart
    def per_iter(n, **kw):
        flush.fill_(1)
        ms, out = _event_ms(torch, stream, lambda: P.solve("primal", outputs=False, eps=0.0, max_iter=n, **ADAPT,
                                                           **kw))
        return ms / out["iters"]
    pit = {"fp32_graph": per_iter(50, precision="fp32", use_graph=1, **TUNED),
           "fp32_plain": per_iter(20, precision="fp32", use_graph=0, check_every=20, **TUNED),
           "fp64_plain_cold_jacobi": per_iter(10, precision="fp64", use_graph=0, check_every=10, warm_start=0),
           "fp64_plain_warm_jacobi": per_iter(10, precision="fp64", use_graph=0, check_every=10, warm_start=16),
           "fp64_graph_warm_jacobi": per_iter(20, precision="fp64", use_graph=1, warm_start=16)}
    pit["ratio_fp64_plain_cold_vs_fp32_graph"] = pit["fp64_plain_cold_jacobi"] / pit["fp32_graph"]
    pit["ratio_fp64_graph_warm_vs_fp32_graph"] = pit["fp64_graph_warm_jacobi"] / pit["fp32_graph"]

    # ---- profiled FP32 solve: per size class, launch durations from CUDA events,
    # classes one after the other on the solve's stream (proj_streams = 1) so that
    # each launch is timed alone; 200 iterations from the cold start
    P.solve("primal", outputs=False, eps=0.0, max_iter=PROFILE_ITERS, precision="fp32", profile=1,
            check_every=PROFILE_ITERS, **ADAPT, **{**TUNED, "proj_streams": 1})
    proj_ms, proj_launches, iter_ms = P.profile()
    cls = P.profile_orders()
    top = max(cls, key=lambda c: c["ms"])
    top_launch_ms = top["ms"] / top["launches"]
    top_tflops = top["nominal_flops"] / (top_launch_ms / 1e3) / 1e12
    all_flops = sum(c["nominal_flops"] for c in cls)
    proj_gflops = all_flops / (proj_ms / proj_launches / 1e3) / 1e9

    # ---- end to end through the public API from host arrays
    e2e_ms, e2e_it, parts_ms = [], [], {"setup": [], "bind_upload": [], "solve_download": []}
    h2d = d2h = 0
    for s in range(2):
        torch.cuda.synchronize()
        t = time.perf_counter()
        Q = cdsdp.Problem.batch(parts)
        t1 = time.perf_counter()
        Q.bind(max_iter=max_iter)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out = Q.solve("primal", **KW)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        it, st, _ = Q.component_results()
        e2e_ms.append((t3 - t) * 1e3)
        e2e_it.append(int(it.sum()))
        parts_ms["setup"].append((t1 - t) * 1e3)
        parts_ms["bind_upload"].append((t2 - t1) * 1e3)
        parts_ms["solve_download"].append((t3 - t2) * 1e3)
        nz = int(Q.info["nnz_pattern"])
        h2d = int(Q.info["upload_bytes"])
        d2h = (2 * nz + int(Q.info["m"])) * 8 + int(out["iters"]) * 8 * 8
        del Q
    e2e_value = sum(e2e_it) / (sum(e2e_ms) / 1e3)
    del P

    extras = {}
    if not args.no_extras:
        extras["hsde"] = _hsde_batch(cdsdp, parts, members, torch, flush, stream)
        extras["banded"] = _banded(cdsdp, workloads, torch, flush, stream)
        extras["affine_sweep"] = _affine_sweep()
        extras["dense_sample"] = _dense_sample(cdsdp, workloads, torch, flush, stream)
        extras["maxcut"] = _maxcut(cdsdp, workloads, torch, flush, stream)
        extras["grad"] = _grad_batch(cdsdp, workloads, torch, stream)
        extras["completion"] = _completion(cdsdp, workloads, torch, stream)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            try:
                cpu = _cpu_baseline_block()
            except Exception as exc:  # report, do not hide
                cpu = {"value": None, "unit": "SDP-iters/s", "cores": None, "kind": "oracle",
                       "sample": f"failed: {exc}"}
        sm_mhz = (clocks or {}).get("sm_mhz")
        iters_max = [s[2] for s in steps]
        nclass = len(cls)
        launches_per_iter = 3 + nclass + 1 + (1 if TUNED.get("x_update") == 2 else 0)
        traffic = None
        if KERNEL_TRAFFIC_BYTES is not None:
            traffic = KERNEL_TRAFFIC_BYTES
        line = {
            "metric": METRIC, "value": value, "unit": "SDP-iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms_steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "primal (Algorithm 1)", "eps": 1e-4, "sdps": len(parts),
                       "n": int(info["n"]), "m": int(info["m"]), "cliques": int(info["p"]),
                       "clique_order_max": int(info["max_clique"]), "nnz_A": int(info["nnz_A"]),
                       "rho": "adaptive (Section 7.1.2) every iteration, mu 2, nu 10, from rho = 1, per SDP",
                       "precision": "fp32 eigensolve, rebuild and clique state; fp64 affine step, reductions",
                       "l2": "workspace (5.8 GB) larger than L2; L2 also flushed (256 MiB write) before every step",
                       "parallelism": f"{world} ranks, SDPs sharded (every {world}th)" if world > 1 else "single"},
            "time_to_eps_ms": statistics.median(ms_steps), "iters_to_eps_max": int(statistics.median(iters_max)),
            "sdp_iters_per_step": int(statistics.median(sdp_iters)),
            "per_iteration_ms_all_active": pit,
            "schedule": TUNED, "autotune_ms_per_iter": tune_ms,
            "parity_vs_oracle": parity,
            "clique_proj_gflops": proj_gflops, "proj_ms_per_iter": proj_ms / proj_launches,
            "proj_share_of_iteration": proj_ms / iter_ms,
            "projection_classes": cls,
            "generate_s": gen_s, "setup_s": setup_s,
            "roofline": {"bound": "alu", "achieved": top_tflops, "peak": peak32, "unit": "TFLOP/s",
                         "frac": top_tflops / peak32, "traffic": traffic,
                         "kernel": f"projection of padded order {top['order']} ({top['cliques']} cliques)",
                         "peak_source": "measured on this GPU: cdsdp_fma_peak, float FMA chains on every SM",
                         "flops_per_launch_nominal": top["nominal_flops"], "launch_ms": top_launch_ms,
                         "fp64_fma_peak_tflops": peak64, "sm_mhz_during_steps": sm_mhz},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "SDP-iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms), "steps": len(e2e_ms),
                    "breakdown_ms": {k: statistics.median(v) for k, v in parts_ms.items()}},
            "gpu_launches": sum(iters_max) * launches_per_iter + len(iters_max),
            "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
