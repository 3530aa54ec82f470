"""Cost of the affine projection against the number of constraints m
(Section 7.4 block-arrow workload with l=100 blocks of size d=10 and an arrow
of width h=20; the m values of the paper's affine-projection table).

    python -m paper_1707_05058_gb300.affine_sweep --m 200 409 699 1000 --iters 100
    python -m paper_1707_05058_gb300.affine_sweep --m 1000 --linear-solver cg --cg-steps 5

For each m: one synthetic block-arrow SDP (A_i dense on the pattern, seeded),
host setup, then for each form a warm-up solve and a profiled solve of
`iters` iterations with no early stop (one launch per phase, each iteration
and each projection launch bracketed by CUDA events on the solve's stream).
Per iteration: the projection launch time, and everything else in the
iteration (the affine projection of Eq. OptCondMinYPrimal / OptCondMinYDual,
or the HSDE elimination of Section 5, with its scatter and the stopping
sums).  One JSON line per m, then a table.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TABLE_M = [  # m values of the affine-projection table (Section 7.4)
    200, 239, 286, 342, 409, 489, 585, 699, 836, 1000]


def sweep_rows(ms, iters, precision="fp32", forms=("primal", "dual", "hsde"), cg=False, cg_steps=5, cg_tol=1e-10,
               verbose=False):
    """One dict per m: sizes, setup time and, per form, the affine and
    projection ms per iteration of a profiled `iters`-iteration solve."""
    import torch

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1707_05058_gb300 import cdsdp, workloads

    rows = []
    for m in ms:
        t0 = time.perf_counter()
        prob = workloads.block_arrow(100, 10, 20, m, seed=7000 + m, name=f"block_arrow_l100_d10_h20_m{m}")
        t1 = time.perf_counter()
        P = cdsdp.Problem(prob).bind(max_iter=max(iters, 20))
        t2 = time.perf_counter()
        row = {"m": m, "n": prob.n, "cliques": int(P.info["p"]), "clique_order": int(P.info["max_clique"]),
               "nnz_A": int(P.info["nnz_A"]), "generate_s": t1 - t0, "setup_s": t2 - t1}
        lin = dict(linear_solver=1, cg_max_steps=cg_steps, cg_tol=cg_tol) if cg else {}
        row["linear_solver"] = "cg, {} steps, tol {:g}".format(cg_steps, cg_tol) if cg else "cached inverse"
        for form in forms:
            P.solve(form, eps=0.0, max_iter=20, precision=precision, use_graph=0, check_every=20,
                    outputs=False, **lin)
            P.solve(form, eps=0.0, max_iter=iters, precision=precision, use_graph=0,
                    check_every=iters, outputs=False, profile=1, **lin)
            torch.cuda.synchronize()
            proj_ms, launches, iter_ms = P.profile()
            row[form] = {"affine_ms_per_iter": (iter_ms - proj_ms) / iters,
                         "proj_ms_per_iter": proj_ms / iters, "iter_ms": iter_ms / iters}
        if "primal" in row and "hsde" in row:
            row["hsde_over_primal_affine"] = row["hsde"]["affine_ms_per_iter"] / row["primal"]["affine_ms_per_iter"]
        if verbose:
            print(json.dumps(row), flush=True)
        rows.append(row)
        del P
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, nargs="+", default=TABLE_M)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--forms", nargs="+", default=["primal", "dual", "hsde"])
    ap.add_argument("--linear-solver", default="factor", choices=["factor", "cg"],
                    help="affine step of Algorithms 1-2: cached inverse or conjugate gradient (HSDE: factor only)")
    ap.add_argument("--cg-steps", type=int, default=5)
    ap.add_argument("--cg-tol", type=float, default=1e-10)
    args = ap.parse_args(argv)
    cg = args.linear_solver == "cg"
    if cg:
        args.forms = [f for f in args.forms if f != "hsde"]

    rows = sweep_rows(args.m, args.iters, args.precision, args.forms, cg, args.cg_steps, args.cg_tol, verbose=True)
    print("| m | " + " | ".join(f"{f} affine ms/it" for f in args.forms) + " | projection ms/it (primal) |")
    print("|---|" + "---|" * (len(args.forms) + 1))
    for r in rows:
        cells = [f"{r[f]['affine_ms_per_iter']:.4f}" for f in args.forms]
        pj = r[args.forms[0]]["proj_ms_per_iter"]
        print(f"| {r['m']} | " + " | ".join(cells) + f" | {pj:.4f} |")


if __name__ == "__main__":
    main()
