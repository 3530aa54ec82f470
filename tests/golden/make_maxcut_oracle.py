"""Write the oracle's solves of two scaled-down MaxCut relaxations (the MaxCut
workload's generator at n = 600 and n = 800; minimum-degree extensions with
cliques above order 128) to maxcut_oracle.json.

  * n = 600, cliques as extended (7 of order 129..198);
  * n = 800, cliques merged (CDSDP_SETUP_MERGE_CLIQUES rule; one of order 296).

For each: Algorithm 1 (FP64, adaptive penalty every iteration) to eps = 1e-4,
and the first 300 iterations of Algorithm 3 (whose single tau, kappa over the
graph's independent components keeps it from eps = 1e-4 within 5000
iterations on these instances).  The eigendecomposition step of the oracle's projection is
LAPACK's (oracle/psd.py, eig="lapack"): its own Jacobi is out of reach at
these orders.  Stored per run: iterations, status, and history columns 0-5
at every iteration.  Only oracle/ and the seeded generators are called.

    python tests/golden/make_maxcut_oracle.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "maxcut_oracle.json")
CASES = [(600, False), (800, True)]
SEED = 4707
HSDE_ITERS = 300


def _solve(args):
    n, merge, form = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import admm
    from paper_1707_05058_gb300 import workloads as W
    prob = W.maxcut(n, 6, SEED + n, name=f"maxcut_n{n}")
    dp = admm.decompose(prob, merge=merge, eig="lapack")
    if form == "primal":
        r = admm.primal_admm(dp, eps=1e-4, max_iter=20000, adapt_every=1)
    else:
        r = admm.hsde_admm(dp, eps=0.0, max_iter=HSDE_ITERS)
    return {"n": n, "merge": merge, "form": form, "iters": int(r.iters), "status": int(r.status),
            "max_clique": max(len(c) for c in dp.cliques), "hist": [[float(v) for v in row[:6]] for row in r.hist]}


def main():
    tasks = [(n, merge, form) for n, merge in CASES for form in ("primal", "hsde")]
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        res = pool.map(_solve, tasks)
    doc = {"what": "oracle runs (FP64) of MaxCut relaxations of G(n, 6/(n-1)) graphs: Algorithm 1 with adaptive "
                   "rho every iteration (mu 2, nu 10) to eps 1e-4; Algorithm 3 for 300 iterations; arXiv 1707.05058",
           "generator": "paper_1707_05058_gb300.workloads.maxcut(n, 6, 4707 + n)", "results": res}
    with open(OUT, "w") as f:
        json.dump(doc, f)


if __name__ == "__main__":
    main()
