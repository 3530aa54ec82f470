"""Write the oracle's solves of selected summands of the 256-SDP block-arrow
batch (the batched workload) to batch_oracle.json.

The oracle (Algorithms 1 and 2, FP64, adaptive penalty of Section 7.1.2
applied every iteration, eps = 1e-4) runs on each listed summand alone.  For
each (summand, form) the file keeps the iteration count, the status, the
objective <C, X> at every iteration (history column 4), the penalty path
(column 2) and the summand's size.  Only oracle/ and the seeded generators
are called; nothing comes from the CUDA library.

Summands: the one with the least projection work (index 135: l=11, d=16,
h=11, m=322), one with cliques of order 50 (index 118: l=13, d=37, h=13, m=99)
and a median one (index 254: l=91, d=18, h=15, m=348).

    python tests/golden/make_batch_oracle.py [--jobs N]
    python tests/golden/make_batch_oracle.py --banded   (banded_oracle.json)
    python tests/golden/make_batch_oracle.py --hsde-scaled
        (batch_hsde_scaled_oracle.json: Algorithm 3 to eps 1e-4 on each summand
        scaled as Section 7.1.3 describes, SCALE_PASSES equilibration passes;
        the eigendecomposition step from LAPACK, which a CPU test holds equal
        to the oracle's own Jacobi)
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_oracle.json")
SUMMANDS = [135, 118, 254]
FORMS = ["primal", "dual"]
SCALE_PASSES = 4


def _solve_hsde_scaled(j):
    """Algorithm 3 on summand j scaled alone, to eps = 1e-4; the unscaled
    objectives <C, X> and b^T y of its result."""
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import admm, scaling
    from paper_1707_05058_gb300 import workloads as W
    prob = W.workload_batch_member(2, j)
    sp, factors = scaling.scale_problem(prob, SCALE_PASSES)
    dp = admm.decompose(sp, eig="lapack")
    r = admm.hsde_admm(dp, eps=1e-4, max_iter=20000)
    X, y, Z = scaling.unscale(dp.lower, dp.lower_values(r.X), r.y, dp.lower_values(r.Z), factors)
    pos = {ij: k for k, ij in enumerate(dp.lower)}
    cx = sum(v * X[pos[(int(a), int(b))]] * (1.0 if a == b else 2.0) for a, b, v in zip(prob.C_row, prob.C_col, prob.C_val))
    return {"summand": j, "form": "hsde", "scale_passes": SCALE_PASSES, "n": int(prob.n), "m": int(prob.m),
            "iters": int(r.iters), "status": int(r.status), "hist_last": [float(v) for v in r.hist[-1, :6]],
            "objective": float(cx), "bty": float(np.dot(prob.b, y))}


def _solve(args):
    j, form = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import admm
    from paper_1707_05058_gb300 import workloads as W
    prob = W.workload_batch_member(2, j)
    dp = admm.decompose(prob)
    fn = admm.primal_admm if form == "primal" else admm.dual_admm
    r = fn(dp, eps=1e-4, max_iter=20000, adapt_every=1)
    out = {"summand": j, "form": form, "n": int(prob.n), "m": int(prob.m), "iters": int(r.iters),
           "status": int(r.status), "objective": [float(v) for v in r.hist[:, 4]],
           "rho": [float(v) for v in r.hist[:, 2]]}
    return out


def _banded():
    """The banded workload (n=2000, w=10, m=500): Algorithm 1, FP64, adaptive
    penalty every iteration, eps = 1e-4; objective path and the KKT
    residuals of the returned (X, y, Z) (primal and dual feasibility relative
    to 1 + ||b||, 1 + ||c||, and the relative duality gap)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import admm
    from paper_1707_05058_gb300 import workloads as W
    dp = admm.decompose(W.workload(1))
    r = admm.primal_admm(dp, eps=1e-4, max_iter=40000, adapt_every=1)
    rp = np.linalg.norm(dp.A @ r.X - dp.b) / (1 + np.linalg.norm(dp.b))
    rd = np.linalg.norm(dp.A.T @ r.y + r.Z - dp.c) / (1 + np.linalg.norm(dp.c))
    cx, by = dp.c @ r.X, dp.b @ r.y
    return {"workload": "banded_n2000_w10_m500", "form": "primal", "iters": int(r.iters), "status": int(r.status),
            "objective": [float(v) for v in r.hist[:, 4]], "rho": [float(v) for v in r.hist[:, 2]],
            "kkt": {"primal": float(rp), "dual": float(rd), "gap": float(abs(cx - by) / (1 + abs(cx) + abs(by)))}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=len(SUMMANDS) * len(FORMS))
    ap.add_argument("--banded", action="store_true", help="write banded_oracle.json instead")
    ap.add_argument("--hsde-scaled", action="store_true",
                    help="write batch_hsde_scaled_oracle.json (Algorithm 3 on the scaled summands) instead")
    a = ap.parse_args()
    if a.hsde_scaled:
        with mp.get_context("spawn").Pool(len(SUMMANDS)) as pool:
            res = pool.map(_solve_hsde_scaled, SUMMANDS)
        doc = {"what": "oracle solves (FP64) of Algorithm 3 of arXiv 1707.05058 to eps 1e-4 on summands of the "
                       "256-SDP block-arrow batch, each scaled alone (Section 7.1.3, 4 equilibration passes); "
                       "objectives of the unscaled result",
               "generator": "paper_1707_05058_gb300.workloads.workload_batch_member(2, index)", "results": res}
        with open(os.path.join(os.path.dirname(OUT), "batch_hsde_scaled_oracle.json"), "w") as f:
            json.dump(doc, f)
        return
    if a.banded:
        with open(os.path.join(os.path.dirname(OUT), "banded_oracle.json"), "w") as f:
            json.dump(_banded(), f)
        return
    tasks = [(j, f) for j in SUMMANDS for f in FORMS]
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        res = pool.map(_solve, tasks)
    doc = {"what": "oracle solves (FP64, adaptive rho every iteration, mu 2, nu 10, eps 1e-4) of summands of the "
                   "256-SDP block-arrow batch, each alone; Algorithms 1 and 2 of arXiv 1707.05058",
           "generator": "paper_1707_05058_gb300.workloads.workload_batch_member(2, index)",
           "results": res}
    with open(OUT, "w") as f:
        json.dump(doc, f)


if __name__ == "__main__":
    main()
