"""Fixed-size solve for profilers (ncu launch lists and kernel captures).

    python -m paper_1707_05058_gb300.profile_case --workload banded --iters 20 --precision fp32

Runs `iters` iterations of one form of the solver on a named workload with one
launch per phase (no CUDA graph, so every kernel shows up individually) and
no early stop.  Workloads:
  banded        n=2000, half-bandwidth 10, m=500 (1990 cliques of order 11)
  block_arrow   l=5, d=10, h=5, m=30 (5 cliques of order 15)
  batched       direct sum of `--count` uneven block-arrow SDPs (l in [10,100],
                d in [10,40], h in [10,20], m in [50,400]; cliques of order
                20..60); --count 256 is the full batch
  maxcut        MaxCut relaxation on G(n, 6/(n-1)) with --n vertices (10^4 is
                the MaxCut workload), cliques merged; the cliques above order
                128 run the tensor-core sign iteration
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="banded", choices=["banded", "block_arrow", "batched", "maxcut"])
    ap.add_argument("--n", type=int, default=10000, help="vertices of the maxcut workload")
    ap.add_argument("--count", type=int, default=256, help="problems in the batched workload")
    ap.add_argument("--form", default="primal", choices=["primal", "dual", "hsde"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--x-update", type=int, default=0, choices=[0, 1, 2],
                    help="Algorithm 1: 0 automatic, 1 inside the projection gather, 2 separate kernel")
    ap.add_argument("--cta-kernel", type=int, default=1, choices=[0, 1],
                    help="float32 orders 36..64: 0 eigenvectors in shared memory, 1 in registers")
    args = ap.parse_args(argv)

    import torch

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1707_05058_gb300 import cdsdp, workloads

    merge = False
    if args.workload == "batched":
        prob = workloads.direct_sum(workloads.block_arrow_batch(args.count, 3707))
    elif args.workload == "maxcut":
        prob = workloads.workload(3) if args.n == 10000 else workloads.maxcut(args.n, 6, 4707 + args.n)
        merge = True
    else:
        prob = workloads.workload(1 if args.workload == "banded" else 0)
    P = cdsdp.Problem(prob, merge_cliques=merge).bind(max_iter=args.iters)
    out = P.solve(args.form, eps=0.0, max_iter=args.iters, precision=args.precision, use_graph=0,
                  check_every=args.iters, outputs=False, x_update=args.x_update, proj_cta_kernel=args.cta_kernel)
    torch.cuda.synchronize()
    print(f"{args.workload} {args.form} {args.precision}: {out['iters']} iterations, status {out['status']}")


if __name__ == "__main__":
    main()
