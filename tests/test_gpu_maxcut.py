"""MaxCut relaxations whose minimum-degree extensions have cliques above
order 128 (the case of the MaxCut workload, whose largest clique is 3,414,
or 3,560 merged): the FP32 form with the tensor-core projection for those
cliques and the warp / thread-block Jacobi for the rest, against the oracle's
solves stored in tests/golden/maxcut_oracle.json (written by
tests/golden/make_maxcut_oracle.py from oracle/ only).

  * n = 600, cliques as extended: 7 cliques of order 129..198 in one batch of
    the tile kernels;
  * n = 800, cliques merged: one clique of order 296.

Algorithm 1 (adaptive penalty every iteration) to eps = 1e-4: solved,
iteration count within 5% (at least 3) of the oracle's, the objective <C, X>
within 1e-4 (relative) of the oracle's at the same iteration.  Algorithm 3:
the first 300 iterations (one tau, kappa over these graphs' independent
components keeps it from 1e-4 in 5000 iterations, on both sides); the
objective c^T u_x / tau and b^T u_y / tau of iteration 300 within 1e-4 of the
oracle's, and its residuals within 10% (at least 1e-6 absolute)."""
import json
import os

import numpy as np
import pytest

from oracle import admm
from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "maxcut_oracle.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return {(g["n"], g["merge"], g["form"]): g for g in json.load(f)["results"]}


@pytest.mark.parametrize("form", ["primal", "hsde"])
@pytest.mark.parametrize("case", [(600, False), (800, True)], ids=["n600", "n800_merged"])
def test_maxcut_large_cliques_fp32(lib, gold, case, form):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, merge = case
    g = gold[(n, merge, form)]
    prob = W.maxcut(n, 6, 4707 + n, name=f"maxcut_n{n}")
    P = lib.Problem(prob, merge_cliques=merge).bind(max_iter=20000)
    assert P.info["max_clique"] == g["max_clique"] > 128
    if form == "hsde":
        # one embedding over the whole graph, as the oracle runs it
        out = P.solve("hsde", eps=0.0, max_iter=g["iters"], precision="fp32", component_stop=0)
        assert out["iters"] == g["iters"]
        h, want = out["hist"][-1], g["hist"][-1]
        for col in (4, 5):  # objective c^T x, b^T y
            assert abs(h[col] - want[col]) <= 1e-4 * abs(want[col]), (col, h[col], want[col])
        for col in (0, 1, 2, 3):  # eps_p, eps_d, eps_g, eps_c
            assert abs(h[col] - want[col]) <= max(1e-6, 0.1 * abs(want[col])), (col, h[col], want[col])
        return
    out = P.solve(form, eps=1e-4, max_iter=20000, precision="fp32", adaptive_rho=1)
    assert out["status"] == 0 and g["status"] == 0
    assert abs(out["iters"] - g["iters"]) <= max(3, 0.05 * g["iters"]), (out["iters"], g["iters"])
    dp = admm.decompose(prob, merge=merge, eig="lapack")
    r, c = P.pattern()
    obj = float(np.sum(np.where(r == c, 1.0, 2.0) * dp.lower_values(dp.c) * out["X"]))
    want = g["hist"][min(out["iters"], len(g["hist"])) - 1][4]
    assert abs(obj - want) <= 1e-4 * abs(want), (obj, want)
