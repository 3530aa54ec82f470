"""The batched workload at full size: 256 uneven block-arrow SDPs (l in
[10, 100], d in [10, 40], h in [10, 20], m in [50, 400]) solved as one direct
sum in the FP32-projection form, CUDA graph, adaptive penalty every
iteration, eps = 1e-4, each SDP stopping on its own test (the configuration
the benchmark times).

Each SDP of a direct sum is solved as if alone (Section 2.1: the pattern,
the cliques and A D^-1 A^T split by summand), so any summand can be checked
against the oracle's solve of that summand alone.  tests/golden/
batch_oracle.json holds those solves for three summands (the smallest, one
with cliques of order 50, a median one), written by
tests/golden/make_batch_oracle.py from oracle/ only.  Checks per summand:
solved, iteration count within 5% (at least 3) of the oracle's, its own
stopping residuals <= 1e-4, and its objective <C, X> within 1e-4 (relative)
of the oracle's objective at the same iteration."""
import json
import os

import numpy as np
import pytest

from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_oracle.json")


@pytest.fixture(scope="module")
def batch(lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    parts = W.workload(2)
    P = lib.Problem(W.direct_sum(parts)).bind(max_iter=10000)
    r, c = P.pattern()
    return parts, P, r, c


def _objective_vector(P, prob, r, c):
    index = {(int(i), int(j)): e for e, (i, j) in enumerate(zip(r, c))}
    cvec = np.zeros(len(r))
    for i, j, v in zip(prob.C_row, prob.C_col, prob.C_val):
        cvec[index[(int(i), int(j))]] += v
    return np.where(r == c, 1.0, 2.0) * cvec


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_batch_full_size_fp32_per_summand(lib, batch, form):
    with open(GOLDEN) as f:
        gold = [g for g in json.load(f)["results"] if g["form"] == form]
    parts, P, r, c = batch
    out = P.solve(form, eps=1e-4, max_iter=10000, precision="fp32", use_graph=1, adaptive_rho=1)
    assert out["status"] == 0
    it, st, res = P.component_results()
    assert np.all(st == 0)
    wc = _objective_vector(P, W.direct_sum(parts), r, c)
    vo = np.concatenate([[0], np.cumsum([q.n for q in parts])])
    for g in gold:
        j = g["summand"]
        assert parts[j].n == g["n"] and parts[j].m == g["m"]
        assert g["status"] == 0
        assert abs(int(it[j]) - g["iters"]) <= max(3, 0.05 * g["iters"]), (j, it[j], g["iters"])
        assert max(res[j, 0], res[j, 1]) <= 1e-4, (j, res[j, :2])
        mask = (c >= vo[j]) & (c < vo[j + 1])
        obj = float(np.sum(wc[mask] * out["X"][mask]))
        want = g["objective"][min(int(it[j]), len(g["objective"])) - 1]
        assert abs(obj - want) <= 1e-4 * abs(want), (j, obj, want)


def test_batch_full_size_hsde_scaled_per_summand(lib):
    """Algorithm 3 on the full batch scaled as Section 7.1.3 describes (each
    SDP scaled alone, 4 equilibration passes), one embedding per SDP, FP32
    projections, CUDA graph, eps = 1e-4: every SDP solved; for the three
    summands of tests/golden/batch_hsde_scaled_oracle.json (the oracle's
    Algorithm 3 on each summand scaled alone) the iteration count is within
    5% (at least 3) of the oracle's, the summand's own stopping residuals are
    <= 1e-4 and its unscaled objectives <C, X> and b^T y are within 1e-4 of
    the oracle's."""
    with open(os.path.join(os.path.dirname(GOLDEN), "batch_hsde_scaled_oracle.json")) as f:
        gold = json.load(f)["results"]
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    parts = W.workload(2)
    P = lib.Problem.batch(parts, scale_passes=gold[0]["scale_passes"]).bind(max_iter=40000)
    out = P.solve("hsde", eps=1e-4, max_iter=40000, precision="fp32", use_graph=1)
    assert out["status"] == 0
    it, st, res = P.component_results()
    assert np.all(st == 0), int(np.sum(st != 0))
    r, c = P.pattern()
    wc = _objective_vector(P, W.direct_sum(parts), r, c)
    vo = np.concatenate([[0], np.cumsum([q.n for q in parts])])
    mo = np.concatenate([[0], np.cumsum([q.m for q in parts])])
    bvec = np.concatenate([q.b for q in parts])
    for g in gold:
        j = g["summand"]
        assert parts[j].n == g["n"] and g["status"] == 0
        assert abs(int(it[j]) - g["iters"]) <= max(3, 0.05 * g["iters"]), (j, it[j], g["iters"])
        assert max(res[j, 0], res[j, 1]) <= 1e-4, (j, res[j, :2])
        mask = (c >= vo[j]) & (c < vo[j + 1])
        obj = float(np.sum(wc[mask] * out["X"][mask]))
        bty = float(np.dot(bvec[mo[j]:mo[j + 1]], out["y"][mo[j]:mo[j + 1]]))
        assert abs(obj - g["objective"]) <= 1e-4 * abs(g["objective"]), (j, obj, g["objective"])
        assert abs(bty - g["bty"]) <= 1e-4 * abs(g["bty"]), (j, bty, g["bty"])
