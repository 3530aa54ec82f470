"""GPU parity for batches of independent SDPs solved as one problem (a direct
sum, Section 2.1: its aggregate pattern is block diagonal, so the chordal
decomposition, A D^-1 A^T and every ADMM step split by summand).

With per-component stopping (the default) each summand's result must be the
oracle's solve of that summand alone: same status, iteration count within
one, same X, y, Z to 1e-7 (FP64).  With one global test, the result must be
the oracle's solve of the whole direct sum.  FP32 projections: every summand's
objective within 1e-4 of the FP64 oracle's (the workload's tolerance)."""
import dataclasses

import numpy as np
import pytest

from oracle import admm
from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _parts():
    return [W.block_arrow(3, 4, 2, 6, seed=21), W.banded(15, 3, 7, seed=22, density=0.4),
            W.lovasz_theta_cycle(5), W.block_arrow(2, 5, 3, 9, seed=23, density=0.5)]


_CACHE = {}


def _oracle(prob, form, eps, max_iter, adapt_every=0):
    key = (prob.name, form, eps, max_iter, adapt_every)
    if key not in _CACHE:
        _CACHE[key] = admm.solve(prob, form, eps=eps, max_iter=max_iter, adapt_every=adapt_every)
    return _CACHE[key]


def _close(a, b, tol, what):
    scale = max(1.0, np.abs(b).max())
    assert np.abs(a - b).max() <= tol * scale, what


def _check_components(P, out, parts, form, eps, max_iter, rows_perm=None, adapt_every=0):
    it, st, res = P.component_results()
    r, c = P.pattern()
    vo = mo = 0
    for j, q in enumerate(parts):
        dp, ref = _oracle(q, form, eps, max_iter, adapt_every)
        assert st[j] == ref.status, j
        assert abs(int(it[j]) - ref.iters) <= 1, (j, it[j], ref.iters)
        if it[j] == ref.iters:
            np.testing.assert_allclose(res[j, :3], ref.hist[ref.iters - 1, :3], rtol=1e-6, atol=1e-12)
        mask = (c >= vo) & (c < vo + q.n)
        rows = np.arange(mo, mo + q.m) if rows_perm is None else rows_perm[mo:mo + q.m]
        _close(out["X"][mask], dp.lower_values(ref.X), 1e-7, f"X[{j}]")
        _close(out["Z"][mask], dp.lower_values(ref.Z), 1e-7, f"Z[{j}]")
        _close(out["y"][rows], ref.y, 1e-7, f"y[{j}]")
        vo += q.n
        mo += q.m
    assert out["iters"] == int(it.max())
    assert out["status"] == 0


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("form", ["primal", "dual"])
def test_direct_sum_per_component_fp64(lib, torch_cuda, form, use_graph):
    parts = _parts()
    prob = W.direct_sum(parts)
    P = lib.Problem(prob).bind(max_iter=5000)
    assert P.info["ncomp"] == len(parts)
    out = P.solve(form, eps=1e-5, max_iter=5000, precision="fp64", use_graph=use_graph, check_every=13)
    _check_components(P, out, parts, form, 1e-5, 5000)
    # column 6 of the history counts the components still running
    h = out["hist"]
    assert h[0, 6] == len(parts) and h[-1, 6] == 0
    assert np.all(np.diff(h[:, 6]) <= 0)


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_direct_sum_per_component_adaptive_rho(lib, torch_cuda, form):
    """Adaptive penalty per component (every 3 iterations): each summand's
    penalty path and result equal the oracle's run of that summand alone."""
    parts = _parts()
    P = lib.Problem(W.direct_sum(parts)).bind(max_iter=5000)
    out = P.solve(form, eps=1e-5, max_iter=5000, precision="fp64", adaptive_rho=3)
    _check_components(P, out, parts, form, 1e-5, 5000, adapt_every=3)


def test_direct_sum_shuffled_constraints(lib, torch_cuda):
    """Constraints of the summands interleaved: the block-diagonal inverse is
    addressed through the constraint lists of each component."""
    parts = _parts()
    s = W.direct_sum(parts)
    perm = np.random.default_rng(3).permutation(s.m).astype(np.int32)  # new index of constraint i
    b = np.empty_like(s.b)
    b[perm] = s.b
    t = dataclasses.replace(s, A_con=perm[s.A_con], b=b, name=s.name + "_shuffled")
    P = lib.Problem(t).bind(max_iter=5000)
    out = P.solve("primal", eps=1e-5, max_iter=5000, precision="fp64")
    _check_components(P, out, parts, "primal", 1e-5, 5000, rows_perm=perm)


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_direct_sum_global_stop(lib, torch_cuda, form):
    """component_stop = 0: one stopping test over the whole direct sum, as the
    oracle runs it on the assembled problem."""
    prob = W.direct_sum(_parts())
    dp, ref = _oracle(prob, form, 1e-4, 5000)
    P = lib.Problem(prob).bind(max_iter=5000)
    out = P.solve(form, eps=1e-4, max_iter=5000, precision="fp64", component_stop=0)
    assert out["status"] == ref.status
    assert abs(out["iters"] - ref.iters) <= 1
    k = min(out["iters"], ref.iters, 50)
    np.testing.assert_allclose(out["hist"][:k, :6], ref.hist[:k, :6], rtol=1e-8, atol=1e-10)
    _close(out["X"], dp.lower_values(ref.X), 1e-7, "X")
    _close(out["y"], ref.y, 1e-7, "y")


def test_direct_sum_hsde_trajectory(lib, torch_cuda):
    """Algorithm 3 on a direct sum (tau and kappa are shared, so it is one
    problem with a block-diagonal inverse): the first 40 FP64 iterates equal
    the oracle's on the normalised instance."""
    prob = W.direct_sum(_parts())
    w = np.where(prob.C_row == prob.C_col, 1.0, 2.0)
    prob = dataclasses.replace(prob, C_val=prob.C_val / np.sqrt(np.sum(w * prob.C_val ** 2)),
                               b=prob.b / np.linalg.norm(prob.b), name=prob.name + "_normalised")
    dp = admm.decompose(prob)
    ref = admm.hsde_admm(dp, eps=0.0, max_iter=40)
    P = lib.Problem(prob).bind(max_iter=40)
    out = P.solve("hsde", eps=0.0, max_iter=40, precision="fp64", component_stop=0)
    assert out["iters"] == 40
    np.testing.assert_allclose(out["hist"][:, :6], ref.hist[:, :6], rtol=1e-7, atol=1e-10)


def _normalised(q):
    w = np.where(q.C_row == q.C_col, 1.0, 2.0)
    return dataclasses.replace(q, C_val=q.C_val / np.sqrt(np.sum(w * q.C_val ** 2)), b=q.b / np.linalg.norm(q.b),
                               name=q.name + "_normalised")


@pytest.mark.parametrize("use_graph", [1, 0])
def test_direct_sum_hsde_per_component(lib, torch_cuda, use_graph):
    """Algorithm 3 with one embedding per summand (component mode, the
    default for a direct sum): each summand stops on its own test, and its
    status, iteration count (within one) and X, y, Z equal the oracle's
    Algorithm 3 on that summand alone (FP64; data normalised as in the
    trajectory test above)."""
    parts = [_normalised(q) for q in _parts()]
    P = lib.Problem(W.direct_sum(parts)).bind(max_iter=5000)
    out = P.solve("hsde", eps=1e-4, max_iter=5000, precision="fp64", use_graph=use_graph, check_every=11)
    it, st, res = P.component_results()
    r, c = P.pattern()
    vo = mo = 0
    for j, q in enumerate(parts):
        dp, ref = admm.solve(q, "hsde", eps=1e-4, max_iter=5000)
        assert st[j] == ref.status == 0, (j, st[j], ref.status)
        assert abs(int(it[j]) - ref.iters) <= 1, (j, it[j], ref.iters)
        mask = (c >= vo) & (c < vo + q.n)
        _close(out["X"][mask], dp.lower_values(ref.X), 1e-6, f"X[{j}]")
        _close(out["Z"][mask], dp.lower_values(ref.Z), 1e-6, f"Z[{j}]")
        _close(out["y"][mo:mo + q.m], ref.y, 1e-6, f"y[{j}]")
        vo += q.n
        mo += q.m
    assert out["status"] == 0 and out["iters"] == int(it.max())


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_block_arrow_batch_fp32(lib, torch_cuda, form):
    """Three uneven block-arrow SDPs (cliques of order 36, 24 and 22, so both
    the warp-per-clique and the block-per-clique projections run) in one FP32
    solve, against the FP64 oracle's run of the same form on each summand.
    Near eps = 1e-4 the objective of these runs still moves by a few 1e-4
    (relative) from one iteration to the next, and float32 rounding can move
    the stopping iteration by a few, so the checks are: every summand solved,
    within 5% (at least 3) of the oracle's iteration count, and its objective
    within 1e-4 of the oracle's objective at the same iteration, for both
    forms."""
    parts = [W.block_arrow(2, 24, 12, 20, seed=91, density=0.3), W.block_arrow(2, 14, 10, 25, seed=92, density=0.3),
             W.block_arrow(3, 10, 12, 20, seed=93, density=0.3)]
    prob = W.direct_sum(parts)
    P = lib.Problem(prob).bind(max_iter=20000)
    assert P.info["ncomp"] == 3 and P.info["max_clique"] == 36
    out = P.solve(form, eps=1e-4, max_iter=20000, precision="fp32")
    it, st, res = P.component_results()
    assert np.all(st == 0) and out["status"] == 0
    r, c = P.pattern()
    wgt = np.where(r == c, 1.0, 2.0)
    cvec = np.zeros(len(r))
    index = {(int(i), int(j)): e for e, (i, j) in enumerate(zip(r, c))}
    for i, j, v in zip(prob.C_row, prob.C_col, prob.C_val):
        cvec[index[(int(i), int(j))]] += v
    vo = 0
    for j, q in enumerate(parts):
        dp, ref = _oracle(q, form, 1e-4, 20000)
        assert ref.status == 0
        assert abs(int(it[j]) - ref.iters) <= max(3, 0.05 * ref.iters), (j, it[j], ref.iters)
        _, traj = _oracle(q, form, 0.0, int(it[j]))
        mask = (c >= vo) & (c < vo + q.n)
        obj = float(np.sum(wgt[mask] * cvec[mask] * out["X"][mask]))
        want = float(traj.hist[-1, 4])
        assert abs(obj - want) <= 1e-4 * abs(want), (j, obj, want)
        vo += q.n
