"""Conjugate-gradient affine step (Section 4.1.1) on the GPU against the
oracle's CG form of Algorithm 1 (oracle/admm.py, linear_solver = ("cg", tol,
steps)): the same residual history and solution; bad options and HSDE are
refused."""
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


def _compare(dp, ref, out, rtol=1e-8):
    assert out["status"] == ref.status
    assert abs(out["iters"] - ref.iters) <= 1
    k = min(out["iters"], ref.iters, 50)
    np.testing.assert_allclose(out["hist"][:k, :6], ref.hist[:k, :6], rtol=rtol, atol=1e-10)
    for name, a, b in (("X", out["X"], dp.lower_values(ref.X)), ("Z", out["Z"], dp.lower_values(ref.Z)),
                       ("y", out["y"], ref.y)):
        assert np.abs(a - b).max() <= 1e-7 * max(1.0, np.abs(b).max()), name


def test_tight_cg_matches_oracle(lib, torch_cuda):
    """Block-arrow l=5, d=10, h=5, m=30, Algorithm 1 in FP64 through the CUDA
    graph: CG to 1e-14 with up to m steps gives the oracle's trajectory."""
    prob = W.workload(0)
    dp, ref = admm.solve(prob, "primal", eps=1e-5, max_iter=3000, linear_solver=("cg", 1e-14, 30))
    P = lib.Problem(prob).bind(max_iter=3000)
    out = P.solve("primal", eps=1e-5, max_iter=3000, precision="fp64", use_graph=1, check_every=7,
                  linear_solver=1, cg_tol=1e-14, cg_max_steps=30)
    _compare(dp, ref, out)


def test_cg_options_are_checked(lib, torch_cuda):
    P = lib.Problem(W.workload(0)).bind(max_iter=100)
    with pytest.raises(lib.CdsdpError) as ex:
        P.solve("hsde", max_iter=100, linear_solver=1)
    assert ex.value.status == -8  # CDSDP_ERR_UNSUPPORTED
    for bad in (dict(linear_solver=2), dict(linear_solver=1, cg_max_steps=2000), dict(linear_solver=1, cg_tol=-1.0)):
        with pytest.raises(lib.CdsdpError) as ex:
            P.solve("primal", max_iter=100, **bad)
        assert ex.value.status == -1  # CDSDP_ERR_ARG


def test_tight_cg_dual_matches_oracle(lib, torch_cuda):
    """Algorithm 2 with the CG affine step (the same system A D^-1 A^T, Section
    4.2), FP64, through the CUDA graph."""
    prob = W.workload(0)
    dp, ref = admm.solve(prob, "dual", eps=1e-5, max_iter=3000, linear_solver=("cg", 1e-14, 30))
    P = lib.Problem(prob).bind(max_iter=3000)
    out = P.solve("dual", eps=1e-5, max_iter=3000, precision="fp64", use_graph=1, check_every=7,
                  linear_solver=1, cg_tol=1e-14, cg_max_steps=30)
    _compare(dp, ref, out)


def test_tight_cg_plain_launches(lib, torch_cuda):
    """The same with one launch per kernel (no graph): the host polls the stop
    flag every 9 iterations, the extra launches return at once."""
    prob = W.workload(0)
    dp, ref = admm.solve(prob, "primal", eps=1e-5, max_iter=3000, linear_solver=("cg", 1e-14, 30))
    P = lib.Problem(prob).bind(max_iter=3000)
    out = P.solve("primal", eps=1e-5, max_iter=3000, precision="fp64", use_graph=0, check_every=9,
                  linear_solver=1, cg_tol=1e-14, cg_max_steps=30)
    _compare(dp, ref, out)


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_one_cg_step_per_iteration(lib, torch_cuda, form):
    """One warm-started CG step per ADMM iteration (tolerance 0): an inexact
    affine step whose iterates the oracle's CG form reproduces step for step
    (first 200 iterations)."""
    prob = W.banded(60, 4, 15, seed=11, density=0.3)
    dp = admm.decompose(prob)
    fn = admm.primal_admm if form == "primal" else admm.dual_admm
    ref = fn(dp, eps=0.0, max_iter=200, linear_solver=("cg", 0.0, 1))
    P = lib.Problem(prob).bind(max_iter=200)
    out = P.solve(form, eps=0.0, max_iter=200, precision="fp64", linear_solver=1, cg_tol=0.0, cg_max_steps=1)
    assert out["iters"] == 200
    np.testing.assert_allclose(out["hist"][:, :6], ref.hist[:, :6], rtol=1e-7, atol=1e-10)


def test_cg_direct_sum(lib, torch_cuda):
    """A direct sum of three SDPs with the CG step (one stopping test over the
    sum, the CG path's only mode) against the oracle's CG solve of the sum."""
    parts = [W.block_arrow(3, 4, 2, 6, seed=21), W.banded(15, 3, 7, seed=22, density=0.4),
             W.block_arrow(2, 5, 3, 9, seed=23, density=0.5)]
    prob = W.direct_sum(parts)
    dp, ref = admm.solve(prob, "primal", eps=1e-5, max_iter=5000, linear_solver=("cg", 1e-14, 40))
    P = lib.Problem(prob).bind(max_iter=5000)
    out = P.solve("primal", eps=1e-5, max_iter=5000, precision="fp64", linear_solver=1, cg_tol=1e-14,
                  cg_max_steps=40)
    _compare(dp, ref, out)


def test_cg_fp32_objective(lib, torch_cuda):
    """FP32 projections with the CG step: the objective at the GPU's stopping
    iteration within 1e-4 of the oracle's (FP64, CG) at that iteration."""
    prob = W.workload(0)
    P = lib.Problem(prob).bind(max_iter=3000)
    out = P.solve("primal", eps=1e-4, max_iter=3000, precision="fp32", linear_solver=1, cg_tol=1e-12,
                  cg_max_steps=30)
    assert out["status"] == 0
    dp = admm.decompose(prob)
    traj = admm.primal_admm(dp, eps=0.0, max_iter=out["iters"], linear_solver=("cg", 1e-12, 30))
    r, c = P.pattern()
    obj = float(np.sum(np.where(r == c, 1.0, 2.0) * dp.lower_values(dp.c) * out["X"]))
    assert abs(obj - traj.hist[-1, 4]) <= 1e-4 * abs(traj.hist[-1, 4])


def test_no_factor_handle_solves_with_cg(lib, torch_cuda):
    """A handle set up without the cached inverses (CDSDP_SETUP_NO_FACTOR) solves
    Algorithms 1-2 with the CG step and matches the oracle; paths that need the
    inverse are refused."""
    prob = W.workload(0)
    P = lib.Problem(prob, cache_factor=False).bind(max_iter=3000)
    assert P.info["cached_factor"] == 0
    for form in ("primal", "dual"):
        dp, ref = admm.solve(prob, form, eps=1e-5, max_iter=3000, linear_solver=("cg", 1e-14, 30))
        out = P.solve(form, eps=1e-5, max_iter=3000, precision="fp64", linear_solver=1, cg_tol=1e-14,
                      cg_max_steps=30)
        _compare(dp, ref, out)
    for form, kw in (("primal", dict(linear_solver=0)), ("hsde", {})):
        with pytest.raises(lib.CdsdpError) as ex:
            P.solve(form, max_iter=10, **kw)
        assert ex.value.status == -8
