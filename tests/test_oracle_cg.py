"""Pins of the conjugate-gradient affine step (Section 4.1.1: an iterative
method in place of the cached factor of A D^-1 A^T), oracle/admm.py.

The CG routine is pinned by facts of exact arithmetic that a wrong step
breaks: termination in as many steps as S has distinct eigenvalues, the
solution of a dense SPD system, monotone decrease of the S-norm error, zero
steps from the exact solution.  The ADMM forms with CG are pinned by the
Cholesky forms (tight tolerance: same trajectory) and by closed-form optima
(loose tolerance, warm starts)."""
import math

import numpy as np
import pytest

from oracle import admm
from paper_1707_05058_gb300 import workloads as W


def _spd_with_spectrum(eigs, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(eigs), len(eigs))))
    return Q @ np.diag(eigs) @ Q.T


def test_terminates_in_number_of_distinct_eigenvalues():
    S = _spd_with_spectrum([1.0] * 10 + [4.0] * 15 + [9.0] * 5, 0)
    r = np.random.default_rng(1).standard_normal(30)
    y, k = admm.conjugate_gradient(lambda v: S @ v, r, np.zeros(30), 1e-12, 100)
    assert k <= 3
    np.testing.assert_allclose(S @ y, r, rtol=0, atol=1e-10 * np.linalg.norm(r))


def test_solves_dense_spd_system_with_monotone_error():
    rng = np.random.default_rng(2)
    G = rng.standard_normal((40, 40))
    S = G @ G.T + 0.5 * np.eye(40)
    r = rng.standard_normal(40)
    ystar = np.linalg.solve(S, r)
    y, k = admm.conjugate_gradient(lambda v: S @ v, r, np.zeros(40), 1e-13, 400)
    np.testing.assert_allclose(y, ystar, rtol=1e-8, atol=1e-10)
    errs = []
    for steps in range(0, 25):
        yk, _ = admm.conjugate_gradient(lambda v: S @ v, r, np.zeros(40), 0.0, steps)
        e = yk - ystar
        errs.append(float(e @ S @ e))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))


def test_warm_start_at_the_solution_takes_no_step():
    S = _spd_with_spectrum(np.linspace(1, 5, 12), 3)
    r = np.ones(12)
    ystar = np.linalg.solve(S, r)
    _, k = admm.conjugate_gradient(lambda v: S @ v, r, ystar, 1e-10, 50)
    assert k == 0


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_tight_cg_reproduces_the_cholesky_trajectory(form):
    prob = W.block_arrow(3, 4, 2, 6, seed=21)
    dp, ref = admm.solve(prob, form, eps=1e-6, max_iter=3000)
    _, cg = admm.solve(prob, form, eps=1e-6, max_iter=3000, linear_solver=("cg", 1e-14, 200))
    assert cg.status == ref.status == admm.SOLVED
    assert abs(cg.iters - ref.iters) <= 1
    k = min(cg.iters, ref.iters, 60)
    np.testing.assert_allclose(cg.hist[:k, :2], ref.hist[:k, :2], rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(cg.X, ref.X, rtol=0, atol=1e-7 * max(1.0, np.abs(ref.X).max()))
    assert max(cg.state["cg_steps"]) <= dp.m


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("prob", [W.lovasz_theta_cycle(5), W.lambda_max_tridiagonal(8, 1.0, 0.5)],
                         ids=lambda p: p.name)
def test_loose_warm_started_cg_reaches_the_closed_form(prob, form):
    """A few warm-started CG steps per iteration (relative tolerance 1e-8,
    at most 5 steps) still converge to the closed-form optimum."""
    dp, r = admm.solve(prob, form, eps=1e-8, max_iter=20000, linear_solver=("cg", 1e-8, 5))
    assert r.status == admm.SOLVED
    obj = float(dp.c @ r.X)
    assert abs(obj - prob.optimum) <= 1e-6 * max(1.0, abs(prob.optimum))
    if prob.name == "lovasz_theta_C5":
        assert abs(-obj - math.sqrt(5)) < 1e-6


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_one_warm_started_cg_step_per_iteration_reaches_the_optimum(form):
    """Truncated inner solves (one CG step per ADMM iteration, warm-started)
    on a block-arrow SDP whose A D^-1 A^T is dense: the same optimum as the
    Cholesky form, in about the same number of iterations."""
    prob = W.block_arrow(3, 4, 2, 6, seed=21)
    dp, ref = admm.solve(prob, form, eps=1e-8, max_iter=20000)
    _, cg = admm.solve(prob, form, eps=1e-8, max_iter=20000, linear_solver=("cg", 1e-10, 1))
    assert cg.status == ref.status == admm.SOLVED
    assert max(cg.state["cg_steps"]) == 1
    assert abs(cg.iters - ref.iters) <= 0.1 * ref.iters
    o_ref, o_cg = float(dp.c @ ref.X), float(dp.c @ cg.X)
    assert abs(o_cg - o_ref) <= 1e-8 * abs(o_ref)
