"""Pins of the data scaling (Section 7.1.3, oracle/scaling.py): the transform
maps solutions to solutions exactly (an identity of the data, checked on random
points), the scaled solve recovers the closed-form optima, and scaled and
unscaled solves reach the same optimum."""
import math

import numpy as np
import pytest

from oracle import admm, scaling
from paper_1707_05058_gb300 import workloads as W


def _lower(dp):
    return dp.lower


def test_transform_is_an_identity_on_random_points():
    """<Abar_i, Xbar> = tau e_i <A_i, X> and Cbar - sum ybar_i Abar_i = sigma D Z D
    for a random X and y (full symmetric matrices)."""
    prob = W.block_arrow(3, 4, 2, 6, seed=5)
    sp, (d, e, tau, sigma) = scaling.scale_problem(prob, 6)
    rng = np.random.default_rng(0)
    n = prob.n
    X = rng.standard_normal((n, n)); X = X + X.T
    y = rng.standard_normal(prob.m)

    def mats(p):
        A = np.zeros((p.m, n, n))
        for k, i, j, v in zip(p.A_con, p.A_row, p.A_col, p.A_val):
            A[k, i, j] += v
            if i != j:
                A[k, j, i] += v
        C = np.zeros((n, n))
        for i, j, v in zip(p.C_row, p.C_col, p.C_val):
            C[i, j] += v
            if i != j:
                C[j, i] += v
        return A, C
    A, C = mats(prob)
    Ab, Cb = mats(sp)
    D = np.diag(d)
    Xb = tau * np.linalg.inv(D) @ X @ np.linalg.inv(D)
    np.testing.assert_allclose(np.einsum("kij,ij->k", Ab, Xb), tau * e * np.einsum("kij,ij->k", A, X), rtol=1e-12)
    yb = sigma * y / e
    Z = C - np.einsum("k,kij->ij", y, A)
    np.testing.assert_allclose(Cb - np.einsum("k,kij->ij", yb, Ab), sigma * D @ Z @ D, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(sp.b), 1.0)


def test_equilibration_brings_row_norms_together():
    prob = W.block_arrow(4, 5, 3, 12, seed=9)
    rng = np.random.default_rng(1)
    prob.A_val = prob.A_val * np.repeat(10.0 ** rng.uniform(-3, 3, prob.m), len(prob.A_val) // prob.m)
    w = np.where(prob.A_row == prob.A_col, 1.0, 2.0)

    def spread(p):
        rn = np.sqrt(np.bincount(p.A_con, weights=w * p.A_val ** 2, minlength=p.m))
        return rn.max() / rn.min()
    sp, _ = scaling.scale_problem(prob, 8)
    assert spread(prob) > 1e4 and spread(sp) < 10.0


@pytest.mark.parametrize("form", ["primal", "dual", "hsde"])
@pytest.mark.parametrize("prob", [W.lambda_max_tridiagonal(8, 1.0, 0.5), W.lovasz_theta_cycle(5), W.maxcut_cycle(5)],
                         ids=lambda p: p.name)
def test_scaled_solve_recovers_closed_forms(prob, form):
    sp, f = scaling.scale_problem(prob, 5)
    dp, r = admm.solve(sp, form, eps=1e-9, max_iter=40000)
    assert r.status == admm.SOLVED
    X, y, Z = scaling.unscale(dp.lower, dp.lower_values(r.X), r.y, dp.lower_values(r.Z), f)
    dpo = admm.decompose(prob)
    obj = float(np.sum(np.where(np.array([i == j for i, j in dpo.lower]), 1.0, 2.0) * dpo.lower_values(dpo.c) * X))
    assert abs(obj - prob.optimum) <= 1e-6 * max(1.0, abs(prob.optimum))


def test_scaled_and_unscaled_reach_the_same_optimum():
    prob = W.block_arrow(3, 4, 2, 6, seed=21)
    dpo, ro = admm.solve(prob, "primal", eps=1e-8, max_iter=20000)
    sp, f = scaling.scale_problem(prob, 5)
    dp, r = admm.solve(sp, "primal", eps=1e-8, max_iter=20000)
    X, y, Z = scaling.unscale(dp.lower, dp.lower_values(r.X), r.y, dp.lower_values(r.Z), f)
    w = np.where(np.array([i == j for i, j in dpo.lower]), 1.0, 2.0)
    o1 = float(dpo.c @ ro.X)
    o2 = float(np.sum(w * dpo.lower_values(dpo.c) * X))
    assert abs(o1 - o2) <= 1e-5 * abs(o1)
    np.testing.assert_allclose(y, ro.y, rtol=1e-3, atol=1e-3 * np.abs(ro.y).max())
