"""Pins for the oracle's Algorithms 1-3 (CPU only): brute-force linear algebra,
closed-form optima, decomposition equivalence, KKT conditions and
infeasibility certificates."""
import math

import numpy as np
import pytest
import scipy.sparse

from oracle import admm
from paper_1707_05058_gb300 import workloads as W


def _dense_H(dp):
    return scipy.sparse.csr_matrix((np.ones(dp.nd), (np.arange(dp.nd), dp.hidx)), shape=(dp.nd, dp.N)).toarray()


def test_primal_x_step_is_the_kkt_solution():
    """The block elimination of Appendix A solves Eq. OptCondMinYPrimal: check
    it against a dense solve of the assembled KKT matrix [[D, A^T], [A, 0]]."""
    prob = W.random_chordal_small(7, 4, seed=1, extra_edges=4)
    dp = admm.decompose(prob)
    states = {}
    admm.primal_admm(dp, rho=1.3, eps=0, max_iter=3, callback=lambda it, st: states.__setitem__(it, {k: v.copy() for k, v in st.items()}))
    rho = 1.3
    A = dp.A.toarray()
    K = np.block([[np.diag(dp.D), A.T], [A, np.zeros((dp.m, dp.m))]])
    H = _dense_H(dp)
    for it in (2, 3):
        prev = states[it - 1]
        rhs = np.concatenate([H.T @ (prev["xk"] + prev["lam"] / rho) - dp.c / rho, dp.b])
        sol = np.linalg.solve(K, rhs)
        np.testing.assert_allclose(states[it]["x"], sol[:dp.N], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(states[it]["y"], sol[dp.N:], rtol=1e-10, atol=1e-10)


def test_dual_kkt_and_multiplier_sign():
    """Eq. OptCondMinYDual by dense solve; and the generic multiplier update
    (Eq. MultUpdateDualSDP) equals -rho H_k x (the sign printed in
    Eq. DualMultUpdate is the opposite)."""
    prob = W.random_chordal_small(6, 3, seed=2, extra_edges=3)
    dp = admm.decompose(prob)
    rho = 0.7
    states = {}
    admm.dual_admm(dp, rho=rho, eps=0, max_iter=4, callback=lambda it, st: states.__setitem__(it, {k: v.copy() for k, v in st.items()}))
    A = dp.A.toarray()
    K = np.block([[np.diag(dp.D), A.T], [A, np.zeros((dp.m, dp.m))]])
    H = _dense_H(dp)
    for it in (2, 3, 4):
        prev, cur = states[it - 1], states[it]
        rhs = np.concatenate([dp.c - H.T @ (cur["z"] + prev["lam"] / rho), -dp.b / rho])
        sol = np.linalg.solve(K, rhs)
        np.testing.assert_allclose(cur["x"], sol[:dp.N], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(cur["lam"], -rho * (H @ cur["x"]), rtol=1e-10, atol=1e-10)


def test_hsde_affine_step_is_dense_solve_of_I_plus_Q():
    """The block eliminations of Section 5.2.1-5.2.2 and Appendix B equal a
    dense solve of (I + Q) u_hat = u + v with Q from Eq. HSDEnotations."""
    prob = W.random_chordal_small(6, 3, seed=5, extra_edges=3)
    dp = admm.decompose(prob)
    op = admm.HSDEOperator(dp)
    A = dp.A.toarray(); H = _dense_H(dp)
    N, nd, m = dp.N, dp.nd, dp.m
    Z = np.zeros
    Q = np.block([
        [Z((N, N)), Z((N, nd)), -A.T, -H.T, dp.c[:, None]],
        [Z((nd, N)), Z((nd, nd)), Z((nd, m)), np.eye(nd), Z((nd, 1))],
        [A, Z((m, nd)), Z((m, m)), Z((m, nd)), -dp.b[:, None]],
        [H, -np.eye(nd), Z((nd, m)), Z((nd, nd)), Z((nd, 1))],
        [-dp.c[None, :], Z((1, nd)), dp.b[None, :], Z((1, nd)), Z((1, 1))],
    ])
    rng = np.random.default_rng(0)
    for _ in range(3):
        w = rng.standard_normal(Q.shape[0])
        np.testing.assert_allclose(op.solve_I_plus_Q(w), np.linalg.solve(np.eye(Q.shape[0]) + Q, w), rtol=1e-9, atol=1e-10)


CLOSED = [
    W.lambda_max_tridiagonal(8, 1.0, 0.5),
    W.lambda_max_tridiagonal(5, -0.5, -2.0),
    W.lovasz_theta_cycle(5),
    W.maxcut_cycle(5),
    W.maxcut_cycle(6),
    W.maxcut_cycle(7),
]


@pytest.mark.parametrize("form", ["primal", "dual", "hsde"])
@pytest.mark.parametrize("prob", CLOSED, ids=lambda p: p.name)
def test_closed_form_optimum(prob, form):
    """lambda_max(S) of a tridiagonal Toeplitz S, theta(C_5) = sqrt(5) and the
    MaxCut relaxation of cycles."""
    dp, r = admm.solve(prob, form, eps=1e-8, max_iter=20000)
    assert r.status == admm.SOLVED
    obj = float(dp.c @ r.X)
    assert abs(obj - prob.optimum) <= 1e-6 * max(1.0, abs(prob.optimum))
    if prob.name == "lovasz_theta_C5":
        assert abs(-obj - math.sqrt(5)) < 1e-6


def _kkt_residuals(dp, r):
    A = dp.A
    X, y, Z = r.X, r.y, r.Z
    rp = np.linalg.norm(A @ X - dp.b) / (1 + np.linalg.norm(dp.b))
    rd = np.linalg.norm(A.T @ y + Z - dp.c) / (1 + np.linalg.norm(dp.c))
    cx, by = dp.c @ X, dp.b @ y
    gap = abs(cx - by) / (1 + abs(cx) + abs(by))
    return rp, rd, gap


def _clique_blocks(dp, v):
    """Blocks E_k X E_k^T of a full-vec vector over the pattern."""
    return [v[ix].reshape(len(cl), len(cl), order="F") for cl, ix in zip(dp.cliques, dp.clique_idx)]


def _stacked_blocks(dp, s):
    """Blocks of a stacked clique vector (x_1, ..., x_p)."""
    return [s[dp.offsets[k]:dp.offsets[k + 1]].reshape(len(cl), len(cl), order="F") for k, cl in enumerate(dp.cliques)]


@pytest.mark.parametrize("form", ["primal", "dual", "hsde"])
def test_kkt_grone_agler_at_convergence(form):
    """At convergence: primal/dual feasibility and zero gap; every clique block
    of X is PSD (Grone, Theorem 1, so X has a PSD completion); Z is a sum of
    PSD clique terms (Agler, Theorem 2)."""
    prob = W.block_arrow(3, 4, 2, 6, seed=11)
    dp, r = admm.solve(prob, form, eps=1e-9, max_iter=20000)
    assert r.status == admm.SOLVED
    rp, rd, gap = _kkt_residuals(dp, r)
    assert max(rp, rd, gap) < 1e-6
    for blk in _clique_blocks(dp, r.X):
        assert np.linalg.eigvalsh(blk).min() > -1e-6 * max(1, np.abs(blk).max())
    if form == "primal":
        parts = r.state["lam"]
    elif form == "dual":
        parts = r.state["z"]
    else:
        parts = r.state["v"][dp.N:dp.N + dp.nd] / r.state["u"][-1]
    for blk in _stacked_blocks(dp, parts):
        assert np.linalg.eigvalsh(blk).min() > -1e-9 * max(1, np.abs(blk).max())
    np.testing.assert_allclose(dp.HT(parts), r.Z, atol=1e-12)


@pytest.mark.parametrize("seed", [3, 4, 8])
def test_decomposition_equivalence(seed):
    """Grone/Agler: the decomposed problem (p > 1 cliques) and the undecomposed
    one (complete pattern, p = 1) have the same optimum."""
    prob = W.random_chordal_small(7, 4, seed=seed, extra_edges=2)
    dp1, r1 = admm.solve(prob, "primal", eps=1e-9, max_iter=50000)
    dense = W.dense_pattern(prob)
    dp2, r2 = admm.solve(dense, "primal", eps=1e-9, max_iter=50000)
    assert len(dp1.cliques) > 1 and len(dp2.cliques) == 1
    o1, o2 = dp1.c @ r1.X, dp2.c @ r2.X
    assert abs(o1 - o2) <= 1e-6 * max(1, abs(o2))


def test_hsde_primal_infeasible_certificate():
    prob = W.primal_infeasible()
    dp, r = admm.solve(prob, "hsde", eps=1e-6, max_iter=5000)
    assert r.status == admm.PRIMAL_INFEASIBLE
    # b^T y = 1 and -A^T y = I (PSD): the unique certificate is y = -1
    np.testing.assert_allclose(r.cert, [-1.0], atol=1e-5)


def test_hsde_dual_infeasible_certificate():
    prob = W.dual_infeasible()
    dp, r = admm.solve(prob, "hsde", eps=1e-6, max_iter=5000)
    assert r.status == admm.DUAL_INFEASIBLE
    x = r.cert
    assert abs(dp.c @ x + 1.0) < 1e-9          # normalised: c^T x = -1
    assert np.linalg.norm(dp.A @ x) < 1e-5      # A x ~ 0
    for blk in _clique_blocks(dp, x):
        assert np.linalg.eigvalsh(blk).min() > -1e-5
    assert abs(x[dp.full_index[(0, 0)]] - 1.0) < 1e-5


def test_block_arrow_workload_converges():
    """The small block-arrow workload (l=5, d=10, h=5, m=30) reaches eps=1e-4
    in the primal and dual forms, and the two optima agree."""
    prob = W.workload(0)
    objs = []
    for form in ("primal", "dual"):
        dp, r = admm.solve(prob, form, eps=1e-4, max_iter=2000)
        assert r.status == admm.SOLVED
        objs.append(dp.c @ r.X)
    assert abs(objs[0] - objs[1]) <= 1e-4 * abs(objs[0])


# ---- adaptive penalty (Section 7.1.2) ---------------------------------------

def test_adapt_rho_rule_cases():
    """mu = 2, nu = 10: primal residual >= 10x dual -> double; dual >= 10x
    primal -> halve; otherwise keep (boundaries inclusive as printed)."""
    assert admm.adapt_rho(1.0, 1e-2, 1e-3, 2.0, 10.0) == 2.0
    assert admm.adapt_rho(1.0, 1e-3, 1e-2, 2.0, 10.0) == 0.5
    assert admm.adapt_rho(1.0, 1e-3, 2e-3, 2.0, 10.0) == 1.0
    assert admm.adapt_rho(4.0, 5.0, 0.5, 2.0, 10.0) == 8.0
    assert admm.adapt_rho(4.0, 0.0, 0.0, 2.0, 10.0) == 8.0  # 0 >= 10 * 0


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("prob", CLOSED[:4], ids=lambda p: p.name)
def test_closed_form_optimum_adaptive_rho(prob, form):
    """With the adaptive penalty the iteration still reaches the closed-form
    optimum (the rule only changes the path, not the fixed point)."""
    dp, r = admm.solve(prob, form, eps=1e-8, max_iter=20000, adapt_every=1)
    assert r.status == admm.SOLVED
    obj = float(dp.c @ r.X)
    assert abs(obj - prob.optimum) <= 1e-6 * max(1.0, abs(prob.optimum))


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_adaptive_rho_same_optimum(form):
    """Banded instance: with the adaptive rule applied every 5 iterations the
    iteration reaches the objective of the fixed-rho run (within 1e-5 at
    eps = 1e-6); the penalty recorded in history column 2 follows the rule
    applied to columns 0-1 of the same row, and does change."""
    prob = W.banded(60, 4, 15, seed=11, density=0.3)
    dp = admm.decompose(prob)
    fn = admm.primal_admm if form == "primal" else admm.dual_admm
    fixed = fn(dp, eps=1e-6, max_iter=30000)
    adapt = fn(dp, eps=1e-6, max_iter=30000, adapt_every=5)
    assert fixed.status == admm.SOLVED and adapt.status == admm.SOLVED
    o1, o2 = float(dp.c @ fixed.X), float(dp.c @ adapt.X)
    assert abs(o1 - o2) <= 1e-5 * abs(o1)
    h = adapt.hist
    assert np.all(fixed.hist[:, 2] == 1.0)
    for n in range(len(h) - 1):
        want = admm.adapt_rho(h[n, 2], h[n, 0], h[n, 1], 2.0, 10.0) if (n + 1) % 5 == 0 else h[n, 2]
        assert h[n + 1, 2] == want
    assert len(set(h[:, 2])) > 1
