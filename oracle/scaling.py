"""Data scaling of Section 7.1.3 (test infrastructure: the oracle; only tests,
smoke() and bench.py's CPU baseline use this package).

The paper scales the decomposed problem by positive diagonal matrices and two
positive scalars, chosen so that rows of the scaled constraint data have
norm near one, and maps the scaled solution back; it defers the cone-preserving
choice to SCS.  Reading used here (one cone-preserving family that keeps the
sparsity pattern): a diagonal congruence X = D Xbar D (D = diag(d), d > 0)
preserves the PSD cone and every clique block, constraint rows are scaled by
e > 0, and b and c by scalars tau and sigma:

    Abar_i = e_i D A_i D,   bbar_i = tau e_i b_i,   Cbar = sigma D C D,

so that Xbar = tau D^-1 X D^-1, ybar_i = sigma y_i / e_i, Zbar = sigma D Z D, and

    X = D Xbar D / tau,   y_i = e_i ybar_i / sigma,   Z = D^-1 Zbar D^-1 / sigma.

d and e come from `passes` rounds of symmetric Ruiz equilibration on the
constraint data (triplets as given, both triangles of an off-diagonal entry
counted): e_i <- e_i / sqrt(||Abar_i||_F), then d_j <- d_j / sqrt(m_j) with m_j
the largest |Abar_i(j, k)| over constraints and k, both clipped to [1e-4, 1e4];
then tau = 1 / ||bbar||_2 and sigma = 1 / ||Cbar||_F (1 when the norm is 0)."""
import dataclasses

import numpy as np


def scaling_factors(prob, passes):
    n, m = prob.n, prob.m
    d = np.ones(n)
    e = np.ones(m)
    r, c, con, v = prob.A_row, prob.A_col, prob.A_con, prob.A_val
    w = np.where(r == c, 1.0, 2.0)
    for _ in range(passes):
        a = e[con] * d[r] * d[c] * v
        rown = np.sqrt(np.bincount(con, weights=w * a * a, minlength=m))
        e = np.clip(e / np.sqrt(np.where(rown > 0, rown, 1.0)), 1e-4, 1e4)
        a = np.abs(e[con] * d[r] * d[c] * v)
        mj = np.zeros(n)
        np.maximum.at(mj, r, a)
        np.maximum.at(mj, c, a)
        d = np.clip(d / np.sqrt(np.where(mj > 0, mj, 1.0)), 1e-4, 1e4)
    bb = e * prob.b
    nb = np.linalg.norm(bb)
    tau = 1.0 / nb if nb > 0 else 1.0
    cw = np.where(prob.C_row == prob.C_col, 1.0, 2.0)
    cc = d[prob.C_row] * d[prob.C_col] * prob.C_val
    nc = np.sqrt(np.sum(cw * cc * cc))
    sigma = 1.0 / nc if nc > 0 else 1.0
    return d, e, tau, sigma


def scale_problem(prob, passes):
    """(scaled problem, (d, e, tau, sigma))."""
    d, e, tau, sigma = scaling_factors(prob, passes)
    sp = dataclasses.replace(
        prob,
        A_val=e[prob.A_con] * d[prob.A_row] * d[prob.A_col] * prob.A_val,
        b=tau * e * prob.b,
        C_val=sigma * d[prob.C_row] * d[prob.C_col] * prob.C_val,
        name=prob.name + "_scaled", optimum=None)
    return sp, (d, e, tau, sigma)


def unscale(lower, X, y, Z, factors):
    """Map a solution of the scaled problem back; X, Z are values on the lower
    pattern `lower` (list of (i, j))."""
    d, e, tau, sigma = factors
    dd = np.array([d[i] * d[j] for i, j in lower])
    return dd * X / tau, e * y / sigma, Z / (dd * sigma)
