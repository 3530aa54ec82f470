"""Pins for the oracle's adjoint of unrolled Algorithm 1 (CPU only): central
finite differences of L = <g, x_N(c, b)> in random directions."""
import numpy as np
import pytest

from oracle import admm
from paper_1707_05058_gb300 import workloads as W


def _sym_dir(dp, rng):
    d = np.zeros(dp.N)
    for (i, j) in dp.lower:
        v = rng.standard_normal()
        d[dp.full_index[(i, j)]] = v
        d[dp.full_index[(j, i)]] = v
    return d


@pytest.mark.parametrize("seed,iters,rho", [(0, 6, 1.0), (1, 15, 0.7), (2, 25, 1.3)])
def test_unrolled_adjoint_matches_finite_differences(seed, iters, rho):
    prob = W.random_chordal_small(7, 4, seed=seed, extra_edges=4)
    dp = admm.decompose(prob)
    rng = np.random.default_rng(seed)
    g = _sym_dir(dp, rng)
    c0, b0 = dp.c.copy(), dp.b.copy()
    cbar, bbar = admm.primal_unrolled_vjp(dp, c0, b0, iters, g, rho=rho)
    h = 1e-6
    for _ in range(3):
        dc = _sym_dir(dp, rng)
        db = rng.standard_normal(dp.m)
        Lp = g @ admm.primal_unrolled(dp, c0 + h * dc, b0 + h * db, iters, rho)
        Lm = g @ admm.primal_unrolled(dp, c0 - h * dc, b0 - h * db, iters, rho)
        fd = (Lp - Lm) / (2 * h)
        an = cbar @ dc + bbar @ db
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (fd, an)


def test_unrolled_matches_solver_iterates():
    """primal_unrolled with the problem's own (c, b) reproduces Algorithm 1."""
    prob = W.random_chordal_small(6, 3, seed=4, extra_edges=3)
    dp = admm.decompose(prob)
    ref = admm.primal_admm(dp, eps=0.0, max_iter=9)
    x = admm.primal_unrolled(dp, dp.c, dp.b, 9)
    np.testing.assert_allclose(x, ref.X, rtol=1e-13, atol=1e-13)
