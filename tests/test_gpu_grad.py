"""GPU reverse pass through unrolled Algorithm 1 (Daleckii-Krein adjoint of the
projection) against the FP64 oracle adjoint and against finite differences.

Coordinates: the solver's x and c are values on the lower pattern (an
off-diagonal value stands for both entries).  For L = <g, x_N> in those
coordinates the oracle (full vec, both triangles) takes the cotangent g on
the diagonal and g/2 on each of the two off-diagonal positions, and the
gradient with respect to a lower value c_e is the sum of the oracle's
gradients at its two positions.  Tolerances: FP64 path 1e-8 (same algorithm,
other rounding order); FP32-projection path 1e-3 relative (the stated
gradient target)."""
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


def _oracle_grad(dp, g_lower, iters, rho):
    gfull = np.zeros(dp.N)
    for e, (i, j) in enumerate(dp.lower):
        if i == j:
            gfull[dp.full_index[(i, j)]] = g_lower[e]
        else:
            gfull[dp.full_index[(i, j)]] = 0.5 * g_lower[e]
            gfull[dp.full_index[(j, i)]] = 0.5 * g_lower[e]
    cbar_full, bbar = admm.primal_unrolled_vjp(dp, dp.c, dp.b, iters, gfull, rho=rho)
    cbar = np.array([cbar_full[dp.full_index[(i, j)]] + (cbar_full[dp.full_index[(j, i)]] if i != j else 0.0)
                     for (i, j) in dp.lower])
    x = admm.primal_unrolled(dp, dp.c, dp.b, iters, rho)
    return dp.lower_values(x), cbar, bbar


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", 1e-3)])
@pytest.mark.parametrize("iters,ckpt", [(30, 10), (23, 7)])
def test_unrolled_gradient_matches_oracle(lib, torch_cuda, prec, tol, iters, ckpt):
    torch = torch_cuda
    prob = W.block_arrow(3, 4, 2, 6, seed=21)
    dp = admm.decompose(prob)
    rho = 0.8
    P = lib.Problem(prob).bind(max_iter=64)
    c, b = P.problem_data()
    rng = np.random.default_rng(iters)
    g = rng.standard_normal(int(P.info["nnz_pattern"]))
    x, gws = P.unrolled_forward(c, b, iters, ckpt, prec, rho)
    cbar, bbar = P.unrolled_backward(c, b, torch.tensor(g, device="cuda"), iters, ckpt, gws, prec, rho)
    x_ref, cbar_ref, bbar_ref = _oracle_grad(dp, g, iters, rho)
    xs = x.cpu().numpy()
    assert np.abs(xs - x_ref).max() <= (1e-9 if prec == "fp64" else 1e-3) * np.abs(x_ref).max()
    for got, want in ((cbar.cpu().numpy(), cbar_ref), (bbar.cpu().numpy(), bbar_ref)):
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), (np.abs(got - want).max(), np.abs(want).max())


def test_autograd_function_and_objective_gradient(lib, torch_cuda):
    """torch.autograd through the library: d<c, x_N>/dc and d/db against the
    oracle adjoint (the direct term of c is added by autograd)."""
    torch = torch_cuda
    prob = W.block_arrow(3, 4, 2, 6, seed=22)
    dp = admm.decompose(prob)
    P = lib.Problem(prob).bind(max_iter=64)
    c, b = P.problem_data()
    c.requires_grad_(True); b.requires_grad_(True)
    r, cpat = P.pattern()
    w = torch.tensor(np.where(r == cpat, 1.0, 2.0), dtype=torch.float64, device="cuda")
    x = lib.unrolled_primal(P, c, b, iters=40, ckpt_every=8, precision="fp64")
    obj = (w * c * x).sum()
    obj.backward()
    x_ref, cbar_ref, bbar_ref = _oracle_grad(dp, (w * c).detach().cpu().numpy(), 40, 1.0)
    cbar_ref = cbar_ref + np.where(r == cpat, 1.0, 2.0) * x_ref
    np.testing.assert_allclose(c.grad.cpu().numpy(), cbar_ref, rtol=1e-7, atol=1e-9 * np.abs(cbar_ref).max())
    np.testing.assert_allclose(b.grad.cpu().numpy(), bbar_ref, rtol=1e-7, atol=1e-9 * np.abs(bbar_ref).max())


def test_banded_gradient_finite_differences_full_size(lib, torch_cuda):
    """Banded n=500, w=8, m=200 (492 cliques of order 9), 500 unrolled
    iterations checkpointed every 50: the FP32 reverse pass against central
    finite differences (h = 1e-6) of the FP64 forward, in random directions."""
    torch = torch_cuda
    prob = W.banded(500, 8, 200, seed=5708)
    P = lib.Problem(prob).bind(max_iter=64)
    c, b = P.problem_data()
    rng = np.random.default_rng(3)
    g = torch.tensor(rng.standard_normal(int(P.info["nnz_pattern"])), device="cuda")
    x, gws = P.unrolled_forward(c, b, 500, 50, "fp32")
    cbar, bbar = P.unrolled_backward(c, b, g, 500, 50, gws, "fp32")
    x64, gws64 = P.unrolled_forward(c, b, 500, 50, "fp64")
    cbar64, bbar64 = P.unrolled_backward(c, b, g, 500, 50, gws64, "fp64")
    h = 1e-6
    for _ in range(2):
        dc = torch.tensor(rng.standard_normal(c.numel()), device="cuda")
        db = torch.tensor(rng.standard_normal(b.numel()), device="cuda")
        xp, _ = P.unrolled_forward(c + h * dc, b + h * db, 500, 50, "fp64")
        xm, _ = P.unrolled_forward(c - h * dc, b - h * db, 500, 50, "fp64")
        fd = float((g * (xp - xm)).sum() / (2 * h))
        an64 = float((cbar64 * dc).sum() + (bbar64 * db).sum())
        an32 = float((cbar * dc).sum() + (bbar * db).sum())
        assert abs(an64 - fd) <= 1e-5 * max(1.0, abs(fd)), (an64, fd)
        assert abs(an32 - fd) <= 1e-3 * max(1.0, abs(fd)), (an32, fd)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", 1e-3)])
def test_unrolled_gradient_direct_sum(lib, torch_cuda, prec, tol):
    """A batch of three SDPs (a direct sum, as the batched gradient workload
    runs): the reverse pass over the sum restricted to each summand equals the
    oracle adjoint of that summand alone."""
    torch = torch_cuda
    parts = [W.block_arrow(3, 4, 2, 6, seed=21), W.banded(15, 3, 7, seed=22, density=0.4),
             W.block_arrow(2, 5, 3, 9, seed=23, density=0.5)]
    prob = W.direct_sum(parts)
    iters, ckpt, rho = 24, 8, 0.8
    P = lib.Problem(prob).bind(max_iter=64)
    assert P.info["ncomp"] == 3
    c, b = P.problem_data()
    rng = np.random.default_rng(5)
    g = rng.standard_normal(int(P.info["nnz_pattern"]))
    x, gws = P.unrolled_forward(c, b, iters, ckpt, prec, rho)
    cbar, bbar = P.unrolled_backward(c, b, torch.tensor(g, device="cuda"), iters, ckpt, gws, prec, rho)
    r, col = P.pattern()
    xs, cb, bb = x.cpu().numpy(), cbar.cpu().numpy(), bbar.cpu().numpy()
    vo = mo = 0
    for q in parts:
        mask = (col >= vo) & (col < vo + q.n)
        dp = admm.decompose(q)
        x_ref, cbar_ref, bbar_ref = _oracle_grad(dp, g[mask], iters, rho)
        assert np.abs(xs[mask] - x_ref).max() <= (1e-9 if prec == "fp64" else 1e-3) * np.abs(x_ref).max()
        for got, want in ((cb[mask], cbar_ref), (bb[mo:mo + q.m], bbar_ref)):
            assert np.abs(got - want).max() <= tol * np.abs(want).max()
        vo += q.n
        mo += q.m
