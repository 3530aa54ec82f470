"""Data scaling of Section 7.1.3 on the GPU: a handle set up scaled runs the
same FP64 trajectory as the oracle on the oracle's scaled problem, and returns
the oracle's scaled solution mapped back to the original units; scaled and
unscaled solves reach the same optimum; certificates keep the normalisation of
an unscaled solve."""
import numpy as np
import pytest

from oracle import admm, scaling
from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _full(dp, lower_vals):
    x = np.zeros(dp.N)
    for (i, j), v in zip(dp.lower, lower_vals):
        x[dp.full_index[(i, j)]] = v
        x[dp.full_index[(j, i)]] = v
    return x


@pytest.mark.parametrize("passes", [0, 4])
@pytest.mark.parametrize("form", ["primal", "dual", "hsde"])
def test_scaled_fp64_trajectory_matches_oracle(lib, torch_cuda, form, passes):
    """Block-arrow l=5, d=10, h=5, m=30: FP64 GPU on the scaled handle vs the
    oracle on scaling.scale_problem: same iterations and residual history
    (scaled units), and X, y, Z equal to the oracle's mapped back."""
    prob = W.workload(0)
    sp, fac = scaling.scale_problem(prob, passes)
    eps, max_iter = 1e-5, 3000
    dp, ref = admm.solve(sp, form, eps=eps, max_iter=max_iter)
    P = lib.Problem(prob, scale_passes=passes).bind(max_iter=max_iter)
    out = P.solve(form, eps=eps, max_iter=max_iter, precision="fp64", check_every=7)
    assert out["status"] == ref.status == 0
    assert abs(out["iters"] - ref.iters) <= 1
    k = min(out["iters"], ref.iters, 50)
    np.testing.assert_allclose(out["hist"][:k, :6], ref.hist[:k, :6], rtol=1e-8, atol=1e-10)
    X, y, Z = scaling.unscale(dp.lower, dp.lower_values(ref.X), ref.y, dp.lower_values(ref.Z), fac)
    for name, a, b in (("X", out["X"], X), ("y", out["y"], y), ("Z", out["Z"], Z)):
        assert np.abs(a - b).max() <= 1e-7 * max(1.0, np.abs(b).max()), name


@pytest.mark.parametrize("form", ["primal", "hsde"])
def test_scaled_and_unscaled_reach_the_same_optimum(lib, torch_cuda, form):
    """Badly scaled constraint rows (row norms spread over 1e-2..1e2): the
    scaled solve, mapped back, satisfies the original KKT conditions and
    matches the unscaled oracle's objective."""
    import dataclasses
    prob = W.workload(0)
    rng = np.random.default_rng(3)
    f = 10.0 ** rng.uniform(-2, 2, prob.m)
    prob = dataclasses.replace(prob, A_val=prob.A_val * f[prob.A_con], b=prob.b * f, name="block_arrow_rows_spread")
    dp0, ref = admm.solve(W.workload(0), "primal", eps=1e-7, max_iter=20000)  # row scaling keeps the optimum
    dp = admm.decompose(prob)
    P = lib.Problem(prob, scale_passes=6).bind(max_iter=20000)
    out = P.solve(form, eps=1e-7, max_iter=20000, precision="fp64")
    assert out["status"] == 0
    X, Z, y = _full(dp, out["X"]), _full(dp, out["Z"]), out["y"]
    obj = float(dp.c @ X)
    ref_obj = float(dp0.c @ ref.X)
    assert abs(obj - ref_obj) <= 1e-5 * max(1.0, abs(ref_obj))
    rp = np.linalg.norm(dp.A @ X - dp.b) / (1 + np.linalg.norm(dp.b))
    rd = np.linalg.norm(dp.A.T @ y + Z - dp.c) / (1 + np.linalg.norm(dp.c))
    assert max(rp, rd) <= 1e-5


def test_scaled_certificates(lib, torch_cuda):
    """Infeasibility certificates of a scaled handle, mapped back: b^T y = 1
    for the primal one, C . X = -1 and A X ~ 0 for the dual one."""
    prob = W.primal_infeasible()
    P = lib.Problem(prob, scale_passes=3).bind(max_iter=5000)
    out = P.solve("hsde", eps=1e-6, max_iter=5000, precision="fp64")
    assert out["status"] == lib.PRIMAL_INFEASIBLE
    assert abs(float(prob.b @ out["cert"]) - 1.0) < 1e-9
    np.testing.assert_allclose(out["cert"], [-1.0], atol=1e-5)
    prob = W.dual_infeasible()
    dp = admm.decompose(prob)
    P = lib.Problem(prob, scale_passes=3).bind(max_iter=5000)
    out = P.solve("hsde", eps=1e-6, max_iter=5000, precision="fp64")
    assert out["status"] == lib.DUAL_INFEASIBLE
    x = _full(dp, out["cert"])
    assert abs(dp.c @ x + 1) < 1e-9 and np.linalg.norm(dp.A @ x) < 1e-5


def test_scaled_handle_refuses_unrolled_gradients(lib, torch_cuda):
    torch = torch_cuda
    P = lib.Problem(W.workload(0), scale_passes=2).bind(max_iter=64)
    with pytest.raises(lib.CdsdpError):
        P.unrolled_forward(torch.zeros(P.info["nnz_pattern"], dtype=torch.float64, device="cuda"),
                           torch.zeros(P.info["m"], dtype=torch.float64, device="cuda"), iters=8, ckpt_every=8)
