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
