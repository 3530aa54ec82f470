"""GPU edge cases of the library through its C ABI: empty and degenerate
projection inputs (order 1, zero blocks, diagonal blocks, exact zero
eigenvalues), the smallest solves (one iteration, a 1x1 SDP inside a batch),
and the error statuses of out-of-order or invalid calls."""
import dataclasses

import numpy as np
import pytest

from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _layout(torch, sizes):
    off = np.concatenate([[0], np.cumsum([s * (s + 1) // 2 for s in sizes])]).astype(np.int32)
    return (torch.tensor(off, device="cuda"), torch.tensor(np.array(sizes, np.int32), device="cuda"))


def _pack(blocks):
    out = []
    for B in blocks:
        for b in range(B.shape[0]):
            out.extend(B[b:, b].tolist())
    return np.array(out)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_projection_degenerate_blocks(lib, torch_cuda, dtype):
    """Order-1 blocks clip (max(w, 0)); zero blocks stay zero; diagonal blocks
    clip elementwise; a block with exact zero eigenvalues (a PSD rank-1 matrix)
    is its own projection; orders 1..64 side by side."""
    torch = torch_cuda
    dt = getattr(torch, dtype)
    rng = np.random.default_rng(3)
    blocks = [np.array([[v]]) for v in (-2.0, 0.0, 3.5)]
    blocks += [np.zeros((s, s)) for s in (5, 33)]
    blocks += [np.diag(rng.standard_normal(s)) for s in (7, 40)]
    u = rng.standard_normal(12)
    blocks.append(np.outer(u, u))  # eigenvalues |u|^2 and eleven exact zeros
    sizes = [B.shape[0] for B in blocks]
    if dtype == "float32":
        blocks = [B.astype(np.float32).astype(np.float64) for B in blocks]
    off, sz = _layout(torch, sizes)
    X = lib.psd_project(torch.tensor(_pack(blocks), dtype=dt, device="cuda"), off, sz)
    torch.cuda.synchronize()
    got = X.double().cpu().numpy()
    want = []
    for B in blocks:
        if B.shape[0] == 1 or np.count_nonzero(B - np.diag(np.diag(B))) == 0:
            want.append(np.diag(np.maximum(np.diag(B), 0.0)))
        else:
            want.append(B)  # zero or PSD
    tol = 1e-12 if dtype == "float64" else 2e-6
    o = 0
    for B, Wt in zip(blocks, want):
        n = B.shape[0] * (B.shape[0] + 1) // 2
        scale = max(1.0, np.abs(B).max()) * B.shape[0]
        assert np.abs(got[o:o + n] - _pack([Wt])).max() <= tol * scale
        o += n


def test_projection_empty_batch(lib, torch_cuda):
    torch = torch_cuda
    W0 = torch.zeros(4, dtype=torch.float32, device="cuda")
    off = torch.zeros(1, dtype=torch.int32, device="cuda")
    sz = torch.zeros(0, dtype=torch.int32, device="cuda")
    X = lib.psd_project(W0, off, sz)  # p = 0: nothing to do, no error
    torch.cuda.synchronize()
    assert X.shape == W0.shape


def test_one_iteration_and_error_statuses(lib, torch_cuda):
    import ctypes
    prob = W.workload(0)
    P = lib.Problem(prob)
    raw = lib._lib.cdsdp_solve
    assert raw(P._h, 0, None, None, None, None, None, None, None, None) < 0  # no workspace bound
    P.bind(max_iter=10)
    out = P.solve("primal", eps=1e-4, max_iter=1, precision="fp64")
    assert out["iters"] == 1 and out["status"] == lib.MAX_ITER
    o = lib.default_opts(max_iter=11)  # beyond the bound workspace's history
    assert raw(P._h, 0, ctypes.byref(o), None, None, None, None, None, None, None) < 0
    assert raw(P._h, 3, None, None, None, None, None, None, None, None) < 0  # no form 3
    with pytest.raises(lib.CdsdpError):  # invalid penalty
        P.solve("primal", eps=1e-4, max_iter=5, rho=0.0)
    out = P.solve("primal", eps=1e-4, max_iter=10, precision="fp64")  # the handle still works
    assert out["iters"] == 10


def test_one_by_one_sdp_in_a_batch(lib, torch_cuda):
    """A 1x1 SDP (min c x s.t. a x = b, x >= 0: x = b/a) as one component of a
    direct sum with a block-arrow SDP: solved on its own test to its closed form."""
    tiny = W.SDPProblem(1, 1, np.array([0], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                        np.array([2.0]), np.array([3.0]), np.array([0], np.int32), np.array([0], np.int32),
                        np.array([1.0]), np.zeros(0, np.int32), np.zeros(0, np.int32), "one_by_one", 1.5)
    prob = W.direct_sum([W.block_arrow(2, 4, 2, 5, seed=8), tiny])
    P = lib.Problem(prob).bind(max_iter=5000)
    assert P.info["ncomp"] == 2
    out = P.solve("primal", eps=1e-8, max_iter=5000, precision="fp64")
    it, st, res = P.component_results()
    assert st[1] == 0
    r, c = P.pattern()
    x_tiny = out["X"][(r == prob.n - 1) & (c == prob.n - 1)][0]
    assert abs(x_tiny - 1.5) < 1e-6
