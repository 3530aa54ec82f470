"""PSD projection of large blocks (order > 128) on the tensor cores
(cdsdp_psd_project_large: Newton-Schulz sign iteration, 3xTF32 tcgen05
products) against the FP64 projection of the same float32 inputs.

Tolerance.  The iteration converges to P(W) = (W + W sign(W)) / 2 for every
eigenvalue with |lambda| >= 1e-8 ||W||_F (an emulation of the schedule in
float64 lands within 1e-11); run in float32 arithmetic it lands within about
3e-6 ||W||_F in the Frobenius norm and 1.5e-7 ||W||_F entrywise (measured by
the same emulation at orders 129..513).  The 3xTF32 products keep float32
accuracy, so the checks are 1e-5 ||W||_F (Frobenius) and 1e-6 ||W||_F
(entrywise), plus the projection invariants."""
import numpy as np
import pytest

from oracle import psd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _sym(rng, s, kind):
    Q, _ = np.linalg.qr(rng.standard_normal((s, s)))
    if kind == "uniform":
        lam = rng.uniform(-1.0, 1.0, s)
    elif kind == "clustered":  # many eigenvalues near zero, as near an ADMM solution
        lam = np.concatenate([rng.uniform(0.5, 2.0, s // 3), rng.uniform(-1e-6, 1e-6, s // 3),
                              rng.uniform(-3.0, -0.5, s - 2 * (s // 3))])
    else:  # low-rank positive part
        lam = np.concatenate([rng.uniform(1.0, 5.0, 4), -rng.uniform(0.1, 1.0, s - 4)])
    W = (Q * lam) @ Q.T
    return np.float32(0.5 * (W + W.T)).astype(np.float64)


def _pack(B):
    return np.concatenate([B[b:, b] for b in range(B.shape[0])])


def _unpack(v, s):
    B = np.zeros((s, s))
    o = 0
    for b in range(s):
        B[b:, b] = v[o:o + s - b]
        B[b, b:] = v[o:o + s - b]
        o += s - b
    return B


def test_large_projection_matches_fp64(lib, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(129)
    cases = [(129, "uniform"), (200, "clustered"), (256, "lowrank"), (300, "uniform"), (513, "clustered"),
             (140, "zero")]
    blocks = [np.zeros((s, s)) if k == "zero" else _sym(rng, s, k) for s, k in cases]
    sizes = [s for s, _ in cases]
    W = torch.tensor(np.concatenate([_pack(B) for B in blocks]), dtype=torch.float32, device="cuda")
    X = lib.psd_project_large(W, sizes).cpu().numpy().astype(np.float64)
    o = 0
    for (s, kind), B in zip(cases, blocks):
        P = _unpack(X[o:o + s * (s + 1) // 2], s)
        o += s * (s + 1) // 2
        lam, V = np.linalg.eigh(B)
        ref = (V * np.maximum(lam, 0)) @ V.T
        nW = max(np.linalg.norm(B), 1e-30)
        if kind == "zero":
            assert np.abs(P).max() == 0.0
            continue
        assert np.linalg.norm(P - ref) <= 1e-5 * nW, (s, kind, np.linalg.norm(P - ref) / nW)
        assert np.abs(P - ref).max() <= 1e-6 * nW, (s, kind, np.abs(P - ref).max() / nW)
        # invariants: P >= 0, <W - P, P> = 0 (up to the same tolerance)
        assert np.linalg.eigvalsh(P).min() >= -1e-5 * nW
        assert abs(np.sum((B - P) * P)) <= 1e-5 * nW * nW


def test_large_projection_matches_oracle(lib, torch_cuda):
    """Order 129 against the oracle's own Jacobi projection."""
    torch = torch_cuda
    rng = np.random.default_rng(7)
    B = _sym(rng, 129, "uniform")
    W = torch.tensor(_pack(B), dtype=torch.float32, device="cuda")
    P = _unpack(lib.psd_project_large(W, [129]).cpu().numpy().astype(np.float64), 129)
    ref = psd.psd_project(B[None])[0]
    assert np.linalg.norm(P - ref) <= 1e-5 * np.linalg.norm(B)


def test_large_projection_diagonal(lib, torch_cuda):
    """A diagonal block projects to its elementwise clip."""
    torch = torch_cuda
    d = np.float32(np.linspace(-2.0, 3.0, 160)).astype(np.float64)
    W = torch.tensor(_pack(np.diag(d)), dtype=torch.float32, device="cuda")
    P = _unpack(lib.psd_project_large(W, [160]).cpu().numpy().astype(np.float64), 160)
    assert np.abs(P - np.diag(np.maximum(d, 0))).max() <= 1e-6 * np.linalg.norm(d)
