"""Maximum-determinant completion (Section 7.1.1) on the GPU against the
oracle (oracle/completion.py): dense blocks equal element by element, log det
per component equal, closed form of the Kac-Murdock-Szego matrix, and a
partial matrix with an indefinite clique block reported as such."""
import numpy as np
import pytest

from oracle import completion
from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _blocks(P, Wflat):
    """Dense blocks of the library output, with the vertices of each."""
    vc, _ = P.components()
    _, _, offs = P.completion_sizes()
    out = []
    Wh = Wflat.cpu().numpy()
    for c in range(int(P.info["ncomp"])):
        verts = np.flatnonzero(vc == c)
        nc = len(verts)
        out.append((verts, Wh[offs[c]:offs[c + 1]].reshape(nc, nc)))
    return out


def _compare(lib, prob, seed=11, rtol=1e-10):
    P = lib.Problem(prob)
    r, c = P.pattern()
    X = W.pd_on_pattern(prob.n, r, c, seed)
    Wg, ldg = P.complete(X)
    lower = list(zip(r.tolist(), c.tolist()))
    Wo, schur, ok = completion.maxdet_completion(prob.n, lower, X)
    assert ok
    scale = np.abs(Wo).max()
    vc, _ = P.components()
    for cidx, (verts, B) in enumerate(_blocks(P, Wg)):
        ref = Wo[np.ix_(verts, verts)]
        assert np.abs(B - ref).max() <= rtol * scale, cidx
        np.testing.assert_allclose(ldg[cidx], np.sum(np.log(schur[verts])), rtol=1e-11, atol=1e-11)
        # given entries are copied, not recomputed
    Wd = np.zeros((prob.n, prob.n))
    for verts, B in _blocks(P, Wg):
        Wd[np.ix_(verts, verts)] = B
    np.testing.assert_array_equal(Wd[r, c], X)
    return P, Wd


CASES = [W.workload(0), W.banded(400, 10, 50, seed=4), W.block_arrow(3, 70, 10, 12, seed=2, density=0.2),
         W.direct_sum([W.banded(120, 6, 20, seed=5), W.workload(0), W.maxcut_cycle(9)])]


@pytest.mark.parametrize("prob", CASES, ids=lambda p: p.name)
def test_completion_matches_oracle(lib, torch_cuda, prob):
    _compare(lib, prob)


def test_completion_full_size_banded(lib, torch_cuda):
    """Banded n=2000, w=10, m=500 (the benchmark's single-SDP workload)."""
    _compare(lib, W.workload(1), rtol=1e-9)


def test_kac_murdock_szego(lib, torch_cuda):
    """Tridiagonal pattern (banded, w=1) with x_ij = rho^|i-j|: the completion
    is rho^|i-j| everywhere and log det = (n-1) log(1 - rho^2)."""
    n, rho = 300, 0.7
    prob = W.banded(n, 1, 30, seed=8)
    P = lib.Problem(prob)
    r, c = P.pattern()
    assert np.all(np.abs(r - c) <= 1)
    Wg, ld = P.complete(rho ** np.abs(r - c).astype(np.float64))
    assert int(P.info["ncomp"]) == 1
    K = rho ** np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    np.testing.assert_allclose(Wg.cpu().numpy().reshape(n, n), K, rtol=1e-11, atol=1e-300)
    assert ld[0] == pytest.approx((n - 1) * np.log(1 - rho ** 2), rel=1e-12)


def test_factor_only_and_not_pd(lib, torch_cuda):
    prob = W.workload(0)
    P = lib.Problem(prob)
    r, c = P.pattern()
    X = W.pd_on_pattern(prob.n, r, c, 3)
    Wg, ld = P.complete(X, dense=False)
    assert Wg is None and np.isfinite(ld).all()
    Xbad = X.copy()
    Xbad[r == c] *= -1.0  # negative diagonal: no clique block is positive definite
    with pytest.raises(lib.CdsdpError) as ex:
        P.complete(Xbad)
    assert ex.value.status == lib.NOT_PD


def test_completion_of_a_solver_iterate(lib, torch_cuda):
    """X returned by an FP64 primal solve of the block-arrow workload, shifted
    by 1e-3 I so that its clique blocks are positive definite: completes, the
    completion is positive definite and equals the oracle's."""
    prob = W.workload(0)
    P = lib.Problem(prob).bind(max_iter=2000)
    out = P.solve("primal", eps=1e-5, max_iter=2000, precision="fp64")
    r, c = P.pattern()
    X = out["X"] + np.where(r == c, 1e-3, 0.0)
    Wg, _ = P.complete(X)
    n = prob.n
    Wd = Wg.cpu().numpy().reshape(n, n)
    assert np.linalg.eigvalsh(Wd).min() > 0
    Wo, _, ok = completion.maxdet_completion(n, list(zip(r.tolist(), c.tolist())), X)
    assert ok and np.abs(Wd - Wo).max() <= 1e-8 * np.abs(Wo).max()
