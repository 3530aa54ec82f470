"""Pins of the maximum-determinant completion oracle (Section 7.1.1,
oracle/completion.py) against closed forms and the characterisation of
Grone et al.: W agrees with X on the pattern, W is positive definite and W^-1
vanishes off the pattern; a matrix whose inverse is sparse on a chordal
pattern is recovered from its pattern entries."""
import numpy as np
import pytest

from oracle import chordal, completion
from paper_1707_05058_gb300 import workloads as W


def _random_chordal_lower(n, nedges, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for _ in range(nedges):
        i, j = rng.integers(0, n, 2)
        if i != j:
            rows.append(max(i, j)); cols.append(min(i, j))
    _, lower, _, _ = chordal.chordal_decomposition(n, [(rows, cols)])
    return lower


def _values(M, lower):
    return np.array([M[i, j] for i, j in lower])


def _off_pattern_mask(n, lower):
    mask = np.ones((n, n), bool)
    for i, j in lower:
        mask[i, j] = mask[j, i] = False
    return mask


def test_three_by_three_closed_form():
    """Path 0-1-2: the free entry of the max-det completion is x01 x12 / x11."""
    a, b, c, d, e = 2.0, 0.7, 1.5, -0.4, 3.0
    lower = [(0, 0), (1, 0), (1, 1), (2, 1), (2, 2)]
    Wc, schur, ok = completion.maxdet_completion(3, lower, [a, b, c, d, e])
    assert ok
    assert Wc[2, 0] == pytest.approx(b * d / c, rel=1e-15)
    assert Wc[0, 2] == Wc[2, 0]


def test_kac_murdock_szego_from_its_tridiagonal_part():
    """The matrix rho^|i-j| has a tridiagonal inverse, so it is the max-det
    completion of its own tridiagonal entries."""
    n, rho = 40, 0.6
    K = rho ** np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    lower = [(i, i) for i in range(n)] + [(i + 1, i) for i in range(n - 1)]
    Wc, schur, ok = completion.maxdet_completion(n, lower, _values(K, lower))
    assert ok
    np.testing.assert_allclose(Wc, K, rtol=1e-12, atol=1e-300)
    # log det of the KMS matrix: (n - 1) log(1 - rho^2)
    assert completion.logdet(schur) == pytest.approx((n - 1) * np.log(1 - rho ** 2), rel=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_recovers_matrix_with_sparse_inverse(seed):
    """P positive definite with its sparsity on a chordal pattern: the
    completion of inv(P) restricted to the pattern is inv(P)."""
    n = 30
    lower = _random_chordal_lower(n, 45, seed)
    rng = np.random.default_rng(100 + seed)
    P = np.zeros((n, n))
    for i, j in lower:
        if i != j:
            P[i, j] = P[j, i] = rng.uniform(-1, 1)
    P += np.diag(1.0 + np.abs(P).sum(axis=1))
    Wt = np.linalg.inv(P)
    Wc, schur, ok = completion.maxdet_completion(n, lower, _values(Wt, lower))
    assert ok
    np.testing.assert_allclose(Wc, Wt, rtol=1e-10, atol=1e-13)
    assert completion.logdet(schur) == pytest.approx(-np.linalg.slogdet(P)[1], rel=1e-11)


@pytest.mark.parametrize("prob", [W.workload(0), W.banded(60, 4, 10, seed=3)], ids=lambda p: p.name)
def test_characterisation_on_workload_patterns(prob):
    """Generic positive definite data on the extended pattern of a workload:
    W = X on the pattern, W > 0, (W^-1) = 0 off the pattern."""
    from oracle import admm
    dp = admm.decompose(prob)
    n = prob.n
    rng = np.random.default_rng(7)
    G = rng.standard_normal((n, 3 * n))
    M = G @ G.T / (3 * n)
    X = _values(M, dp.lower)
    Wc, schur, ok = completion.maxdet_completion(n, dp.lower, X)
    assert ok
    np.testing.assert_allclose(_values(Wc, dp.lower), X, rtol=0, atol=0)
    assert np.linalg.eigvalsh(Wc).min() > 0
    Winv = np.linalg.inv(Wc)
    assert np.abs(Winv[_off_pattern_mask(n, dp.lower)]).max() <= 1e-10 * np.abs(Winv).max()
    assert completion.logdet(schur) == pytest.approx(np.linalg.slogdet(Wc)[1], rel=1e-11)


def test_free_entries_are_stationary_for_log_det():
    """Moving any free entry (symmetrically) by +-delta lowers log det."""
    n = 8
    lower = _random_chordal_lower(n, 9, 4)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((n, 2 * n))
    Wc, _, ok = completion.maxdet_completion(n, lower, _values(G @ G.T, lower))
    assert ok
    base = np.linalg.slogdet(Wc)[1]
    free = np.argwhere(np.tril(_off_pattern_mask(n, lower), -1))
    assert len(free) > 0
    for i, j in free:
        for dlt in (1e-3, -1e-3):
            Wp = Wc.copy()
            Wp[i, j] += dlt; Wp[j, i] += dlt
            s, ld = np.linalg.slogdet(Wp)
            assert s < 0 or ld < base


def test_direct_sum_completes_blockwise():
    """Two disconnected components: entries between them come out zero."""
    lower = [(0, 0), (1, 0), (1, 1), (2, 2), (3, 2), (3, 3)]
    Wc, _, ok = completion.maxdet_completion(4, lower, [2.0, 0.5, 1.0, 3.0, -1.0, 2.0])
    assert ok
    assert np.all(Wc[:2, 2:] == 0) and np.all(Wc[2:, :2] == 0)


def test_not_positive_definite_clique_is_reported():
    lower = [(0, 0), (1, 0), (1, 1), (2, 1), (2, 2)]
    _, _, ok = completion.maxdet_completion(3, lower, [1.0, 2.0, 1.0, 0.1, 1.0])
    assert not ok


def test_non_chordal_pattern_is_rejected():
    lower = [(i, i) for i in range(4)] + [(1, 0), (2, 1), (3, 2), (3, 0)]
    with pytest.raises(ValueError):
        completion.maxdet_completion(4, lower, np.ones(len(lower)))

