"""Randomised pin of the maximum-determinant completion oracle (Section 7.1.1,
oracle/completion.py): on random chordal patterns (possibly disconnected) the
characterisation of Grone et al. holds."""
import numpy as np
import pytest

from oracle import chordal, completion

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _values(M, lower):
    return np.array([M[i, j] for i, j in lower])


def _off_pattern_mask(n, lower):
    mask = np.ones((n, n), bool)
    for i, j in lower:
        mask[i, j] = mask[j, i] = False
    return mask


@settings(max_examples=60, deadline=None)
@given(st.integers(min_value=2, max_value=24), st.floats(min_value=0.05, max_value=0.6),
       st.integers(min_value=0, max_value=2**31 - 1))
def test_characterisation_on_random_chordal_patterns(n, p, seed):
    """Random graphs, chordally extended (possibly disconnected): the completion
    of generic positive definite data agrees on the pattern, is positive
    definite, and its inverse vanishes off the pattern."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        for j in range(i):
            if rng.random() < p:
                rows.append(i); cols.append(j)
    _, lower, _, _ = chordal.chordal_decomposition(n, [(rows, cols)])
    G = rng.standard_normal((n, 2 * n))
    X = _values(G @ G.T / (2 * n) + 0.1 * np.eye(n), lower)
    Wc, schur, ok = completion.maxdet_completion(n, lower, X)
    assert ok
    np.testing.assert_array_equal(_values(Wc, lower), X)
    assert np.linalg.eigvalsh(Wc).min() > 0
    Winv = np.linalg.inv(Wc)
    assert np.abs(Winv[_off_pattern_mask(n, lower)]).max(initial=0.0) <= 1e-9 * np.abs(Winv).max()
    assert completion.logdet(schur) == pytest.approx(np.linalg.slogdet(Wc)[1], rel=1e-9, abs=1e-9)
