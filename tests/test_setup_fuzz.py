"""Randomised agreement of the library's host setup with the oracle's chordal
decomposition (Section 2.1; minimum-degree extension with ties to the
smallest vertex): on random graphs, mostly not chordal and with many ties, the
cliques, the extended pattern and the fill agree bit for bit.  Host only."""
import numpy as np
import pytest

from oracle import chordal

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from paper_1707_05058_gb300.workloads import SDPProblem, _empty_i32  # noqa: E402


def _problem(n, edges):
    rows = np.array([max(i, j) for i, j in edges] + list(range(n)), np.int32)
    cols = np.array([min(i, j) for i, j in edges] + list(range(n)), np.int32)
    vals = np.ones(rows.size)
    i = np.arange(n, dtype=np.int32)
    return SDPProblem(n, n, i, i, i, np.ones(n), np.ones(n), rows, cols, vals, _empty_i32(), _empty_i32(), "fuzz")


@st.composite
def graphs(draw):
    n = draw(st.integers(min_value=2, max_value=80))
    p = draw(st.floats(min_value=0.02, max_value=0.5))
    seed = draw(st.integers(min_value=0, max_value=2**31 - 1))
    rng = np.random.default_rng(seed)
    edges = [(i, j) for i in range(n) for j in range(i) if rng.random() < p]
    return n, edges


@settings(max_examples=300, deadline=None)
@given(graphs())
def test_setup_matches_oracle_on_random_graphs(lib, g):
    n, edges = g
    prob = _problem(n, edges)
    P = lib.Problem(prob)
    cl, lower, nfill, is_chordal = chordal.chordal_decomposition(n, [(prob.C_row, prob.C_col)])
    assert P.clique_list() == cl
    r, c = P.pattern()
    assert list(zip(r.tolist(), c.tolist())) == lower
    assert P.info["n_fill"] == nfill
    assert bool(P.info["chordal"]) == is_chordal
