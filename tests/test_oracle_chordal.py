"""Pins for the oracle's chordal preprocessing (CPU only)."""
import os

import networkx as nx
import numpy as np
import pytest

from oracle import admm, chordal
from paper_1707_05058_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig1():
    n, edges, fill, cliques = 0, [], [], []
    with open(os.path.join(GOLD, "fig1_chordal.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
            elif tok[0] == "edge":
                edges.append((int(tok[1]) - 1, int(tok[2]) - 1))
            elif tok[0] == "fill":
                fill.append((int(tok[1]) - 1, int(tok[2]) - 1))
            elif tok[0] == "clique":
                cliques.append(tuple(int(t) - 1 for t in tok[1:]))
    return n, edges, fill, cliques


def test_fig1_worked_example():
    n, edges, fill, cliques = _read_fig1()
    rows = [max(e) for e in edges]
    cols = [min(e) for e in edges]
    got_cliques, lower, nfill, is_chordal = chordal.chordal_decomposition(n, [(rows, cols)])
    assert not is_chordal
    assert got_cliques == cliques
    assert nfill == len(fill)
    off = {e for e in lower if e[0] != e[1]}
    assert off == {(max(e), min(e)) for e in edges} | {(max(e), min(e)) for e in fill}


def test_selector_example_section_2_2():
    """E_C1 X E_C1^T picks rows/cols {1,2,4}; E_C1^T Y E_C1 puts Y back with
    zeros in row/column 3 (Section 2.2 example)."""
    n, edges, _, _ = _read_fig1()
    prob = W.SDPProblem(n, 1, np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32),
                        np.ones(1), np.ones(1),
                        np.array([max(e) for e in edges], np.int32), np.array([min(e) for e in edges], np.int32),
                        np.ones(len(edges)), np.zeros(0, np.int32), np.zeros(0, np.int32))
    dp = admm.decompose(prob)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, n)); X = X + X.T
    X[0, 2] = X[2, 0] = 0.0          # (1,3) is outside the extended pattern
    x = np.zeros(dp.N)
    for (i, j), k in dp.full_index.items():
        x[k] = X[i, j]
    sel = [0, 1, 3]
    blk = dp.H(x)[dp.offsets[0]:dp.offsets[1]].reshape(3, 3, order="F")
    np.testing.assert_array_equal(blk, X[np.ix_(sel, sel)])
    Y = rng.standard_normal((3, 3)); Y = Y + Y.T
    s = np.zeros(dp.nd)
    s[dp.offsets[0]:dp.offsets[1]] = Y.reshape(-1, order="F")
    back = dp.HT(s)
    full = np.zeros((n, n))
    for (i, j), k in dp.full_index.items():
        full[i, j] = back[k]
    expect = np.zeros((n, n))
    expect[np.ix_(sel, sel)] = Y
    np.testing.assert_array_equal(full, expect)


@pytest.mark.parametrize("l,d,h", [(5, 10, 5), (3, 4, 2), (7, 3, 6)])
def test_block_arrow_closed_form(l, d, h):
    """Section 7.4: the block-arrow pattern is chordal with l maximal cliques
    of size d + h (block k plus the arrow head)."""
    rows, cols = W._lower_pairs_block_arrow(l, d, h)
    cl, lower, nfill, is_chordal = chordal.chordal_decomposition(l * d + h, [(rows, cols)])
    assert is_chordal and nfill == 0
    head = tuple(range(l * d, l * d + h))
    assert cl == [tuple(range(k * d, (k + 1) * d)) + head for k in range(l)]


@pytest.mark.parametrize("n,w", [(20, 3), (2000, 10), (9, 8)])
def test_banded_closed_form(n, w):
    """A banded pattern with half-bandwidth w is chordal with n - w maximal
    cliques {i, ..., i + w} of size w + 1."""
    rows, cols = W._lower_pairs_banded(n, w)
    cl, lower, nfill, is_chordal = chordal.chordal_decomposition(n, [(rows, cols)])
    assert is_chordal and nfill == 0
    assert cl == [tuple(range(i, i + w + 1)) for i in range(n - w)]


def _random_graph(rng, n, p):
    edges = [(i, j) for i in range(n) for j in range(i) if rng.random() < p]
    return edges


@pytest.mark.parametrize("seed", range(12))
def test_extension_against_networkx(seed):
    """Independent library check: the extension is chordal, contains the input
    edges, and the cliques are exactly its maximal cliques."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 13))
    edges = _random_graph(rng, n, float(rng.uniform(0.15, 0.6)))
    rows = [e[0] for e in edges]; cols = [e[1] for e in edges]
    cl, lower, nfill, is_chordal = chordal.chordal_decomposition(n, [(rows, cols)])
    G = nx.Graph(); G.add_nodes_from(range(n)); G.add_edges_from(edges)
    H = nx.Graph(); H.add_nodes_from(range(n))
    H.add_edges_from([(i, j) for (i, j) in lower if i != j])
    assert nx.is_chordal(H)
    assert set(G.edges()) <= {tuple(sorted(e, reverse=True)) for e in H.edges()} | set(H.edges())
    assert is_chordal == nx.is_chordal(G)
    if is_chordal:
        assert nfill == 0
    want = sorted(tuple(sorted(c)) for c in nx.find_cliques(H))
    assert cl == want
    # every lower entry of the extension lies in some clique
    for (i, j) in lower:
        assert any(i in c and j in c for c in cl)


def test_min_degree_tie_break():
    """Path-of-cliques graph K4 - v - K4: v has the minimum degree (2) and is
    eliminated first, which joins its two neighbours (a fill edge) even though
    the graph is chordal.  Chordal inputs therefore take the MCS order and get
    no fill, while the minimum-degree game alone would add one."""
    a = [0, 1, 2, 3]; b = [5, 6, 7, 8]; v = 4
    edges = [(x, y) for grp in (a, b) for i, x in enumerate(grp) for y in grp[:i]]
    edges += [(v, 3), (5, v)]
    n = 9
    adj = chordal.adjacency(n, {(max(e), min(e)) for e in edges})
    elim, filled = chordal.min_degree_elimination(n, adj)
    assert elim[0] == v
    assert 5 in filled[3]
    rows = [max(e) for e in edges]; cols = [min(e) for e in edges]
    cl, lower, nfill, is_chordal = chordal.chordal_decomposition(n, [(rows, cols)])
    assert is_chordal and nfill == 0
    assert cl == [(0, 1, 2, 3), (3, 4), (4, 5), (5, 6, 7, 8)]


def test_rejects_upper_entries():
    with pytest.raises(ValueError):
        chordal.chordal_decomposition(3, [([0], [1])])
