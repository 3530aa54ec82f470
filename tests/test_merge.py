"""Clique merging (an option of the setup, CDSDP_SETUP_MERGE_CLIQUES; not in
the paper): the oracle's rule is pinned by a closed form and by invariants,
and the library's host setup must reproduce it bit for bit (cliques, extended
pattern, fill count)."""
import networkx as nx
import numpy as np
import pytest

from oracle import admm, chordal
from paper_1707_05058_gb300 import workloads as W


def test_banded_closed_form():
    """Banded pattern, half-bandwidth w: maximal cliques {i..i+w}, the clique
    tree is the path (weights w), every adjacent pair gains
    2 (w+1)^3 - (w+2)^3 > 0 (w >= 3), while a merged clique of w+2 and the
    next one would lose (w+2)^3 + (w+1)^3 - (w+3)^3 < 0 (w <= 4), so for
    w = 3, 4 the cliques merge in pairs from the left: {2k .. 2k+w+1}, with a
    trailing clique left alone."""
    for n, w in [(20, 3), (17, 4), (31, 3), (40, 4)]:
        cl = [tuple(range(i, i + w + 1)) for i in range(n - w)]
        got = chordal.merge_cliques(cl)
        want = [tuple(range(2 * k, 2 * k + w + 2)) for k in range((n - w) // 2)]
        if (n - w) % 2:
            want.append(cl[-1])
        assert got == sorted(want)


def test_fig1_example_unchanged():
    """The paper's 4-cycle example (cliques {1,2,4}, {2,3,4}): merging them
    would cost 4^3 > 2 * 3^3, so nothing merges."""
    assert chordal.merge_cliques([(0, 1, 3), (1, 2, 3)]) == [(0, 1, 3), (1, 2, 3)]


@pytest.mark.parametrize("seed", range(8))
def test_merge_invariants(seed):
    """On the minimum-degree extension of a random graph: every original
    clique lies inside a merged one, the merged pattern is chordal with
    exactly the merged cliques as its maximal cliques, and the projection
    work sum |C|^3 does not grow."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 60))
    g = nx.gnp_random_graph(n, 4.0 / n, seed=seed)
    edges = [(max(a, b), min(a, b)) for a, b in g.edges()]
    rows = [e[0] for e in edges]
    cols = [e[1] for e in edges]
    cl, lower, nfill, _ = chordal.chordal_decomposition(n, [(rows, cols)])
    mc, mlower, mnfill, _ = chordal.chordal_decomposition(n, [(rows, cols)], merge=True)
    for c in cl:
        assert any(set(c) <= set(m) for m in mc)
    assert sum(len(c) ** 3 for c in mc) <= sum(len(c) ** 3 for c in cl)
    h = nx.Graph()
    h.add_nodes_from(range(n))
    h.add_edges_from((i, j) for i, j in mlower if i != j)
    assert nx.is_chordal(h)
    assert sorted(tuple(sorted(c)) for c in nx.find_cliques(h)) == mc
    assert set(lower) <= set(mlower)
    assert mnfill == len(mlower) - n - len(set(edges))


def _compare_merged(lib, prob):
    P = lib.Problem(prob, merge_cliques=True)
    dp = admm.decompose(prob, merge=True)
    assert P.clique_list() == dp.cliques
    r, c = P.pattern()
    assert list(zip(r.tolist(), c.tolist())) == dp.lower
    assert P.info["n_fill"] == dp.nfill
    assert P.info["max_clique"] == max(len(k) for k in dp.cliques)
    return P


@pytest.mark.parametrize("seed", range(6))
def test_library_merge_matches_oracle_maxcut(lib, seed):
    _compare_merged(lib, W.maxcut(int(60 + 20 * seed), 6, 300 + seed, name=f"mc{seed}"))


@pytest.mark.parametrize("prob", [W.banded(40, 3, 8, seed=2, density=0.3), W.block_arrow(4, 5, 3, 6, seed=9),
                                  W.maxcut_cycle(11)], ids=lambda p: p.name)
def test_library_merge_matches_oracle_families(lib, prob):
    _compare_merged(lib, prob)


def test_merged_handle_refuses_completion(lib):
    P = lib.Problem(W.maxcut(80, 6, 5, name="mc80"), merge_cliques=True)
    with pytest.raises(lib.CdsdpError):
        P.completion_sizes()
