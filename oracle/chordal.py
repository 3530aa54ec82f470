"""Oracle: chordal extension and maximal cliques (plain Python, no speed tricks).

Test infrastructure only.  Nothing in the product path (the CUDA library, its
binding, or bench.py's timed arms) may import this module.

Follows Section 2.1 (chordal graphs, maximal cliques, chordal extension) and
the data-preprocessing step of Algorithms 1-3 (Section 7.1.1: chordal
extension from a minimum-degree elimination, maximal cliques read off it).

Canonical rules (the paper does not fix them; the CUDA library's host setup
implements the same rules independently so both sides agree bit for bit):
  * aggregate pattern E* = union of the patterns of C, every A_i and the
    optional extra edges, plus every diagonal entry (Section 2.1, E*).
  * chordality is tested with maximum cardinality search (Tarjan and
    Yannakakis): unnumbered vertex with most numbered neighbours next, ties to
    the smallest index; the reverse visiting order must be a perfect
    elimination order.  A chordal pattern gets no fill and that order.
  * otherwise the exact minimum-degree elimination game is run (ties to the
    smallest index); eliminating v joins all its remaining neighbours.
  * candidate cliques {v} U {later neighbours of v}; the maximal ones are
    kept; each clique is sorted ascending (Section 2.1, natural ordering) and
    the clique list is sorted lexicographically.
"""
from __future__ import annotations


def aggregate_edges(n, pairs_iterables):
    """Set of off-diagonal edges (i, j), i > j, from (row, col) iterables."""
    edges = set()
    for rows, cols in pairs_iterables:
        for r, c in zip(rows, cols):
            r = int(r); c = int(c)
            if not (0 <= r < n and 0 <= c < n):
                raise ValueError("index out of range")
            if r < c:
                raise ValueError("upper-triangle entry given; only row >= col is accepted")
            if r != c:
                edges.add((r, c))
    return edges


def adjacency(n, edges):
    adj = [set() for _ in range(n)]
    for i, j in edges:
        adj[i].add(j)
        adj[j].add(i)
    return adj


def mcs_visit_order(n, adj):
    """Maximum cardinality search; returns the visiting order."""
    numbered = [False] * n
    weight = [0] * n
    order = []
    for _ in range(n):
        best = -1
        for v in range(n):
            if not numbered[v] and (best < 0 or weight[v] > weight[best]):
                best = v
        numbered[best] = True
        order.append(best)
        for u in adj[best]:
            if not numbered[u]:
                weight[u] += 1
    return order


def is_perfect_elimination_order(elim, adj):
    """True when, for every v, its neighbours eliminated after v form a clique."""
    pos = {v: k for k, v in enumerate(elim)}
    for v in elim:
        later = [u for u in adj[v] if pos[u] > pos[v]]
        for a in range(len(later)):
            for b in range(a + 1, len(later)):
                if later[b] not in adj[later[a]]:
                    return False
    return True


def min_degree_elimination(n, adj):
    """Elimination game with exact minimum degree (ties to smallest index).
    Returns (elimination order, filled adjacency)."""
    work = [set(s) for s in adj]
    filled = [set(s) for s in adj]
    alive = set(range(n))
    elim = []
    for _ in range(n):
        v = min(alive, key=lambda u: (len(work[u]), u))
        nb = list(work[v])
        for a in range(len(nb)):
            for b in range(a + 1, len(nb)):
                x, y = nb[a], nb[b]
                if y not in work[x]:
                    work[x].add(y); work[y].add(x)
                    filled[x].add(y); filled[y].add(x)
        for u in nb:
            work[u].discard(v)
        work[v] = set()
        alive.discard(v)
        elim.append(v)
    return elim, filled


def cliques_from_elimination(elim, filled):
    """Maximal cliques of a chordal graph given a perfect elimination order."""
    pos = {v: k for k, v in enumerate(elim)}
    cand = {}
    for v in elim:
        cand[v] = frozenset([v] + [u for u in filled[v] if pos[u] > pos[v]])
    maximal = []
    for v in elim:
        kv = cand[v]
        # any strict superset K_u of K_v contains v as a later neighbour of u
        contained = any(v in filled[u] and pos[u] < pos[v] and kv <= cand[u] for u in filled[v])
        if not contained:
            maximal.append(tuple(sorted(kv)))
    return sorted(set(maximal))


def merge_cliques(cliques):
    """Coarser clique cover of a further chordal extension (an option, not in
    the paper): merge cliques adjacent in a clique tree while that lowers the
    projection work sum |C|^3.

    Clique tree: the maximum-weight spanning forest of the clique intersection
    graph (a clique tree of a chordal graph is exactly such a forest), built by
    Kruskal's rule over the pairs i < j with |C_i & C_j| > 0 in the order
    (weight descending, i ascending, j ascending).  Then, as long as some tree
    edge has a positive gain |C_i|^3 + |C_j|^3 - |C_i | C_j|^3, the edge with
    the largest gain (ties: smaller min(i, j), then smaller max(i, j)) is
    contracted: node min(i, j) holds the union and takes over the other
    node's tree edges.  Returns the cliques, each ascending, in lexicographic
    order.  Plain search over all pairs and edges (small inputs only)."""
    sets = [set(c) for c in cliques]
    p = len(sets)
    pairs = []
    for i in range(p):
        for j in range(i + 1, p):
            w = len(sets[i] & sets[j])
            if w > 0:
                pairs.append((-w, i, j))
    pairs.sort()
    root = list(range(p))

    def find(x):
        while root[x] != x:
            x = root[x]
        return x

    tree = set()
    for _, i, j in pairs:
        ri, rj = find(i), find(j)
        if ri != rj:
            root[ri] = rj
            tree.add((i, j))
    while True:
        best = None
        for i, j in tree:
            g = len(sets[i]) ** 3 + len(sets[j]) ** 3 - len(sets[i] | sets[j]) ** 3
            key = (-g, i, j)
            if g > 0 and (best is None or key < best):
                best = key
        if best is None:
            break
        _, lo, hi = best
        sets[lo] = sets[lo] | sets[hi]
        sets[hi] = None
        new_tree = set()
        for i, j in tree:
            if (i, j) == (lo, hi):
                continue
            i2 = lo if i == hi else i
            j2 = lo if j == hi else j
            new_tree.add((min(i2, j2), max(i2, j2)))
        tree = new_tree
    return sorted(tuple(sorted(c)) for c in sets if c is not None)


def chordal_decomposition(n, pairs_iterables, merge=False):
    """Returns (cliques, lower edge list of the extended pattern incl. diagonal
    in column-major order, number of fill edges, chordal flag).  With merge,
    the cliques are those of merge_cliques and the extended pattern is every
    pair within one of them."""
    edges = aggregate_edges(n, pairs_iterables)
    adj = adjacency(n, edges)
    elim = list(reversed(mcs_visit_order(n, adj)))
    chordal = is_perfect_elimination_order(elim, adj)
    if chordal:
        filled = adj
    else:
        elim, filled = min_degree_elimination(n, adj)
    cliques = cliques_from_elimination(elim, filled)
    lower = set((i, i) for i in range(n))
    if merge:
        cliques = merge_cliques(cliques)
        for c in cliques:
            for a in range(len(c)):
                for bb in range(a + 1, len(c)):
                    lower.add((c[bb], c[a]))
    else:
        for v in range(n):
            for u in filled[v]:
                lower.add((max(u, v), min(u, v)))
    lower = sorted(lower, key=lambda t: (t[1], t[0]))
    nfill = len(lower) - n - len(edges)
    return cliques, lower, nfill, chordal
