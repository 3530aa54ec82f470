"""Maximum-determinant positive definite completion (Section 7.1.1).

Test infrastructure: the oracle.  Only tests, smoke() and bench.py's CPU
baseline may import this module; nothing in the product path does.

After a solve, the decomposed methods return X only on the extended pattern
E*; Section 7.1.1 builds a full primal matrix from it by the maximum
determinant completion (Grone, Johnson, Sa and Wolkowicz 1984; the chordal
algorithm of Vandenberghe and Andersen, Chapter 10.2).  The completion exists
when every clique block of the partial matrix is positive definite.  It is
the unique positive definite W with W = X on E* and (W^-1)_ij = 0 off E*.

Algorithm written out (dense, plain numpy): take a perfect elimination order
v_1, ..., v_n of the chordal pattern (the reverse of a maximum cardinality
search), and, for k = n-1 down to 1, with N = the neighbours of v_k that come
later in the order (a clique) and L = every vertex that comes later,

    W[j, v_k] = W[j, N] W[N, N]^-1 X[N, v_k]      for j in L \\ N,

the other entries of column v_k being given.  The Schur complements
s_k = X[v_k, v_k] - X[v_k, N] W[N, N]^-1 X[N, v_k] are all positive exactly
when every clique block is positive definite, and log det W = sum_k log s_k.
"""
import numpy as np

from oracle import chordal


def perfect_elimination_order(n, lower):
    """A perfect elimination order of the pattern (list of (i, j), i >= j);
    ValueError when the pattern is not chordal."""
    adj = chordal.adjacency(n, [(i, j) for i, j in lower if i != j])
    elim = list(reversed(chordal.mcs_visit_order(n, adj)))
    if not chordal.is_perfect_elimination_order(elim, adj):
        raise ValueError("pattern is not chordal")
    return elim, adj


def maxdet_completion(n, lower, values):
    """Returns (W dense n x n, schur complements per vertex, ok).  ok is False
    when some Schur complement is not positive (a clique block of the partial
    matrix is not positive definite: no completion); W is then None."""
    elim, adj = perfect_elimination_order(n, lower)
    pos = {v: k for k, v in enumerate(elim)}
    W = np.full((n, n), np.nan)
    for (i, j), x in zip(lower, values):
        W[i, j] = x
        W[j, i] = x
    schur = np.zeros(n)
    for k in range(n - 1, -1, -1):
        v = elim[k]
        N = sorted(u for u in adj[v] if pos[u] > k)
        later = [u for u in elim[k + 1:] if u not in adj[v]]
        if N:
            MN = W[np.ix_(N, N)]
            try:
                np.linalg.cholesky(MN)
            except np.linalg.LinAlgError:
                return None, schur, False
            t = np.linalg.solve(MN, W[N, v])
            schur[v] = W[v, v] - W[v, N] @ t
        else:
            t = np.zeros(0)
            schur[v] = W[v, v]
        if not schur[v] > 0:
            return None, schur, False
        if later:
            col = W[np.ix_(later, N)] @ t if N else np.zeros(len(later))
            W[later, v] = col
            W[v, later] = col
    return W, schur, True


def logdet(schur):
    return float(np.sum(np.log(schur)))
