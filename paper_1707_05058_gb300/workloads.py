"""Seeded synthetic SDP instances (inputs only; no solver arithmetic).

Every instance is a standard-form SDP (Section 1, Eqs. PrimalSDP/DualSDP)

    min <C, X>  s.t.  <A_i, X> = b_i (i = 1..m),  X PSD

given as 0-based lower-triangle triplets (row >= col).  A_i is the symmetric
matrix whose lower triangle holds the listed values.  Off-diagonal entries
count twice in <A_i, X>.

The random families follow the block-arrow recipe of Section 7.4 (a strictly
feasible X0 gives b, a strictly feasible (y0, Z0) gives C) with N(0,1) draws
instead of the paper's U(0,1).  Every random value is rounded to float32 and
stored as float64, so float32 and float64 consumers read identical numbers.
The derived data (b, C) are rounded to float32 too.

Both the CUDA library tests and the CPU oracle read instances from here;
this module holds none of the solver's arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class SDPProblem:
    n: int
    m: int
    A_con: np.ndarray   # int32 [nnzA], constraint index in [0, m)
    A_row: np.ndarray   # int32 [nnzA], row >= col
    A_col: np.ndarray   # int32 [nnzA]
    A_val: np.ndarray   # float64 [nnzA]
    b: np.ndarray       # float64 [m]
    C_row: np.ndarray   # int32 [nnzC]
    C_col: np.ndarray   # int32 [nnzC]
    C_val: np.ndarray   # float64 [nnzC]
    P_row: np.ndarray   # int32 [nnzP] extra pattern edges (may be empty)
    P_col: np.ndarray
    name: str = ""
    optimum: float | None = None   # known optimal <C,X> when a closed form exists

    def arrays(self):
        """Contiguous arrays in the order the C ABI takes them."""
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        return (i32(self.A_con), i32(self.A_row), i32(self.A_col), f64(self.A_val), f64(self.b),
                i32(self.C_row), i32(self.C_col), f64(self.C_val), i32(self.P_row), i32(self.P_col))


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _empty_i32():
    return np.zeros(0, dtype=np.int32)


def _lower_pairs_block_arrow(l, d, h):
    """Lower-triangle (row, col) pairs, diagonal included, of the block-arrow
    pattern of Fig. BlockArrowSDP: l diagonal d x d blocks, then an arrow head
    of h rows/columns coupled to everything."""
    rows, cols = [], []
    for blk in range(l):
        base = blk * d
        for i in range(d):
            for j in range(i + 1):
                rows.append(base + i)
                cols.append(base + j)
    nb = l * d
    for i in range(nb, nb + h):
        for j in range(i + 1):
            rows.append(i)
            cols.append(j)
    return np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64)


def _lower_pairs_banded(n, w):
    rows, cols = [], []
    for j in range(n):
        for i in range(j, min(n, j + w + 1)):
            rows.append(i)
            cols.append(j)
    return np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64)


def _feasible_data(rng, n, m, prow, pcol, A_con, A_ent, A_val, x0_of=None):
    """b from a strictly feasible X0 = G G^T + I and C = Z0 + sum y0_i A_i with
    Z0 = W + alpha I (W N(0,1) on the pattern, alpha a Gershgorin bound).
    `x0_of(G)`, when given, returns G G^T on the pattern entries (a faster
    route for structured patterns)."""
    npat = prow.size
    wgt = np.where(prow == pcol, 1.0, 2.0)
    G = rng.standard_normal((n, n))
    if x0_of is not None:
        x0 = x0_of(G)
    else:
        x0 = np.empty(npat)
        chunk = 1 << 14
        for s in range(0, npat, chunk):
            e = slice(s, s + chunk)
            x0[e] = np.einsum("ij,ij->i", G[prow[e]], G[pcol[e]])
    x0 += (prow == pcol)
    b = np.bincount(A_con, weights=wgt[A_ent] * A_val * x0[A_ent], minlength=m)
    W = rng.standard_normal(npat)
    absrow = np.bincount(prow, weights=np.abs(W), minlength=n)
    absrow += np.bincount(pcol, weights=np.where(prow == pcol, 0.0, np.abs(W)), minlength=n)
    alpha = absrow.max() + 1.0
    z0 = W + alpha * (prow == pcol)
    y0 = rng.standard_normal(m)
    c = z0 + np.bincount(A_ent, weights=A_val * y0[A_con], minlength=npat)
    return _f32(b), _f32(c)


def _bernoulli_positions(rng, total, density):
    """Sorted positions in [0, total) of a Bernoulli(density) process, drawn
    as geometric gaps (O(density * total) draws instead of `total`)."""
    est = int(total * density * 1.1) + 64
    pos = np.cumsum(rng.geometric(density, size=est)) - 1
    while pos[-1] < total:
        more = pos[-1] + np.cumsum(rng.geometric(density, size=est))
        pos = np.concatenate([pos, more])
    return pos[pos < total]


def block_arrow(l, d, h, m, seed, name=None, density=None):
    """Random block-arrow SDP (Section 7.4 recipe, N(0,1) draws): every A_i is
    dense on the lower block-arrow pattern, or, with `density`, each lower
    pattern entry of each A_i is nonzero with that probability."""
    rng = np.random.default_rng(seed)
    n = l * d + h
    prow, pcol = _lower_pairs_block_arrow(l, d, h)
    npat = prow.size
    if density is None:
        A_val = _f32(rng.standard_normal((m, npat))).ravel()
        A_con = np.repeat(np.arange(m), npat)
        A_ent = np.tile(np.arange(npat), m)
    else:
        pos = _bernoulli_positions(rng, m * npat, density)
        A_con, A_ent = pos // npat, pos % npat
        A_val = _f32(rng.standard_normal(pos.size))

    def x0_of(G):  # G G^T on the pattern from l diagonal-block products and the head rows
        x0 = np.empty(npat)
        nb = l * d
        for blk in range(l):
            sel = (pcol >= blk * d) & (pcol < (blk + 1) * d) & (prow < nb)
            B = G[blk * d:(blk + 1) * d]
            x0[sel] = (B @ B.T)[prow[sel] - blk * d, pcol[sel] - blk * d]
        sel = prow >= nb
        x0[sel] = (G[nb:] @ G.T)[prow[sel] - nb, pcol[sel]]
        return x0

    b, c = _feasible_data(rng, n, m, prow, pcol, A_con, A_ent, A_val, x0_of if density is not None else None)
    return SDPProblem(n, m, A_con.astype(np.int32), prow[A_ent].astype(np.int32),
                      pcol[A_ent].astype(np.int32), A_val, b,
                      prow.astype(np.int32), pcol.astype(np.int32), c,
                      _empty_i32(), _empty_i32(),
                      name or f"block_arrow_l{l}_d{d}_h{h}_m{m}")


def banded(n, w, m, seed, density=0.05, name=None):
    """Random banded SDP: half-bandwidth w, each lower band entry of each A_i
    nonzero with probability `density`, N(0,1) values."""
    rng = np.random.default_rng(seed)
    prow, pcol = _lower_pairs_banded(n, w)
    npat = prow.size
    mask = rng.random((m, npat)) < density
    A_con, A_ent = np.nonzero(mask)
    A_val = _f32(rng.standard_normal(A_con.size))
    b, c = _feasible_data(rng, n, m, prow, pcol, A_con, A_ent, A_val)
    return SDPProblem(n, m, A_con.astype(np.int32), prow[A_ent].astype(np.int32),
                      pcol[A_ent].astype(np.int32), A_val, b,
                      prow.astype(np.int32), pcol.astype(np.int32), c,
                      _empty_i32(), _empty_i32(), name or f"banded_n{n}_w{w}_m{m}")


def maxcut(n, avg_degree, seed, name=None):
    """MaxCut relaxation on a G(n, p) graph with p = avg_degree/(n-1) and
    U(0,1) edge weights: min <-L/4, X> s.t. X_ii = 1."""
    rng = np.random.default_rng(seed)
    p = avg_degree / (n - 1)
    # draw edges row by row to keep memory at O(edges)
    er, ec = [], []
    for i in range(1, n):
        hits = np.nonzero(rng.random(i) < p)[0]
        er.append(np.full(hits.size, i))
        ec.append(hits)
    er = np.concatenate(er)
    ec = np.concatenate(ec)
    wts = _f32(rng.random(er.size))
    deg = np.bincount(er, weights=wts, minlength=n) + np.bincount(ec, weights=wts, minlength=n)
    C_row = np.concatenate([np.arange(n), er])
    C_col = np.concatenate([np.arange(n), ec])
    C_val = _f32(np.concatenate([-deg / 4.0, wts / 4.0]))
    A_con = np.arange(n)
    return SDPProblem(n, n, A_con.astype(np.int32), A_con.astype(np.int32), A_con.astype(np.int32),
                      np.ones(n), np.ones(n), C_row.astype(np.int32), C_col.astype(np.int32), C_val,
                      _empty_i32(), _empty_i32(), name or f"maxcut_n{n}_deg{avg_degree}")


def block_arrow_batch(count, seed, density=0.05, l_range=(10, 100), d_range=(10, 40), h_range=(10, 20),
                      m_range=(50, 400)):
    """Batch of block-arrow SDPs of uneven size: l, d, h, m uniform on the
    given inclusive ranges, each problem with its own seed; A_i sparse on the
    pattern with the given density (None: dense on the pattern)."""
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(l_range[0], l_range[1] + 1)), int(rng.integers(d_range[0], d_range[1] + 1)),
               int(rng.integers(h_range[0], h_range[1] + 1)), int(rng.integers(m_range[0], m_range[1] + 1)))
              for _ in range(count)]
    return [block_arrow(l, d, h, m, seed + 1 + i, density=density) for i, (l, d, h, m) in enumerate(shapes)]


def block_arrow_batch_member(count, seed, index, density=0.05, l_range=(10, 100), d_range=(10, 40),
                            h_range=(10, 20), m_range=(50, 400)):
    """Problem `index` of block_arrow_batch(count, seed, ...) alone (the same
    shape and seed), without generating the others."""
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(l_range[0], l_range[1] + 1)), int(rng.integers(d_range[0], d_range[1] + 1)),
               int(rng.integers(h_range[0], h_range[1] + 1)), int(rng.integers(m_range[0], m_range[1] + 1)))
              for _ in range(count)]
    l, d, h, m = shapes[index]
    return block_arrow(l, d, h, m, seed + 1 + index, density=density)


def workload_batch_member(index: int, member: int):
    """Member `member` of the batched workload `index` (2: 256 block-arrows)."""
    if index == 2:
        return block_arrow_batch_member(256, 3707, member)
    raise ValueError(index)


def direct_sum(problems, name=None):
    """The block-diagonal SDP whose summands are `problems`: vertices and
    constraints of problem j are shifted past those of problems 0..j-1.  Its
    optimum is the sum of theirs."""
    vo = np.cumsum([0] + [p.n for p in problems])
    mo = np.cumsum([0] + [p.m for p in problems])
    cat = lambda f, sh: np.concatenate([getattr(p, f).astype(np.int64) + s for p, s in zip(problems, sh)]).astype(np.int32)
    opt = None
    if all(p.optimum is not None for p in problems):
        opt = float(sum(p.optimum for p in problems))
    return SDPProblem(int(vo[-1]), int(mo[-1]), cat("A_con", mo), cat("A_row", vo), cat("A_col", vo),
                      np.concatenate([p.A_val for p in problems]), np.concatenate([p.b for p in problems]),
                      cat("C_row", vo), cat("C_col", vo), np.concatenate([p.C_val for p in problems]),
                      cat("P_row", vo), cat("P_col", vo),
                      name or "direct_sum_" + "+".join(p.name for p in problems), opt)


def pd_on_pattern(n, rows, cols, seed, rank=16, shift=0.5):
    """Entries (rows[k], cols[k]) of the positive definite matrix
    shift I + U U^T, U an n x rank matrix of N(0, 1/rank) draws: a partial
    matrix every clique block of which is positive definite (input of the
    maximum-determinant completion)."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, rank)) / math.sqrt(rank)
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    return np.einsum("kr,kr->k", U[rows], U[cols]) + np.where(rows == cols, shift, 0.0)


def banded_batch(count, n, w, m, seed):
    return [banded(n, w, m, seed + 1 + i) for i in range(count)]


# ---------------------------------------------------------------------------
# Instances with a known optimum (closed forms), used to pin the solvers.

def lambda_max_tridiagonal(n, a, bb):
    """lambda_max(S) = min t s.t. tI - S PSD; its primal is
    min <-S, X> s.t. <I, X> = 1, optimum -lambda_max(S).  S is tridiagonal
    Toeplitz (a on the diagonal, bb off it): lambda_max = a + 2|bb| cos(pi/(n+1)).
    The pattern is banded with half-bandwidth 1 (n-1 cliques of size 2)."""
    i = np.arange(n)
    C_row = np.concatenate([i, i[1:]])
    C_col = np.concatenate([i, i[:-1]])
    C_val = np.concatenate([np.full(n, -a, dtype=np.float64), np.full(n - 1, -bb, dtype=np.float64)])
    opt = -(a + 2 * abs(bb) * math.cos(math.pi / (n + 1)))
    return SDPProblem(n, 1, np.zeros(n, np.int32), i.astype(np.int32), i.astype(np.int32),
                      np.ones(n), np.ones(1), C_row.astype(np.int32), C_col.astype(np.int32), C_val,
                      _empty_i32(), _empty_i32(), f"lambda_max_tridiag_n{n}", opt)


def lovasz_theta_cycle(n=5):
    """Lovasz theta of the n-cycle: max <J, X> s.t. tr X = 1, X_ij = 0 on the
    cycle's edges.  theta(C_5) = sqrt(5).  J is dense, so the pattern is
    complete and there is one clique (p = 1)."""
    rows, cols = np.tril_indices(n)
    C_val = -np.ones(rows.size)
    con, r, c, v = [], [], [], []
    for i in range(n):
        con.append(0); r.append(i); c.append(i); v.append(1.0)
    bvec = [1.0]
    for k in range(n):
        i, j = max(k, (k + 1) % n), min(k, (k + 1) % n)
        con.append(len(bvec)); r.append(i); c.append(j); v.append(1.0)
        bvec.append(0.0)
    opt = -n * math.cos(math.pi / n) / (1 + math.cos(math.pi / n)) if n % 2 else None
    return SDPProblem(n, len(bvec), np.array(con, np.int32), np.array(r, np.int32), np.array(c, np.int32),
                      np.array(v), np.array(bvec), rows.astype(np.int32), cols.astype(np.int32), C_val,
                      _empty_i32(), _empty_i32(), f"lovasz_theta_C{n}", opt)


def maxcut_cycle(n):
    """MaxCut relaxation of the unit-weight n-cycle: min <-L/4, X> s.t. X_ii = 1.
    Optimum -(n/2)(1 + cos(pi/n)) for odd n, -n for even n.  The cycle is not
    chordal, so the decomposition needs fill edges."""
    i = np.arange(n)
    er = np.array([max(k, (k + 1) % n) for k in range(n)])
    ec = np.array([min(k, (k + 1) % n) for k in range(n)])
    C_row = np.concatenate([i, er])
    C_col = np.concatenate([i, ec])
    C_val = np.concatenate([np.full(n, -0.5), np.full(n, 0.25)])
    opt = -(n / 2) * (1 + math.cos(math.pi / n)) if n % 2 else -float(n)
    return SDPProblem(n, n, i.astype(np.int32), i.astype(np.int32), i.astype(np.int32), np.ones(n), np.ones(n),
                      C_row.astype(np.int32), C_col.astype(np.int32), C_val, _empty_i32(), _empty_i32(),
                      f"maxcut_cycle_C{n}", opt)


def primal_infeasible():
    """<I, X> = -1 has no PSD solution (certificate y = -1: -y I = I PSD and
    b^T y = 1 > 0).  Pattern: two 2x2 blocks."""
    n = 4
    C_row = np.array([0, 1, 1, 2, 3, 3], np.int32)
    C_col = np.array([0, 0, 1, 2, 2, 3], np.int32)
    C_val = np.array([1.0, 0.5, 2.0, 1.0, -0.25, 1.5])
    i = np.arange(n, dtype=np.int32)
    return SDPProblem(n, 1, np.zeros(n, np.int32), i, i, np.ones(n), np.array([-1.0]),
                      C_row, C_col, C_val, _empty_i32(), _empty_i32(), "primal_infeasible")


def dual_infeasible():
    """C = -e_0 e_0^T with the single constraint X_11 = 1 on the path pattern
    0-1-2: the ray X = e_0 e_0^T is feasible with <C, ray> = -1 < 0, so the
    primal is unbounded and the dual infeasible."""
    C_row = np.array([0, 1, 2, 1], np.int32)
    C_col = np.array([0, 0, 1, 1], np.int32)
    C_val = np.array([-1.0, 0.0, 0.0, 0.0])
    return SDPProblem(3, 1, np.zeros(1, np.int32), np.array([1], np.int32), np.array([1], np.int32),
                      np.ones(1), np.ones(1), C_row, C_col, C_val, _empty_i32(), _empty_i32(),
                      "dual_infeasible")


def random_chordal_small(n, m, seed, extra_edges=0):
    """Tiny random SDP on a random (usually non-chordal) pattern, strictly
    feasible by construction; used for decomposition-equivalence tests."""
    rng = np.random.default_rng(seed)
    pairs = {(i, i) for i in range(n)}
    for i in range(1, n):
        pairs.add((i, int(rng.integers(0, i))))
    for _ in range(extra_edges):
        i, j = sorted(rng.choice(n, 2, replace=False))[::-1]
        pairs.add((int(i), int(j)))
    pairs = sorted(pairs, key=lambda t: (t[1], t[0]))
    prow = np.array([p[0] for p in pairs])
    pcol = np.array([p[1] for p in pairs])
    npat = prow.size
    A_val = _f32(rng.standard_normal((m, npat))).ravel()
    A_con = np.repeat(np.arange(m), npat)
    A_ent = np.tile(np.arange(npat), m)
    b, c = _feasible_data(rng, n, m, prow, pcol, A_con, A_ent, A_val)
    return SDPProblem(n, m, A_con.astype(np.int32), prow[A_ent].astype(np.int32), pcol[A_ent].astype(np.int32),
                      A_val, b, prow.astype(np.int32), pcol.astype(np.int32), c, _empty_i32(), _empty_i32(),
                      f"random_small_n{n}_m{m}_s{seed}")


def dense_pattern(prob: SDPProblem) -> SDPProblem:
    """The same SDP with every lower entry added to the pattern (one clique)."""
    r, c = np.tril_indices(prob.n)
    return dataclasses.replace(prob, P_row=r.astype(np.int32), P_col=c.astype(np.int32),
                               name=prob.name + "_dense")


def random_symmetric_batch(count, s, seed, scale=1.0):
    """`count` random symmetric s x s matrices (float32-representable), N(0,1)."""
    rng = np.random.default_rng(seed)
    g = _f32(rng.standard_normal((count, s, s)) * scale)
    return _f32(0.5 * (g + np.transpose(g, (0, 2, 1))))


# The five workloads (seed = 1707 + 1000 * index).
def workload(index: int):
    if index == 0:
        return block_arrow(5, 10, 5, 30, 1707, name="block_arrow_n55_m30")
    if index == 1:
        return banded(2000, 10, 500, 2707, name="banded_n2000_w10_m500")
    if index == 2:
        return block_arrow_batch(256, 3707)
    if index == 3:
        return maxcut(10000, 6, 4707, name="maxcut_gnp_n10000_deg6")
    if index == 4:
        return banded_batch(64, 500, 8, 200, 5707)
    raise ValueError(index)
