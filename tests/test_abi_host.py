"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
and its host preprocessing (chordal extension, cliques, pattern) agrees bit
for bit with the oracle.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import admm, chordal
from paper_1707_05058_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "cdsdp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|size_t|const char\*)\s+(cdsdp_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    declared = _declared_symbols()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(so, name), name
    assert sorted(lib.EXPORTED) == declared


def _compare(prob):
    P = pytest.importorskip("paper_1707_05058_gb300.cdsdp").Problem(prob)
    cl, lower, nfill, is_chordal = chordal.chordal_decomposition(
        prob.n, [(prob.C_row, prob.C_col), (prob.A_row, prob.A_col), (prob.P_row, prob.P_col)])
    assert P.clique_list() == cl
    r, c = P.pattern()
    assert list(zip(r.tolist(), c.tolist())) == lower
    assert P.info["n_fill"] == nfill
    assert bool(P.info["chordal"]) == is_chordal
    assert P.info["p"] == len(cl)
    assert P.info["n_d_lower"] == sum(len(k) * (len(k) + 1) // 2 for k in cl)
    return P


@pytest.mark.parametrize("seed", range(25))
def test_setup_matches_oracle_random(lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 30))
    prob = W.random_chordal_small(n, 2, seed=seed, extra_edges=int(rng.integers(0, 3 * n)))
    _compare(prob)


@pytest.mark.parametrize("prob", [W.workload(0), W.maxcut_cycle(9), W.lovasz_theta_cycle(5),
                                  W.lambda_max_tridiagonal(12, 1.0, 0.3), W.primal_infeasible(),
                                  W.dual_infeasible(), W.block_arrow(7, 3, 4, 3, seed=5),
                                  W.banded(60, 4, 10, seed=3, density=0.3)], ids=lambda p: p.name)
def test_setup_matches_oracle_families(lib, prob):
    _compare(prob)


def test_setup_banded_workload_sizes(lib):
    """Banded n=2000, w=10: 1990 cliques of size 11, no fill."""
    P = lib.Problem(W.workload(1))
    assert P.info["p"] == 1990 and P.info["max_clique"] == 11
    assert P.info["chordal"] == 1 and P.info["n_fill"] == 0
    assert P.info["nnz_pattern"] == 2000 * 11 - 55
    assert P.clique_list() == [tuple(range(i, i + 11)) for i in range(1990)]


def test_setup_maxcut_random_matches_oracle(lib):
    prob = W.maxcut(300, 6, seed=9)
    P = _compare(prob)
    assert P.info["diag_factor"] == 1 and P.info["chordal"] == 0


def test_setup_rejects_bad_input(lib):
    good = W.workload(0)
    bad = W.SDPProblem(**{**good.__dict__})
    bad.C_row = good.C_col.copy()
    bad.C_col = good.C_row.copy()        # upper-triangle entries
    with pytest.raises(lib.CdsdpError) as e:
        lib.Problem(bad)
    assert e.value.status == -1
    bad2 = W.SDPProblem(**{**good.__dict__})
    bad2.A_con = good.A_con.copy()
    bad2.A_con[0] = good.m                # constraint index out of range
    with pytest.raises(lib.CdsdpError):
        lib.Problem(bad2)


def test_setup_rank_deficient(lib):
    """Two identical constraints: A D^-1 A^T is singular -> CDSDP_ERR_RANK."""
    p = W.lambda_max_tridiagonal(4, 1.0, 0.5)
    q = W.SDPProblem(p.n, 2, np.concatenate([p.A_con, p.A_con + 1]), np.concatenate([p.A_row, p.A_row]),
                     np.concatenate([p.A_col, p.A_col]), np.concatenate([p.A_val, p.A_val]),
                     np.array([1.0, 1.0]), p.C_row, p.C_col, p.C_val, p.P_row, p.P_col)
    with pytest.raises(lib.CdsdpError) as e:
        lib.Problem(q)
    assert e.value.status == -2


def test_workspace_bytes_without_gpu(lib):
    P = lib.Problem(W.workload(0))
    a, b = P.workspace_bytes(10), P.workspace_bytes(2000)
    assert 0 < a < b and a % 256 == 0


def _summands():
    return [W.block_arrow(3, 4, 2, 6, seed=21), W.banded(15, 3, 7, seed=22, density=0.4),
            W.lovasz_theta_cycle(5), W.block_arrow(2, 5, 3, 9, seed=23, density=0.5)]


def test_components_of_direct_sum(lib):
    """A direct sum has one independent component per summand, numbered in
    vertex order; its cliques are the summands' cliques, shifted."""
    parts = _summands()
    prob = W.direct_sum(parts)
    P = _compare(prob)
    assert P.info["ncomp"] == len(parts)
    vc, rc = P.components()
    np.testing.assert_array_equal(vc, np.repeat(np.arange(len(parts)), [p.n for p in parts]))
    np.testing.assert_array_equal(rc, np.repeat(np.arange(len(parts)), [p.m for p in parts]))
    shifted, vo = [], 0
    for q in parts:
        shifted += [tuple(v + vo for v in cl) for cl in lib.Problem(q).clique_list()]
        vo += q.n
    assert sorted(P.clique_list()) == sorted(shifted)


def test_components_joined_by_a_constraint(lib):
    """A constraint whose entries touch two summands merges them (the pattern
    alone would not): A D^-1 A^T then couples their constraints."""
    import dataclasses
    a, b = W.block_arrow(2, 3, 2, 4, seed=31), W.block_arrow(2, 4, 1, 5, seed=32)
    s = W.direct_sum([a, b, W.lovasz_theta_cycle(5)])
    # constraint 0 gets one more (diagonal) entry in the second summand
    s = dataclasses.replace(s, A_con=np.append(s.A_con, 0).astype(np.int32),
                            A_row=np.append(s.A_row, a.n).astype(np.int32),
                            A_col=np.append(s.A_col, a.n).astype(np.int32), A_val=np.append(s.A_val, 1.0))
    P = lib.Problem(s)
    assert P.info["ncomp"] == 2
    vc, rc = P.components()
    assert set(vc[:a.n + b.n].tolist()) == {0} and set(vc[a.n + b.n:].tolist()) == {1}
    assert set(rc[:a.m + b.m].tolist()) == {0} and set(rc[a.m + b.m:].tolist()) == {1}


def test_components_interleaved_numbering(lib):
    """Components are found from the structure, not from index ranges: with
    the vertices of two summands interleaved and the constraints shuffled,
    each vertex and constraint still lands in its summand's component."""
    import dataclasses
    a, b = W.banded(10, 2, 4, seed=41, density=0.5), W.block_arrow(2, 3, 2, 5, seed=42)
    s = W.direct_sum([a, b])
    rng = np.random.default_rng(0)
    vperm = rng.permutation(s.n).astype(np.int32)  # new label of each vertex
    cperm = rng.permutation(s.m).astype(np.int32)

    def relabel(r, c):
        r2, c2 = vperm[r], vperm[c]
        return np.maximum(r2, c2).astype(np.int32), np.minimum(r2, c2).astype(np.int32)

    Ar, Ac = relabel(s.A_row, s.A_col)
    Cr, Cc = relabel(s.C_row, s.C_col)
    b_new = np.empty_like(s.b)
    b_new[cperm] = s.b
    t = dataclasses.replace(s, A_row=Ar, A_col=Ac, C_row=Cr, C_col=Cc, A_con=cperm[s.A_con], b=b_new)
    P = _compare(t)
    assert P.info["ncomp"] == 2
    vc, rc = P.components()
    owner = np.repeat([0, 1], [a.n, b.n])
    first = owner[np.argmin(vperm)]  # the summand holding new vertex 0 is component 0
    want_v = np.empty(s.n, np.int64)
    want_v[vperm] = (owner != first).astype(np.int64)
    np.testing.assert_array_equal(vc, want_v)
    cowner = np.repeat([0, 1], [a.m, b.m])
    want_c = np.empty(s.m, np.int64)
    want_c[cperm] = (cowner != first).astype(np.int64)
    np.testing.assert_array_equal(rc, want_c)
