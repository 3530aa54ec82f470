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
