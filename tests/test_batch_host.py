"""cdsdp_setup_batch (host only): a batch of SDPs with local indices sets up
exactly as their direct sum, every summand keeps its own pattern, and a local
index outside its problem is rejected.  No GPU call."""
import dataclasses

import numpy as np
import pytest

from paper_1707_05058_gb300 import workloads as W

PARTS = [W.banded(50, 3, 10, seed=1), W.workload(0), W.maxcut_cycle(7), W.block_arrow(2, 6, 3, 5, seed=4)]


def test_batch_equals_direct_sum(lib):
    B = lib.Problem.batch(PARTS)
    S = lib.Problem(W.direct_sum(PARTS))
    assert B.info == S.info
    assert B.clique_list() == S.clique_list()
    for a, b in zip(B.pattern(), S.pattern()):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(B.components(), S.components()):
        np.testing.assert_array_equal(a, b)
    assert B.info["ncomp"] >= len(PARTS)


def test_split_gives_each_problems_own_pattern(lib):
    B = lib.Problem.batch(PARTS)
    nz = int(B.info["nnz_pattern"])
    fake = {"X": np.arange(nz, dtype=float), "Z": -np.arange(nz, dtype=float), "y": np.arange(B.info["m"], dtype=float)}
    parts = B.split(fake)
    assert len(parts) == len(PARTS)
    off = 0
    for prob, part in zip(PARTS, parts):
        r, c = lib.Problem(prob).pattern()
        np.testing.assert_array_equal(part["rows"], r)
        np.testing.assert_array_equal(part["cols"], c)
        np.testing.assert_array_equal(part["X"], np.arange(off, off + r.size, dtype=float))
        off += r.size
        assert part["y"].size == prob.m
    assert off == nz


def test_batch_rejects_a_local_index_out_of_range(lib):
    bad = dataclasses.replace(PARTS[2], C_row=PARTS[2].C_row.copy())
    bad.C_row[-1] = bad.n  # valid in the sum, not in its own problem
    with pytest.raises(lib.CdsdpError) as ex:
        lib.Problem.batch([PARTS[0], bad])
    assert ex.value.status == -1  # CDSDP_ERR_ARG


def test_split_components_partitions_the_solution(lib):
    P = lib.Problem(W.direct_sum(PARTS))
    nz, m = int(P.info["nnz_pattern"]), int(P.info["m"])
    fake = {"X": np.arange(nz, dtype=float), "Z": None, "y": np.arange(m, dtype=float)}
    parts = P.split_components(fake)
    assert len(parts) == P.info["ncomp"]
    ents = np.sort(np.concatenate([p["entries"] for p in parts]))
    cons = np.sort(np.concatenate([p["constraints"] for p in parts]))
    np.testing.assert_array_equal(ents, np.arange(nz))
    np.testing.assert_array_equal(cons, np.arange(m))
    for p in parts:
        np.testing.assert_array_equal(p["X"], p["entries"].astype(float))
        assert p["Z"] is None
