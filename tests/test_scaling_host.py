"""Data scaling of Section 7.1.3 in the library's host setup: the factors
cdsdp_setup_scaled computes equal the oracle's, the scaled handle keeps the
pattern and cliques of the unscaled one, and bad arguments are rejected.
Host only: no GPU call."""
import numpy as np
import pytest

from oracle import scaling
from paper_1707_05058_gb300 import workloads as W

CASES = [W.workload(0), W.block_arrow(3, 4, 2, 6, seed=5), W.maxcut_cycle(7),
         W.lambda_max_tridiagonal(8, 1.0, 0.5), W.direct_sum([W.block_arrow(2, 3, 2, 4, seed=1),
                                                              W.maxcut_cycle(5)])]


@pytest.mark.parametrize("passes", [0, 1, 5])
@pytest.mark.parametrize("prob", CASES, ids=lambda p: p.name)
def test_scaling_factors_match_oracle(lib, prob, passes):
    P = lib.Problem(prob, scale_passes=passes)
    d, e, tau, sigma = P.scaling()
    rd, re, rtau, rsigma = scaling.scaling_factors(prob, passes)
    np.testing.assert_allclose(d, rd, rtol=1e-14)
    np.testing.assert_allclose(e, re, rtol=1e-14)
    assert abs(tau - rtau) <= 1e-13 * rtau
    assert abs(sigma - rsigma) <= 1e-13 * rsigma


@pytest.mark.parametrize("passes", [0, 4])
def test_batch_scaling_factors_per_sdp(lib, passes):
    """A scaled batch (cdsdp_setup_batch) scales every SDP as if alone: d and e
    of the sum and tau_j, sigma_j of each SDP equal the oracle's factors of that
    SDP scaled on its own."""
    parts = [W.block_arrow(2, 3, 2, 4, seed=1), W.maxcut_cycle(5), W.block_arrow(3, 4, 2, 6, seed=5),
             W.lambda_max_tridiagonal(8, 1.0, 0.5)]
    P = lib.Problem.batch(parts, scale_passes=passes)
    d, e, tau0, sigma0 = P.scaling()
    tau, sigma = P.scaling_batch()
    assert len(tau) == len(sigma) == len(parts)
    assert tau0 == tau[0] and sigma0 == sigma[0]
    vo = np.concatenate([[0], np.cumsum([q.n for q in parts])])
    mo = np.concatenate([[0], np.cumsum([q.m for q in parts])])
    for j, q in enumerate(parts):
        rd, re, rtau, rsigma = scaling.scaling_factors(q, passes)
        np.testing.assert_allclose(d[vo[j]:vo[j + 1]], rd, rtol=1e-14)
        np.testing.assert_allclose(e[mo[j]:mo[j + 1]], re, rtol=1e-14)
        assert abs(tau[j] - rtau) <= 1e-13 * rtau and abs(sigma[j] - rsigma) <= 1e-13 * rsigma
    t1, s1 = lib.Problem(parts[0], scale_passes=passes).scaling_batch()
    assert len(t1) == 1
    tu, su = lib.Problem.batch(parts).scaling_batch()
    assert len(tu) == 1 and tu[0] == 1.0 and su[0] == 1.0


def test_unscaled_handle_reports_unit_factors(lib):
    prob = W.workload(0)
    d, e, tau, sigma = lib.Problem(prob).scaling()
    assert np.all(d == 1.0) and np.all(e == 1.0) and tau == 1.0 and sigma == 1.0


@pytest.mark.parametrize("prob", CASES[:3], ids=lambda p: p.name)
def test_scaled_setup_keeps_pattern_and_cliques(lib, prob):
    P0 = lib.Problem(prob)
    P1 = lib.Problem(prob, scale_passes=4)
    for k in ("n", "m", "p", "max_clique", "nnz_pattern", "n_d_lower", "nnz_A", "n_fill", "ncomp"):
        assert P0.info[k] == P1.info[k], k
    assert P0.clique_list() == P1.clique_list()
    for a, b in zip(P0.pattern(), P1.pattern()):
        np.testing.assert_array_equal(a, b)


def test_scaled_setup_rejects_bad_arguments(lib):
    prob = W.workload(0)
    with pytest.raises(lib.CdsdpError) as ex:
        lib.Problem(prob, scale_passes=-1)
    assert ex.value.status == -1  # CDSDP_ERR_ARG
    import dataclasses
    bad = dataclasses.replace(prob, A_row=prob.A_row.copy())
    bad.A_row[3] = prob.n  # out of range
    with pytest.raises(lib.CdsdpError) as ex:
        lib.Problem(bad, scale_passes=2)
    assert ex.value.status == -1  # CDSDP_ERR_ARG


def test_setup_without_the_cached_factor(lib):
    """CDSDP_SETUP_NO_FACTOR: same structure, no inverse blocks in the
    workspace (about 2 x 8 m^2 bytes fewer for a one-component problem), and a
    component above 8192 constraints, refused with the factor, is accepted."""
    prob = W.workload(0)
    P1 = lib.Problem(prob)
    P0 = lib.Problem(prob, cache_factor=False)
    assert P1.info["cached_factor"] == 1 and P0.info["cached_factor"] == 0
    for k in ("n", "m", "p", "nnz_pattern", "nnz_A", "ncomp"):
        assert P0.info[k] == P1.info[k]
    m = prob.m
    assert P1.workspace_bytes(10) - P0.workspace_bytes(10) >= 2 * (8 * m * m - 256)  # sections 256-byte aligned
    big = W.banded(9000, 2, 9000, seed=12, density=0.01)
    with pytest.raises(lib.CdsdpError) as ex:
        lib.Problem(big)
    assert ex.value.status == -8  # CDSDP_ERR_UNSUPPORTED: dense block above 8192
    Pb = lib.Problem(big, cache_factor=False)
    assert Pb.info["m"] == 9000 and Pb.info["ncomp"] == 1 and Pb.info["cached_factor"] == 0


def test_unknown_setup_flag_is_rejected(lib):
    import ctypes
    prob = W.workload(0)
    arrs = prob.arrays()
    ptr = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t)) if a.size else None
    A_con, A_row, A_col, A_val, b, C_row, C_col, C_val, P_row, P_col = arrs
    h = ctypes.c_void_p()
    st = lib._lib.cdsdp_setup_flags(prob.n, prob.m, A_con.size, ptr(A_con, ctypes.c_int), ptr(A_row, ctypes.c_int),
                                    ptr(A_col, ctypes.c_int), ptr(A_val, ctypes.c_double), ptr(b, ctypes.c_double),
                                    C_row.size, ptr(C_row, ctypes.c_int), ptr(C_col, ctypes.c_int),
                                    ptr(C_val, ctypes.c_double), 0, None, None, -1, 6, ctypes.byref(h))
    assert st == -1 and not h.value
