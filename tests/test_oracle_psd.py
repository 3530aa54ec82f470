"""Pins for the oracle's Jacobi eigensolver and PSD projection (CPU only)."""
import numpy as np
import pytest

from oracle import psd
from paper_1707_05058_gb300 import workloads as W


@pytest.mark.parametrize("s", [1, 2, 3, 5, 11, 15, 32, 40])
def test_jacobi_matches_lapack(s):
    Wb = W.random_symmetric_batch(6, s, seed=s)
    lam, V = psd.jacobi_eigh(Wb)
    ref = np.linalg.eigh(Wb)[0]
    scale = np.abs(ref).max()
    np.testing.assert_allclose(np.sort(lam, axis=-1), ref, atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(np.einsum("bki,bkj->bij", V, V), np.broadcast_to(np.eye(s), V.shape), atol=1e-13)
    rebuilt = np.einsum("bik,bk,bjk->bij", V, lam, V)
    np.testing.assert_allclose(rebuilt, Wb, atol=1e-12 * scale)


def test_jacobi_repeated_and_zero_eigenvalues():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([2.0, 2.0, 0.0, 0.0, -1.0, -1.0])
    Wm = (Q * lam) @ Q.T
    got = psd.psd_project(Wm[None])[0]
    want = (Q * np.maximum(lam, 0)) @ Q.T
    np.testing.assert_allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("s", [3, 11, 24])
def test_projection_invariants(s):
    """P(P(W)) = P(W); P(W) PSD; <W - P(W), P(W)> = 0; W - P(W) NSD;
    nonexpansive; W = P(W) - P(-W) (Moreau)."""
    Wb = W.random_symmetric_batch(8, s, seed=100 + s)
    Vb = W.random_symmetric_batch(8, s, seed=200 + s)
    P = psd.psd_project(Wb)
    np.testing.assert_allclose(psd.psd_project(P), P, atol=1e-12)
    assert np.linalg.eigvalsh(P).min() > -1e-12
    assert np.abs(np.einsum("bij,bij->b", Wb - P, P)).max() < 1e-11
    assert np.linalg.eigvalsh(Wb - P).max() < 1e-12
    PV = psd.psd_project(Vb)
    lhs = np.linalg.norm(P - PV, axis=(1, 2))
    rhs = np.linalg.norm(Wb - Vb, axis=(1, 2))
    assert np.all(lhs <= rhs + 1e-12)
    np.testing.assert_allclose(P - psd.psd_project(-Wb), Wb, atol=1e-12)


def test_projection_special_cases():
    d = np.diag([3.0, -2.0, 0.0, 1.5])
    np.testing.assert_array_equal(psd.psd_project(d[None])[0], np.diag([3.0, 0.0, 0.0, 1.5]))
    G = np.random.default_rng(1).standard_normal((5, 5))
    S = G @ G.T
    np.testing.assert_allclose(psd.psd_project(S[None])[0], S, atol=1e-12)
    np.testing.assert_allclose(psd.psd_project(-S[None])[0], 0.0, atol=1e-12)
    np.testing.assert_array_equal(psd.psd_project(np.zeros((1, 4, 4))), np.zeros((1, 4, 4)))


@pytest.mark.parametrize("s", [2, 5, 9])
def test_daleckii_krein_matches_finite_differences(s):
    Wm = W.random_symmetric_batch(1, s, seed=7 + s)[0]
    G = W.random_symmetric_batch(1, s, seed=70 + s)[0]
    lam, V = psd.jacobi_eigh(Wm)
    g = psd.daleckii_krein_vjp(lam, V, G)
    rng = np.random.default_rng(s)
    for _ in range(3):
        dW = rng.standard_normal((s, s)); dW = dW + dW.T
        h = 1e-6
        fd = (np.sum(G * psd.psd_project((Wm + h * dW)[None])[0]) -
              np.sum(G * psd.psd_project((Wm - h * dW)[None])[0])) / (2 * h)
        np.testing.assert_allclose(np.sum(g * dW), fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("s", [1, 2, 5, 17, 40])
def test_lapack_step_equals_jacobi(s):
    """The oracle's two eigendecomposition steps give the same projection
    (the LAPACK step serves the problems with cliques of order in the
    hundreds)."""
    rng = np.random.default_rng(s)
    G = rng.standard_normal((3, s, s))
    W = G + np.swapaxes(G, 1, 2)
    Pj = psd.psd_project(W)
    Pl = psd.psd_project(W, eig="lapack")
    assert np.abs(Pj - Pl).max() <= 1e-12 * max(1.0, np.abs(W).max())
