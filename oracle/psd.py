"""Oracle: symmetric eigendecomposition by cyclic Jacobi and the PSD projection.

Test infrastructure only (see oracle/__init__.py).

The projection onto the PSD cone in the Frobenius norm is
    P(W) = V max(Lambda, 0) V^T,  W = V Lambda V^T
(Section 4.1.2, Eq. XkUpdate; the paper calls an eigensolver for it).  The
eigensolver here is the classical cyclic-by-row Jacobi method (Jacobi 1846;
Golub and Van Loan, Matrix Computations, Section 8.5: the 2x2 symmetric
Schur step, then J^T A J on rows/columns p and q), with a threshold: a
rotation is skipped when |a_pq| <= 1e-16 ||W||_F, and sweeps stop when a
whole sweep skips every rotation.  All arithmetic is float64.

Matrices of the same size are processed together along a leading batch axis;
each matrix undergoes exactly the rotations it would undergo alone.
"""
from __future__ import annotations

import numpy as np

MAX_SWEEPS = 60


def jacobi_eigh(W):
    """Eigenvalues (unsorted) and eigenvectors (columns) of a batch of
    symmetric matrices W[..., s, s], float64."""
    A = np.array(W, dtype=np.float64, copy=True)
    batch_shape = A.shape[:-2]
    s = A.shape[-1]
    A = A.reshape(-1, s, s)
    nb = A.shape[0]
    V = np.broadcast_to(np.eye(s), (nb, s, s)).copy()
    if s == 1 or nb == 0:
        return np.diagonal(A, axis1=1, axis2=2).reshape(batch_shape + (s,)), V.reshape(batch_shape + (s, s))
    tol = 1e-16 * np.sqrt(np.sum(A * A, axis=(1, 2)))
    for sweep in range(MAX_SWEEPS):
        rotated = False
        for p in range(s - 1):
            for q in range(p + 1, s):
                apq = A[:, p, q]
                active = np.abs(apq) > tol
                if not active.any():
                    continue
                rotated = True
                app = A[:, p, p]
                aqq = A[:, q, q]
                safe = np.where(active, apq, 1.0)
                tau = (aqq - app) / (2.0 * safe)
                t = np.where(tau >= 0, 1.0, -1.0) / (np.abs(tau) + np.sqrt(1.0 + tau * tau))
                t = np.where(active, t, 0.0)
                c = 1.0 / np.sqrt(1.0 + t * t)
                sn = t * c
                new_pp = app - t * apq
                new_qq = aqq + t * apq
                # rows p, q:  J^T A
                rp = A[:, p, :].copy()
                rq = A[:, q, :].copy()
                A[:, p, :] = c[:, None] * rp - sn[:, None] * rq
                A[:, q, :] = sn[:, None] * rp + c[:, None] * rq
                # columns p, q:  (J^T A) J
                cp = A[:, :, p].copy()
                cq = A[:, :, q].copy()
                A[:, :, p] = c[:, None] * cp - sn[:, None] * cq
                A[:, :, q] = sn[:, None] * cp + c[:, None] * cq
                # the 2x2 block is set by the Schur step exactly
                A[:, p, p] = np.where(active, new_pp, A[:, p, p])
                A[:, q, q] = np.where(active, new_qq, A[:, q, q])
                A[:, p, q] = np.where(active, 0.0, A[:, p, q])
                A[:, q, p] = np.where(active, 0.0, A[:, q, p])
                vp = V[:, :, p].copy()
                vq = V[:, :, q].copy()
                V[:, :, p] = c[:, None] * vp - sn[:, None] * vq
                V[:, :, q] = sn[:, None] * vp + c[:, None] * vq
        if not rotated:
            break
    else:
        raise RuntimeError("Jacobi did not converge")
    lam = np.diagonal(A, axis1=1, axis2=2).copy()
    return lam.reshape(batch_shape + (s,)), V.reshape(batch_shape + (s, s))


def psd_project(W, eig="jacobi"):
    """P(W) = V diag(max(lambda, 0)) V^T for a batch of symmetric matrices.

    eig="jacobi" (the default) takes the eigendecomposition from jacobi_eigh
    above; eig="lapack" takes it from LAPACK's symmetric eigensolver through
    numpy.linalg.eigh, a library primitive serving as that one step, for the
    problems whose cliques (orders in the hundreds, many sizes) put the
    pure-Python Jacobi out of reach (seconds per block).  Both give P(W) to
    rounding; tests/test_oracle_psd.py holds them equal."""
    if eig == "lapack":
        lam, V = np.linalg.eigh(np.asarray(W, dtype=np.float64))
    else:
        lam, V = jacobi_eigh(W)
    lp = np.maximum(lam, 0.0)
    return np.einsum("...ik,...k,...jk->...ij", V, lp, V)


def psd_project_with_eig(W):
    lam, V = jacobi_eigh(W)
    lp = np.maximum(lam, 0.0)
    return np.einsum("...ik,...k,...jk->...ij", V, lp, V), lam, V


def daleckii_krein_vjp(lam, V, G):
    """Adjoint of W -> P(W) at W = V diag(lam) V^T applied to a symmetric
    upstream gradient G: V (Gamma o (V^T G V)) V^T with the divided
    differences Gamma_ij = (f(l_i) - f(l_j)) / (l_i - l_j), f = max(., 0),
    and Gamma_ij = f'(l_i) (1, 0, or 1/2 at 0) when l_i == l_j
    (Daleckii-Krein; Bhatia, Matrix Analysis, Thm V.3.3).  Not in the paper."""
    li = lam[..., :, None]
    lj = lam[..., None, :]
    fi = np.maximum(li, 0.0)
    fj = np.maximum(lj, 0.0)
    diff = li - lj
    same = diff == 0
    deriv = np.where(li > 0, 1.0, np.where(li < 0, 0.0, 0.5))
    gam = np.where(same, deriv, (fi - fj) / np.where(same, 1.0, diff))
    inner = np.einsum("...ki,...kl,...lj->...ij", V, G, V)
    return np.einsum("...ik,...kl,...jl->...ij", V, gam * inner, V)
