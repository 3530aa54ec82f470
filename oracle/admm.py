"""Oracle: decomposed ADMM for sparse SDPs, Algorithms 1, 2 and 3, in float64.

Test infrastructure only (see oracle/__init__.py).  Plain and slow on purpose:
each step is written as the paper states it, in the paper's vectorised form.

Storage follows Section 4 literally: vec() stacks columns, and x = vec(X) is
kept on every entry (i, j) of the extended pattern E* in BOTH triangles (the
entries outside E* have c = A = D = 0 and decouple).  The clique vectors
x_k = H_k x are full |C_k|^2 column-major vectors.  H_k is never formed as a
matrix: H_k x is the index gather x[idx_k] and H_k^T y the scatter-add.

Readings where the paper is silent (each is also stated where it is used):
  * initial guesses are zero; HSDE starts from u = (0,..,0, tau=1),
    v = (0,..,0, kappa=1) as in O'Donoghue et al. (the paper defers to them);
  * eps_lambda divides by max(||lambda||, 1e-300) and no stop at n = 1;
  * dual multiplier update uses the generic rule lambda += rho (z - v)
    (Eq. MultUpdateDualSDP), which with Eq. vkEqn equals -rho H_k x;
  * recovered variables: Alg. 1 gives X = x, y = -rho y_kkt, Z = sum H_k^T
    lambda_k; Alg. 2 gives X = -rho x, y, Z = sum H_k^T z_k;
  * HSDE: optimality is tested when tau > 0, infeasibility otherwise, each
    certificate on its own (b^T u_y > 0 and ||A^T u_y + H^T v_z|| <= eps b^T u_y / ||b||
    for primal infeasibility; c^T u_x < 0 and ||A u_x|| <= -eps c^T u_x / ||c||
    for dual infeasibility); no over-relaxation.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg
import scipy.sparse

from . import chordal
from .psd import psd_project

SOLVED, MAX_ITER, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 0, 1, 2, 3


@dataclasses.dataclass
class Decomposed:
    n: int
    m: int
    cliques: list            # sorted vertex tuples, lexicographic order
    lower: list              # extended pattern, lower (i >= j), column-major order
    full_index: dict         # (i, j) -> position in the full vec over E*
    N: int                   # number of full-vec entries (both triangles)
    c: np.ndarray            # [N]
    A: scipy.sparse.csr_matrix  # [m, N]
    b: np.ndarray            # [m]
    clique_idx: list         # per clique: positions of vec(E_k X E_k^T) in x
    hidx: np.ndarray         # concatenation of clique_idx (stacked H)
    offsets: np.ndarray      # clique k occupies hidx[offsets[k]:offsets[k+1]]
    D: np.ndarray            # diag(sum_k H_k^T H_k), [N]
    nfill: int
    chordal: bool
    eig: str = "jacobi"      # eigendecomposition step of the projection (oracle/psd.py)

    @property
    def nd(self):
        return int(self.hidx.size)

    def H(self, x):
        return x[self.hidx]

    def HT(self, s):
        return np.bincount(self.hidx, weights=s, minlength=self.N)

    def lower_values(self, x):
        """Values of a full-vec vector on the lower pattern entries."""
        return np.array([x[self.full_index[e]] for e in self.lower])

    def project_cliques(self, w):
        """Apply the PSD projection to every clique block of a stacked vector."""
        out = np.empty_like(w)
        by_size = {}
        for k, cl in enumerate(self.cliques):
            by_size.setdefault(len(cl), []).append(k)
        for s, ks in by_size.items():
            blocks = np.stack([w[self.offsets[k]:self.offsets[k + 1]].reshape(s, s, order="F") for k in ks])
            proj = psd_project(blocks, self.eig)
            for j, k in enumerate(ks):
                out[self.offsets[k]:self.offsets[k + 1]] = proj[j].reshape(-1, order="F")
        return out


def decompose(prob, merge=False, eig="jacobi") -> Decomposed:
    """Data preprocessing of Algorithms 1-3: aggregate pattern, chordal
    extension and maximal cliques (Section 2.1), selectors H_k (Section 4) and
    D = sum_k H_k^T H_k."""
    n, m = prob.n, prob.m
    cliques, lower, nfill, is_chordal = chordal.chordal_decomposition(
        n, [(prob.C_row, prob.C_col), (prob.A_row, prob.A_col), (prob.P_row, prob.P_col)], merge=merge)
    full = []
    for (i, j) in lower:
        full.append((i, j))
        if i != j:
            full.append((j, i))
    full.sort(key=lambda t: (t[1], t[0]))     # vec(): stack columns
    full_index = {e: k for k, e in enumerate(full)}
    N = len(full)
    c = np.zeros(N)
    for r, cc, v in zip(prob.C_row, prob.C_col, prob.C_val):
        c[full_index[(int(r), int(cc))]] += v
        if r != cc:
            c[full_index[(int(cc), int(r))]] += v
    rows, cols, vals = [], [], []
    for k, r, cc, v in zip(prob.A_con, prob.A_row, prob.A_col, prob.A_val):
        rows.append(int(k)); cols.append(full_index[(int(r), int(cc))]); vals.append(v)
        if r != cc:
            rows.append(int(k)); cols.append(full_index[(int(cc), int(r))]); vals.append(v)
    A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(m, N))
    A.sum_duplicates()
    clique_idx = []
    for cl in cliques:
        idx = [full_index[(cl[a], cl[bb])] for bb in range(len(cl)) for a in range(len(cl))]
        clique_idx.append(np.array(idx, dtype=np.int64))
    hidx = np.concatenate(clique_idx) if clique_idx else np.zeros(0, np.int64)
    offsets = np.concatenate([[0], np.cumsum([len(ix) for ix in clique_idx])]).astype(np.int64)
    D = np.bincount(hidx, minlength=N).astype(np.float64)
    return Decomposed(n, m, cliques, lower, full_index, N, c, A, np.asarray(prob.b, np.float64),
                      clique_idx, hidx, offsets, D, nfill, is_chordal, eig)


def _cholesky(M):
    return scipy.linalg.cho_factor(M, lower=True)


def _norm(v):
    return float(np.sqrt(np.dot(v, v)))


@dataclasses.dataclass
class Result:
    status: int
    iters: int
    X: np.ndarray        # full vec over E*
    y: np.ndarray
    Z: np.ndarray        # full vec over E*
    hist: np.ndarray     # [iters, 8]
    cert: np.ndarray | None = None
    state: dict | None = None


def adapt_rho(rho, eps_p, eps_d, mu, nu):
    """Adaptive penalty rule of Section 7.1.2: multiply rho by mu when the
    primal residual is at least nu times the dual one, divide by mu in the
    opposite case, keep it otherwise.  For Algorithms 1-2 the residual pair
    is (eps_c, eps_lambda) of their stopping tests."""
    if eps_p >= nu * eps_d:
        return rho * mu
    if eps_d >= nu * eps_p:
        return rho / mu
    return rho


def conjugate_gradient(matvec, r, y0, tol, max_iter):
    """Conjugate gradient method (Hestenes and Stiefel 1952; the textbook form
    in Saad 2003, Section 6.7) for S y = r with S symmetric positive definite
    given as a product v -> S v.  Starts from y0 and stops once
    ||r - S y|| <= tol ||r|| or after max_iter steps.  Returns (y, steps)."""
    y = np.array(y0, dtype=float)
    res = r - matvec(y)
    p = res.copy()
    rr = float(res @ res)
    target = tol * float(np.linalg.norm(r))
    k = 0
    while k < max_iter and np.sqrt(rr) > target:
        q = matvec(p)
        alpha = rr / float(p @ q)
        y = y + alpha * p
        res = res - alpha * q
        rr_new = float(res @ res)
        p = res + (rr_new / rr) * p
        rr = rr_new
        k += 1
    return y, k


def _kkt_solver(A, AT, D, linear_solver):
    """Solver of (A D^-1 A^T) y = r, the only system of Eqs. OptCondMinYPrimal
    and OptCondMinYDual after eliminating x (Section 4.1.1).  linear_solver
    None: the cached Cholesky factor (Eq. ADMMprimalFatorization).  ("cg", tol,
    max_iter): the conjugate gradient method the same section names for when
    the factorisation is too expensive, warm-started from the previous
    iteration's y.  Returns solve(r, y_prev) -> (y, cg_steps)."""
    if linear_solver is None:
        fac = _cholesky((A @ scipy.sparse.diags(1.0 / D) @ A.T).toarray())
        return lambda r, y_prev: (scipy.linalg.cho_solve(fac, r), 0)
    kind, tol, max_steps = linear_solver
    if kind != "cg":
        raise ValueError(f"unknown linear solver {kind!r}")

    def matvec(v):
        return A @ ((AT @ v) / D)
    return lambda r, y_prev: conjugate_gradient(matvec, r, y_prev, tol, max_steps)


def primal_admm(dp: Decomposed, rho=1.0, eps=1e-4, max_iter=2000, callback=None, adapt_every=0, mu=2.0, nu=10.0,
                linear_solver=None):
    """Algorithm 1 (ADMM for the domain-space decomposition).
    x-step: KKT system Eq. OptCondMinYPrimal by block elimination with the
    cached Cholesky factor of A D^-1 A^T (Eq. ADMMprimalFatorization, and
    Appendix A: L L^T y = A D^-1 bhat - b, x = D^-1 (bhat - A^T y));
    x_k-step: Eq. XkUpdate; multipliers: Eq. LambdakUpdate; stopping:
    Eq. PrimalConsensusResidual and eps_lambda (Section 4.1.4).
    adapt_every = N > 0 applies the adaptive penalty rule (Section 7.1.2,
    `adapt_rho`) after every N-th iteration whose stopping test failed; the
    multipliers are unscaled, so nothing else changes with rho.  History
    column 2 holds the rho of each iteration.  linear_solver: see
    `_kkt_solver` (None: cached Cholesky factor; ("cg", tol, steps): conjugate
    gradient, steps per iteration kept in state["cg_steps"])."""
    A, b, c, D = dp.A, dp.b, dp.c, dp.D
    AT = A.T.tocsr()
    kkt = _kkt_solver(A, AT, D, linear_solver)
    xk = np.zeros(dp.nd)
    lam = np.zeros(dp.nd)
    y = np.zeros(dp.m)
    cg_steps = []
    hist = []
    status = MAX_ITER
    for it in range(1, max_iter + 1):
        bhat = dp.HT(xk + lam / rho) - c / rho
        y, steps = kkt(A @ (bhat / D) - b, y)
        cg_steps.append(steps)
        x = (bhat - AT @ y) / D
        Hx = dp.H(x)
        xk_new = dp.project_cliques(Hx - lam / rho)
        lam = lam + rho * (xk_new - Hx)
        eps_c = _norm(xk_new - Hx) / max(_norm(xk_new), _norm(Hx), 1e-300)
        eps_l = rho * _norm(xk_new - xk) / max(_norm(lam), 1e-300)
        xk = xk_new
        hist.append([eps_c, eps_l, rho, 0.0, float(c @ x), float(-rho * (b @ y)), 0.0, 0.0])
        if callback is not None:
            callback(it, dict(x=x, y=y, xk=xk, lam=lam))
        rho_it = rho  # the penalty this iteration ran with
        if it > 1 and max(eps_c, eps_l) <= eps:
            status = SOLVED
            break
        if adapt_every > 0 and it % adapt_every == 0:
            rho = adapt_rho(rho, eps_c, eps_l, mu, nu)
    return Result(status, it, x, -rho_it * y, dp.HT(lam), np.array(hist),
                  state=dict(x=x, y_kkt=y, xk=xk, lam=lam, rho=rho_it, cg_steps=cg_steps))


def dual_admm(dp: Decomposed, rho=1.0, eps=1e-4, max_iter=2000, callback=None, adapt_every=0, mu=2.0, nu=10.0,
              linear_solver=None):
    """Algorithm 2 (ADMM for the range-space decomposition).
    z-step Eq. zkUpdate; (y, x) from the KKT system Eq. OptCondMinYDual with the
    same cached factor of A D^-1 A^T; v_k from Eq. vkEqn; lambda_k from the
    generic rule Eq. MultUpdateDualSDP; stopping Section 4.2.4.  Adaptive
    penalty, history column 2 and linear_solver as in `primal_admm`."""
    A, b, c, D = dp.A, dp.b, dp.c, dp.D
    AT = A.T.tocsr()
    kkt = _kkt_solver(A, AT, D, linear_solver)
    z = np.zeros(dp.nd)
    v = np.zeros(dp.nd)
    lam = np.zeros(dp.nd)
    y = np.zeros(dp.m)
    cg_steps = []
    hist = []
    status = MAX_ITER
    for it in range(1, max_iter + 1):
        z_new = dp.project_cliques(v - lam / rho)
        rhs1 = c - dp.HT(z_new + lam / rho)
        rhs2 = -b / rho
        y, steps = kkt(A @ (rhs1 / D) - rhs2, y)
        cg_steps.append(steps)
        x = (rhs1 - AT @ y) / D
        Hx = dp.H(x)
        v = z_new + lam / rho + Hx
        lam = lam + rho * (z_new - v)
        eps_c = _norm(z_new - v) / max(_norm(z_new), _norm(v), 1e-300)
        eps_l = rho * _norm(z_new - z) / max(_norm(lam), 1e-300)
        z = z_new
        hist.append([eps_c, eps_l, rho, 0.0, float(-rho * (c @ x)), float(b @ y), 0.0, 0.0])
        if callback is not None:
            callback(it, dict(x=x, y=y, z=z, v=v, lam=lam))
        rho_it = rho  # the penalty this iteration ran with
        if it > 1 and max(eps_c, eps_l) <= eps:
            status = SOLVED
            break
        if adapt_every > 0 and it % adapt_every == 0:
            rho = adapt_rho(rho, eps_c, eps_l, mu, nu)
    return Result(status, it, -rho_it * x, y, dp.HT(z), np.array(hist),
                  state=dict(x=x, y=y, z=z, v=v, lam=lam, rho=rho_it, cg_steps=cg_steps))


class HSDEOperator:
    """Cached data of Section 5.2: P = I + D/2, the Cholesky factor of
    I + A P^-1 A^T (Eq. HSDEFactorizationFinal), zeta = (c_hat, -b_hat)
    (Eq. MDef) and zeta_hat = M^-1 zeta / (1 + zeta^T M^-1 zeta)
    (Proposition 2)."""

    def __init__(self, dp: Decomposed):
        self.dp = dp
        self.A = dp.A
        self.AT = dp.A.T.tocsr()
        self.P = 1.0 + 0.5 * dp.D
        K = np.eye(dp.m) + (self.A @ scipy.sparse.diags(1.0 / self.P) @ self.A.T).toarray()
        self.fac = _cholesky(K)
        N, nd, m = dp.N, dp.nd, dp.m
        self.sizes = (N, nd, m, nd)
        self.zeta = np.concatenate([dp.c, np.zeros(nd), -dp.b, np.zeros(nd)])
        Minv_zeta = self.solve_M(self.zeta)
        self.zeta_hat = Minv_zeta / (1.0 + self.zeta @ Minv_zeta)

    def split(self, w):
        N, nd, m, _ = self.sizes
        return w[:N], w[N:N + nd], w[N + nd:N + nd + m], w[N + nd + m:]

    def solve_M(self, nu):
        """Inner system Eq. SecondBlockElimination, M sigma = nu, by the block
        eliminations of Appendix B: eta, sigma_11 by the matrix inversion
        lemma (Eq. MatrixInvFlops), sigma_12 (Eq. ThirBlkFlops_s2), then
        sigma_21, sigma_22 (Eq. AppendixEqSigma2)."""
        dp = self.dp
        nu11, nu12, nu21, nu22 = self.split(nu)
        eta = nu11 + self.AT @ nu21 + 0.5 * dp.HT(nu12 + nu22)
        Pe = eta / self.P
        s11 = Pe - (self.AT @ scipy.linalg.cho_solve(self.fac, self.A @ Pe)) / self.P
        Hs = dp.H(s11)
        s12 = 0.5 * (nu12 - nu22 + Hs)
        s21 = nu21 - self.A @ s11
        s22 = nu22 - Hs + s12
        return np.concatenate([s11, s12, s21, s22])

    def solve_I_plus_Q(self, w):
        """Outer system Eq. LinearSystem: u_hat_1 by Eq. MatrixInverseResult,
        u_hat_2 by Eq. FirstBlockElimination."""
        w1, w2 = w[:-1], w[-1]
        sig = self.solve_M(w1 - w2 * self.zeta)
        u1 = sig - self.zeta_hat * (self.zeta @ sig)
        u2 = w2 + self.zeta @ u1
        return np.concatenate([u1, [u2]])


def hsde_admm(dp: Decomposed, eps=1e-4, max_iter=2000, callback=None):
    """Algorithm 3 (simplified ADMM for the HSDE, Eqs. HsdeStep1-3) with the
    stopping tests of Section 5.2.3 (Eqs. HSDEerror, HSDEconsensusResidual,
    Infeasibility)."""
    op = HSDEOperator(dp)
    A, AT, b, c = op.A, op.AT, dp.b, dp.c
    N, nd, m, _ = op.sizes
    L = N + 2 * nd + m + 1
    u = np.zeros(L); u[-1] = 1.0
    v = np.zeros(L); v[-1] = 1.0
    nb, nc = _norm(b), _norm(c)
    hist = []
    status = MAX_ITER
    cert = None
    for it in range(1, max_iter + 1):
        uh = op.solve_I_plus_Q(u + v)
        w = uh - v
        u_new = w.copy()                   # free cones: identity
        sl = slice(N, N + nd)
        u_new[sl] = dp.project_cliques(w[sl])
        u_new[-1] = max(0.0, w[-1])        # R_+
        v = v - uh + u_new
        u = u_new
        ux, us, uy, ut = u[:N], u[sl], u[N + nd:N + nd + m], u[N + nd + m:-1]
        vz = v[sl]
        tau, kappa = u[-1], v[-1]
        Hux = dp.H(ux)
        pc = _norm(us - Hux) / max(_norm(us), _norm(Hux), 1e-300)
        dc = _norm(vz - ut) / max(_norm(vz), _norm(ut), 1e-300)
        row = [0.0] * 8
        row[6], row[7] = tau, kappa
        if tau > 0:
            x = ux / tau
            y = uy / tau
            z = dp.HT(vz) / tau
            cx, by = float(c @ x), float(b @ y)
            ep = _norm(A @ x - b) / (1 + nb)
            ed = _norm(AT @ y + z - c) / (1 + nc)
            eg = abs(cx - by) / (1 + abs(cx) + abs(by))
            ec = max(pc, dc)
            row[:6] = [ep, ed, eg, ec, cx, by]
            hist.append(row)
            if callback is not None:
                callback(it, dict(u=u, v=v))
            if max(ep, ed, eg, ec) <= eps:
                status = SOLVED
                break
        else:
            bty = float(b @ uy)
            ctx = float(c @ ux)
            r_p = _norm(AT @ uy + dp.HT(vz))
            r_d = _norm(A @ ux)
            row[:4] = [r_p, r_d, bty, ctx]
            hist.append(row)
            if callback is not None:
                callback(it, dict(u=u, v=v))
            if bty > 0 and r_p <= eps * bty / max(nb, 1e-300):
                status = PRIMAL_INFEASIBLE
                cert = uy / bty
                break
            if ctx < 0 and r_d <= -eps * ctx / max(nc, 1e-300):
                status = DUAL_INFEASIBLE
                cert = -ux / ctx
                break
    tau = u[-1]
    scale = tau if tau > 0 else 1.0
    return Result(status, it, u[:N] / scale, u[N + nd:N + nd + m] / scale, dp.HT(v[N:N + nd]) / scale,
                  np.array(hist), cert, state=dict(u=u, v=v))


def solve(prob, form="primal", **kw):
    dp = decompose(prob)
    fn = {"primal": primal_admm, "dual": dual_admm, "hsde": hsde_admm}[form]
    return dp, fn(dp, **kw)


# ---------------------------------------------------------------------------
# Differentiation through unrolled Algorithm 1 (not in the paper; the
# projection's derivative is the Daleckii-Krein formula, oracle/psd.py).

def primal_unrolled(dp: Decomposed, c, b, iters, rho=1.0, keep=False):
    """`iters` iterations of Algorithm 1 from the zero start with data (c, b)
    in place of the problem's (full vec over E*, m).  Returns x after the last
    affine step; with keep=True also the projection inputs W_n of every
    iteration (for the adjoint)."""
    A, D = dp.A, dp.D
    AT = A.T.tocsr()
    fac = _cholesky((A @ scipy.sparse.diags(1.0 / D) @ A.T).toarray())
    xk = np.zeros(dp.nd)
    lam = np.zeros(dp.nd)
    Ws = []
    x = None
    for _ in range(iters):
        bhat = dp.HT(xk + lam / rho) - c / rho
        y = scipy.linalg.cho_solve(fac, A @ (bhat / D) - b)
        x = (bhat - AT @ y) / D
        Hx = dp.H(x)
        Wn = Hx - lam / rho
        if keep:
            Ws.append(Wn.copy())
        xk_new = dp.project_cliques(Wn)
        lam = lam + rho * (xk_new - Hx)
        xk = xk_new
    return (x, Ws) if keep else x


def _project_cliques_vjp(dp: Decomposed, Wn, gbar):
    """Adjoint of the stacked clique projection at W_n (Daleckii-Krein)."""
    from .psd import daleckii_krein_vjp, jacobi_eigh
    out = np.empty_like(gbar)
    for k, cl in enumerate(dp.cliques):
        s = len(cl)
        sl = slice(dp.offsets[k], dp.offsets[k + 1])
        lam, V = jacobi_eigh(Wn[sl].reshape(s, s, order="F"))
        out[sl] = daleckii_krein_vjp(lam, V, gbar[sl].reshape(s, s, order="F")).reshape(-1, order="F")
    return out


def primal_unrolled_vjp(dp: Decomposed, c, b, iters, xbar, rho=1.0):
    """Reverse-mode adjoint of primal_unrolled: given the upstream gradient
    xbar of the returned x, the gradients (cbar, bbar) with respect to c and b.
    Each step of Algorithm 1 is linear except the projection, so the reverse
    pass transposes the steps in reverse order (plain transposes in the full
    vec coordinates)."""
    A, D = dp.A, dp.D
    AT = A.T.tocsr()
    fac = _cholesky((A @ scipy.sparse.diags(1.0 / D) @ A.T).toarray())
    _, Ws = primal_unrolled(dp, c, b, iters, rho, keep=True)
    xk_bar = np.zeros(dp.nd)
    lam_bar = np.zeros(dp.nd)
    cbar = np.zeros(dp.N)
    bbar = np.zeros(dp.m)
    for n in range(iters - 1, -1, -1):
        # lambda' = lambda + rho (x_k' - Hx)
        xkp_bar = xk_bar + rho * lam_bar
        hx_bar = -rho * lam_bar
        lam_prev_bar = lam_bar.copy()
        # x_k' = P(W),  W = Hx - lambda / rho
        W_bar = _project_cliques_vjp(dp, Ws[n], xkp_bar)
        hx_bar = hx_bar + W_bar
        lam_prev_bar = lam_prev_bar - W_bar / rho
        # Hx = H x
        x_bar = dp.HT(hx_bar) + (xbar if n == iters - 1 else 0.0)
        # x = (bhat - A^T y) / D
        bhat_bar = x_bar / D
        y_bar = -(A @ (x_bar / D))
        # y = (A D^-1 A^T)^-1 (A D^-1 bhat - b)
        r_bar = scipy.linalg.cho_solve(fac, y_bar)
        bhat_bar = bhat_bar + (AT @ r_bar) / D
        bbar -= r_bar
        # bhat = H^T (x_k + lambda / rho) - c / rho
        g = dp.H(bhat_bar)
        xk_bar = g
        lam_bar = lam_prev_bar + g / rho
        cbar -= bhat_bar / rho
    return cbar, bbar
