// Kernels specific to Algorithm 2 (dual) and Algorithm 3 (HSDE) of
// arXiv 1707.05058, and the result-assembly kernels.
#pragma once

#include "affine.cuh"

namespace cdsdp_dev {

// Algorithm 2, after the KKT solve: v_k = z_k + lambda_k/rho + H_k x (Eq. vkEqn),
// lambda_k <- lambda_k + rho (z_k - v_k) (Eq. MultUpdateDualSDP), one warp per
// clique; per-block sums of |z_k - v_k|^2, |z_k|^2, |v_k|^2, |lambda_k|^2 in
// columns 0-3 of the partial table.
__device__ void finish_dual_block(const Dev& d, const FinishArgs& fa);

template <typename T>
__global__ void __launch_bounds__(128) k_vlam_dual(Dev d, FinishArgs fa) {
    if (stopped(d)) return;
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const T* z = reinterpret_cast<const T*>(d.ck0);
    T* v = reinterpret_cast<T*>(d.ck1);
    T* lam = reinterpret_cast<T*>(d.ck2);
    double acc[4] = {0, 0, 0, 0};
    for (int k = w0; k < d.p; k += nw) {
        if (frozen_clique(d, k)) continue;  // warp-uniform
        const double rho = rho_clique(d, k);
        const int off = d.pk_off[k], s = d.csize[k], npk = s * (s + 1) / 2;
        // v and lambda are formed in float64 (z + lambda/rho + x cancels) and
        // stored in T; the per-clique sums of the stopping test are in T
        T p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        double cx = 0;
        for (int f = lane; f < npk; f += 32) {
            const int ent = d.gmap[off + f];
            if (d.comp_mode && d.owner[off + f]) cx += d.wgt[ent] * d.c[ent] * d.x[ent];
            const T zt = z[off + f];
            const double zz = zt, ll = lam[off + f];
            const T vn = T(zz + ll / rho + d.x[ent]);
            const T ln = T(ll + rho * (zz - double(vn)));
            v[off + f] = vn;
            lam[off + f] = ln;
            const T wt = T(d.wgt[ent]);
            const T dv = zt - vn;
            p0 += wt * dv * dv;
            p1 += wt * zt * zt;
            p2 += wt * vn * vn;
            p3 += wt * ln * ln;
        }
        const double q[4] = {double(warp_sum(p0)), double(warp_sum(p1)), double(warp_sum(p2)), double(warp_sum(p3))};
        if (d.comp_mode) {  // per-clique row (column 6: <c, x> over the entries the clique owns)
            const double cxk = warp_sum(cx);
            if (lane == 0) {
                double* pr = d.part + (size_t)k * PART_COLS;
                for (int c = 0; c < 4; ++c) pr[c] = q[c];
                pr[6] = cxk;
            }
        } else {
            for (int c = 0; c < 4; ++c) acc[c] += q[c];
        }
    }
    if (d.comp_mode) return;
    const int cols[4] = {0, 1, 2, 3};
    block_partial_row<4>(acc, d.part, blockIdx.x, cols);
    if (fa.enabled && last_block_single_writer(d)) finish_dual_block(d, fa);
}

// Algorithm 2 stopping test (Eq. DualConsensusResidual, eps_lambda), run by
// every thread of the block that finishes the iteration.
__device__ void finish_dual_block(const Dev& d, const FinishArgs& fa) {
    __shared__ double sh[32 * 5];
    const int cols[5] = {0, 1, 2, 3, 5};
    double s[5];
    sum_cols<5>(d.part, fa.npart, cols, s, sh);
    const double cx = sum_col(d.parte, fa.nbe, 0, sh);
    const double by = sum_col(d.partr, fa.nbr, 0, sh);
    if (threadIdx.x == 0) {
        const int it = d.ctl[CTL_ITER] + 1;
        const double rho = d.rho[0];
        const double ec = sqrt(s[0]) / fmax(fmax(sqrt(s[1]), sqrt(s[2])), 1e-300);
        const double el = rho * sqrt(s[4]) / fmax(sqrt(s[3]), 1e-300);
        double* h = d.hist + (size_t)(it - 1) * HIST_COLS;
        h[0] = ec; h[1] = el; h[2] = rho; h[3] = 0; h[4] = -rho * cx; h[5] = by; h[6] = 0; h[7] = 0;
        const bool bad = !isfinite(ec) || !isfinite(el);
        d.ctl[CTL_COUNTER] = 0;
        finish_common(d, bad, it > 1 && fmax(ec, el) <= fa.eps, it, fa.use_cond, fa.hnd);
        if (!d.ctl[CTL_DONE] && fa.adapt_every > 0 && it % fa.adapt_every == 0)
            d.rho[0] = adapt_rho(rho, ec, el, fa.mu, fa.nu);
    }
}

// Global state after the per-component tests, run by the block that arrives
// last: the solve ends once every component has stopped (status: NaN, else a
// component at max_iter, else an infeasible component's status, else solved);
// the history row holds the largest of the first two test columns over the
// components tested in this iteration, the summed objectives and (column 6)
// the number of components still running.
__device__ void components_global_state(const Dev& d, const FinishArgs& fa, int it) {
    __shared__ int s_nan, s_maxit, s_inf;
    __shared__ double sh[32 * 8];
    __shared__ double shm[32 * 2];
    if (threadIdx.x == 0) { s_nan = 0; s_maxit = 0; s_inf = 0; }
    __syncthreads();
    double mx[2] = {0.0, 0.0};     // largest eps_c, eps_lambda tested in this iteration
    double sm[3] = {0.0, 0.0, 0.0};  // summed objectives, components still running
    for (int j = threadIdx.x; j < d.ncomp; j += blockDim.x) {
        const volatile double* r = d.comp_res + (size_t)j * HIST_COLS;
        if (*((volatile int*)d.comp_iter + j) == it) {
            mx[0] = fmax(mx[0], r[0]);
            mx[1] = fmax(mx[1], r[1]);
        }
        sm[0] += r[4];
        sm[1] += r[5];
        if (!*((volatile int*)d.comp_done + j)) {
            sm[2] += 1.0;
        } else {
            const int st = *((volatile int*)d.comp_status + j);
            if (st == -6) s_nan = 1;
            if (st == 1) s_maxit = 1;
            if (st == 2 || st == 3) s_inf = st;
        }
    }
    block_sum<3>(sm, sh);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        mx[0] = fmax(mx[0], __shfl_xor_sync(0xffffffffu, mx[0], o));
        mx[1] = fmax(mx[1], __shfl_xor_sync(0xffffffffu, mx[1], o));
    }
    if (lane == 0) { shm[warp * 2] = mx[0]; shm[warp * 2 + 1] = mx[1]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) { mx[0] = fmax(mx[0], shm[w * 2]); mx[1] = fmax(mx[1], shm[w * 2 + 1]); }
        double* h = d.hist + (size_t)(it - 1) * HIST_COLS;
        h[0] = mx[0]; h[1] = mx[1]; h[2] = 0; h[3] = 0; h[4] = sm[0]; h[5] = sm[1]; h[6] = sm[2]; h[7] = 0;
        const int done = sm[2] == 0.0;
        d.ctl[CTL_COUNTER] = 0;
        d.ctl[CTL_ITER] = it;
        if (done) {
            d.ctl[CTL_STATUS] = s_nan ? -6 : (s_maxit ? 1 : (s_inf ? s_inf : 0));
            d.ctl[CTL_DONE] = 1;
        }
        if (fa.use_cond) cudaGraphSetConditional(fa.hnd, done ? 0u : 1u);
    }
}

// Stopping tests of Algorithms 1-2 per independent component (one block per
// component).  A direct sum of SDPs decouples: every step of the iteration
// acts on each summand separately, so each component's iterates are those of
// a solve of that component alone, and its test (Eq. PrimalConsensusResidual /
// DualConsensusResidual with eps_lambda) uses its own clique rows of the
// partial table (columns as in the single-problem tests; <c, x> in column 5
// for Algorithm 1, column 6 for Algorithm 2) and its own <b, y>.  A component
// that passes, reaches max_iter or meets a NaN is frozen from the next
// iteration on.  The block that arrives last sets the global state: the solve
// ends once every component has stopped; the history row holds the largest
// eps_c and eps_lambda over the components tested in this iteration, the
// summed objectives, and (column 6) the number of components still running.
__global__ void __launch_bounds__(256) k_finish_components(Dev d, int form, FinishArgs fa) {
    __shared__ double sh[32 * 8];
    __shared__ int s_was_done;
    if (stopped(d)) return;
    const int c = blockIdx.x;
    const int it = d.ctl[CTL_ITER] + 1;
    if (threadIdx.x == 0) s_was_done = d.comp_done[c];
    __syncthreads();
    if (!s_was_done) {
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int j = d.ccl_ptr[c] + threadIdx.x; j < d.ccl_ptr[c + 1]; j += blockDim.x) {
            const double* pr = d.part + (size_t)d.ccl_idx[j] * PART_COLS;
#pragma unroll
            for (int q = 0; q < 7; ++q) v[q] += __ldcg(pr + q);
        }
        for (int j = d.crow_ptr[c] + threadIdx.x; j < d.crow_ptr[c + 1]; j += blockDim.x) {
            const int i = d.crow_idx[j];
            v[7] += d.b[i] * __ldcg(d.y + i);
        }
        block_sum<8>(v, sh);
        if (threadIdx.x == 0) {
            double ec, el, cost, dobj;
            const double rho = d.rho[c];
            ec = sqrt(v[0]) / fmax(fmax(sqrt(v[1]), sqrt(v[2])), 1e-300);
            if (form == 0) {
                el = rho * sqrt(v[3]) / fmax(sqrt(v[4]), 1e-300);
                cost = v[5];
                dobj = -rho * v[7];
            } else {
                el = rho * sqrt(v[5]) / fmax(sqrt(v[3]), 1e-300);
                cost = -rho * v[6];
                dobj = v[7];
            }
            double* r = d.comp_res + (size_t)c * HIST_COLS;
            r[0] = ec; r[1] = el; r[2] = rho; r[3] = 0; r[4] = cost; r[5] = dobj; r[6] = 0; r[7] = 0;
            int st = 1, done = 0;
            if (!isfinite(ec) || !isfinite(el)) { st = -6; done = 1; }
            else if (it > 1 && fmax(ec, el) <= fa.eps) { st = 0; done = 1; }
            else if (it >= d.max_iter) { st = 1; done = 1; }
            d.comp_iter[c] = it;
            if (done) {
                d.comp_status[c] = st;
                d.comp_done[c] = 1;
            } else if (fa.adapt_every > 0 && it % fa.adapt_every == 0) {
                d.rho[c] = adapt_rho(rho, ec, el, fa.mu, fa.nu);
            }
        }
    }
    if (!last_block_single_writer(d)) return;
    components_global_state(d, fa, it);
}

// ---- Algorithm 3 ------------------------------------------------------------
// Per iteration, with omega = u + v, omega_2 = tau + kappa, nu = omega_1 - omega_2 zeta
// (Eqs. LinearSystem-MatrixInverseResult, Appendix B); h = r = w = 0 in v stay
// exactly zero from the zero start, so only v_z and kappa are stored.

// eta / P with eta = nu_11 + A^T nu_21 + H^T (nu_12 + nu_22)/2 (Eq. ThirBlkFlops_s1),
// nu_11 = u_x - omega_2 c, nu_21 = u_y + omega_2 b, nu_12 = u_s + v_z, nu_22 = u_t.
template <typename T>
__global__ void __launch_bounds__(ETHREADS) k_hsde_eta(Dev d, int G) {
    if (stopped(d)) return;
    const T* us = reinterpret_cast<const T*>(d.ck0);
    const T* vz = reinterpret_cast<const T*>(d.ck1);
    const T* ut = reinterpret_cast<const T*>(d.ck2);
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, lig = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int nloop = (d.NE + ng - 1) / ng;
    for (int it = 0; it < nloop; ++it) {
        const int e = gid + it * ng;
        double acc = 0.0;
        if (e < d.NE) {
            const int j1 = d.sc_ptr[e + 1];
            for (int j = d.sc_ptr[e] + lig; j < j1; j += G) {
                const int q = d.sc_idx[j];
                acc += double(us[q]) + double(vz[q]) + double(ut[q]);
            }
        }
        acc = group_sum(acc, G);
        if (e < d.NE && lig == 0 && !frozen_entry(d, e)) {
            const int c = comp_e(d, e);
            const double w2 = hs_tau_c(d, c) + hs_kappa_c(d, c);
            const double eta = d.x[e] - w2 * d.c[e] + d.atuy[e] + w2 * d.atb[e] + 0.5 * acc;
            d.q[e] = eta * d.pinv[e];
        }
    }
}

// sigma_11 = P^-1 eta - P^-1 A^T (I + A P^-1 A^T)^-1 A P^-1 eta (Eq. MatrixInvFlops);
// partial <c, sigma_11> in parte[block][2].
__global__ void __launch_bounds__(ETHREADS) k_hsde_sigma11(Dev d, int G) {
    __shared__ double sh[32];
    if (stopped(d)) return;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, lig = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int nloop = (d.NE + ng - 1) / ng;
    double cs[1] = {0.0};
    for (int it = 0; it < nloop; ++it) {
        const int e = gid + it * ng;
        double s = 0.0;
        if (e < d.NE) {
            const int q1 = d.at_ptr[e + 1];
            for (int q = d.at_ptr[e] + lig; q < q1; q += G) s += d.at_val[q] * d.hh[d.at_col[q]];
        }
        s = group_sum(s, G);
        if (e < d.NE && lig == 0 && !frozen_entry(d, e)) {
            const double v = d.q[e] - d.pinv[e] * s;
            d.s11[e] = v;
            cs[0] += d.wgt[e] * d.c[e] * v;
        }
    }
    block_sum<1>(cs, sh);
    if (threadIdx.x == 0) d.parte[blockIdx.x * PART_COLS + 2] = cs[0];
}

// sigma_21 = nu_21 - A sigma_11 (Eq. AppendixEqSigma2); partial <b, sigma_21>
// in partr[block][2]; A sigma_11 kept for the primal residual.
__device__ void hsde_gamma_block(const Dev& d, int nbe, int nbr);

__global__ void __launch_bounds__(RTHREADS) k_hsde_sigma21(Dev d, int TPR, int nbe) {
    __shared__ double sh[RTHREADS / 32];
    __shared__ double sh2[32];
    if (stopped(d)) return;
    const int rpb = blockDim.x / TPR, gi = threadIdx.x / TPR, tig = threadIdx.x % TPR;
    const int nloop = (d.m + gridDim.x * rpb - 1) / (gridDim.x * rpb);
    double bs[1] = {0.0};
    for (int it = 0; it < nloop; ++it) {
        const int i = (it * gridDim.x + blockIdx.x) * rpb + gi;
        double s = 0.0;
        if (i < d.m) {
            const int q1 = d.a_ptr[i + 1];
            for (int q = d.a_ptr[i] + tig; q < q1; q += TPR) s += d.a_valw[q] * d.s11[d.a_col[q]];
        }
        s = row_group_sum(s, TPR, sh);
        if (i < d.m && tig == 0 && !frozen_row(d, i)) {
            const int c = comp_r(d, i);
            const double w2 = hs_tau_c(d, c) + hs_kappa_c(d, c);
            d.as11[i] = s;
            const double v = d.y[i] + w2 * d.b[i] - s;
            d.s21[i] = v;
            bs[0] += d.b[i] * v;
        }
    }
    block_sum<1>(bs, sh2);
    if (threadIdx.x == 0) d.partr[blockIdx.x * PART_COLS + 2] = bs[0];
    if (d.comp_mode) return;  // k_hsde_gamma_components runs next, one block per component
    if (last_block_single_writer(d)) hsde_gamma_block(d, nbe, gridDim.x);
}

// The same update per independent component, each with its own embedding
// (component mode; one block per component): gamma_c = zeta_c^T sigma over the
// component's entries and rows, then tau_c, kappa_c.
__global__ void __launch_bounds__(256) k_hsde_gamma_components(Dev d) {
    __shared__ double sh[32 * 2];
    if (stopped(d)) return;
    const int c = blockIdx.x;
    if (d.comp_done[c]) return;
    double v[2] = {0.0, 0.0};
    for (int j = d.cent_ptr[c] + threadIdx.x; j < d.cent_ptr[c + 1]; j += blockDim.x) {
        const int e = d.cent_idx[j];
        v[0] += d.wgt[e] * d.c[e] * d.s11[e];
    }
    for (int j = d.crow_ptr[c] + threadIdx.x; j < d.crow_ptr[c + 1]; j += blockDim.x) {
        const int i = d.crow_idx[j];
        v[1] += d.b[i] * d.s21[i];
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        const double tau = d.hs_tau[c], kappa = d.hs_kappa[c];
        const double gamma = v[0] - v[1];
        const double tauhat = tau + kappa + gamma * (1.0 - d.hs_zdz[c]);
        const double tn = fmax(0.0, tauhat - kappa);
        d.hs_gamma[c] = gamma;
        d.hs_tau[c] = tn;
        d.hs_kappa[c] = kappa - tauhat + tn;
    }
}

// gamma = zeta^T sigma, u_hat_2 = omega_2 + zeta^T u_hat_1 = omega_2 + gamma (1 - zeta^T zeta_hat)
// (Eqs. MatrixInverseResult, FirstBlockElimination); tau <- max(0, u_hat_tau - kappa),
// kappa <- kappa - u_hat_tau + tau (Eqs. HsdeStep2-3 on the R_+ component).
__device__ void hsde_gamma_block(const Dev& d, int nbe, int nbr) {
    __shared__ double sh[32];
    const double cs = sum_col(d.parte, nbe, 2, sh);
    const double bs = sum_col(d.partr, nbr, 2, sh);
    if (threadIdx.x == 0) {
        const double tau = d.scal[SC_TAU], kappa = d.scal[SC_KAPPA];
        const double w2 = tau + kappa;
        const double gamma = cs - bs;
        const double tauhat = w2 + gamma * (1.0 - d.zeta_dot_zhat);
        const double tn = fmax(0.0, tauhat - kappa);
        d.scal[SC_GAMMA] = gamma;
        d.scal[SC_TAUHAT] = tauhat;
        d.scal[SC_TAU] = tn;
        d.scal[SC_KAPPA] = kappa - tauhat + tn;
        d.ctl[CTL_COUNTER] = 0;
    }
}

// u_x <- sigma_11 - gamma zeta_hat_x; A^T u_y with u_y = sigma_21 - gamma zeta_hat_y;
// partials: |A^T u_y + H^T v_z - tau c|^2 (parte col 0) and <c, u_x> (col 1).
template <typename T>
__global__ void __launch_bounds__(ETHREADS) k_hsde_entry_update(Dev d, int G) {
    __shared__ double sh[64];
    if (stopped(d)) return;
    const T* vz = reinterpret_cast<const T*>(d.ck1);
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, lig = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int nloop = (d.NE + ng - 1) / ng;
    double p[2] = {0.0, 0.0};
    for (int it = 0; it < nloop; ++it) {
        const int e = gid + it * ng;
        double a = 0.0, hv = 0.0;
        const bool live = e < d.NE && !frozen_entry(d, e);
        const int ce = live ? comp_e(d, e) : 0;
        const double gamma = live ? hs_gamma_c(d, ce) : 0.0, tau = live ? hs_tau_c(d, ce) : 0.0;
        if (live) {
            const int q1 = d.at_ptr[e + 1];
            for (int q = d.at_ptr[e] + lig; q < q1; q += G) {
                const int i = d.at_col[q];
                a += d.at_val[q] * (d.s21[i] - gamma * d.zhy[i]);
            }
            const int j1 = d.sc_ptr[e + 1];
            for (int j = d.sc_ptr[e] + lig; j < j1; j += G) hv += double(vz[d.sc_idx[j]]);
        }
        a = group_sum(a, G);
        hv = group_sum(hv, G);
        if (live && lig == 0) {
            const double ux = d.s11[e] - gamma * d.zhx[e];
            d.x[e] = ux;
            d.atuy[e] = a;
            const double r = a + hv - tau * d.c[e];
            p[0] += d.wgt[e] * r * r;
            p[1] += d.wgt[e] * d.c[e] * ux;
            if (d.comp_mode) {  // per-entry terms, summed per component by k_finish_hsde_components
                d.t[e] = d.wgt[e] * r * r;
                d.q[e] = d.wgt[e] * d.c[e] * ux;
            }
        }
    }
    block_sum<2>(p, sh);
    if (threadIdx.x == 0) {
        d.parte[blockIdx.x * PART_COLS + 0] = p[0];
        d.parte[blockIdx.x * PART_COLS + 1] = p[1];
    }
}

// u_y <- sigma_21 - gamma zeta_hat_y; A u_x = A sigma_11 - gamma A zeta_hat_x;
// partials |A u_x - tau b|^2 (partr col 0) and <b, u_y> (col 1).
__device__ void finish_hsde_block(const Dev& d, const FinishArgs& fa);

__global__ void __launch_bounds__(RTHREADS) k_hsde_row_update(Dev d, FinishArgs fa) {
    __shared__ double sh[64];
    if (stopped(d)) return;
    double p[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        if (frozen_row(d, i)) continue;
        const int c = comp_r(d, i);
        const double gamma = hs_gamma_c(d, c), tau = hs_tau_c(d, c);
        const double uy = d.s21[i] - gamma * d.zhy[i];
        d.y[i] = uy;
        const double r = d.as11[i] - gamma * d.azhx[i] - tau * d.b[i];
        p[0] += r * r;
        p[1] += d.b[i] * uy;
        if (d.comp_mode) {  // per-row terms, summed per component by k_finish_hsde_components
            d.g[i] = r * r;
            d.hh[i] = d.b[i] * uy;
        }
    }
    block_sum<2>(p, sh);
    if (threadIdx.x == 0) {
        d.partr[blockIdx.x * PART_COLS + 0] = p[0];
        d.partr[blockIdx.x * PART_COLS + 1] = p[1];
    }
    if (d.comp_mode) return;  // k_finish_hsde_components runs next
    if (last_block_single_writer(d)) finish_hsde_block(d, fa);
}

// Algorithm 3 stopping tests: Eqs. HSDEerror and HSDEconsensusResidual when
// tau > 0; otherwise the infeasibility tests (each certificate on its own):
// b^T u_y > 0 and |A^T u_y + H^T v_z| <= eps b^T u_y / |b|  -> primal infeasible,
// c^T u_x < 0 and |A u_x| <= -eps c^T u_x / |c|             -> dual infeasible.
__device__ void finish_hsde_block(const Dev& d, const FinishArgs& fa) {
    __shared__ double sh[32 * 6];
    const double eps = fa.eps;
    const int nbe = fa.nbe, nbr = fa.nbr;
    const int cols6[6] = {0, 1, 2, 3, 4, 5}, cols2[2] = {0, 1};
    double s[6], pe[2], pr[2];
    sum_cols<6>(d.part, fa.npart, cols6, s, sh);
    sum_cols<2>(d.parte, nbe, cols2, pe, sh);
    sum_cols<2>(d.partr, nbr, cols2, pr, sh);
    const double rd2 = pe[0], cux = pe[1], rp2 = pr[0], buy = pr[1];
    if (threadIdx.x == 0) {
        const int it = d.ctl[CTL_ITER] + 1;
        const double tau = d.scal[SC_TAU], kappa = d.scal[SC_KAPPA];
        double* h = d.hist + (size_t)(it - 1) * HIST_COLS;
        h[6] = tau; h[7] = kappa;
        bool bad = !isfinite(tau) || !isfinite(kappa);
        bool stop = false;
        if (tau > 0) {
            const double pc = sqrt(s[0]) / fmax(fmax(sqrt(s[1]), sqrt(s[2])), 1e-300);
            const double dc = sqrt(s[3]) / fmax(fmax(sqrt(s[4]), sqrt(s[5])), 1e-300);
            const double ep = sqrt(rp2) / tau / (1.0 + d.norm_b);
            const double ed = sqrt(rd2) / tau / (1.0 + d.norm_c);
            const double cx = cux / tau, by = buy / tau;
            const double eg = fabs(cx - by) / (1.0 + fabs(cx) + fabs(by));
            const double ec = fmax(pc, dc);
            h[0] = ep; h[1] = ed; h[2] = eg; h[3] = ec; h[4] = cx; h[5] = by;
            bad = bad || !isfinite(ep) || !isfinite(ed) || !isfinite(eg) || !isfinite(ec);
            if (!bad && fmax(fmax(ep, ed), fmax(eg, ec)) <= eps) { d.ctl[CTL_STATUS] = 0; stop = true; }
        } else {
            const double rp = sqrt(rd2), rdd = sqrt(rp2);
            h[0] = rp; h[1] = rdd; h[2] = buy; h[3] = cux; h[4] = 0; h[5] = 0;
            bad = bad || !isfinite(rp) || !isfinite(rdd);
            if (!bad && buy > 0 && rp <= eps * buy / fmax(d.norm_b, 1e-300)) { d.ctl[CTL_STATUS] = 2; stop = true; }
            else if (!bad && cux < 0 && rdd <= -eps * cux / fmax(d.norm_c, 1e-300)) { d.ctl[CTL_STATUS] = 3; stop = true; }
        }
        int done = 0;
        if (bad) { d.ctl[CTL_STATUS] = -6; done = 1; }
        else if (stop) done = 1;
        else if (it >= d.max_iter) { d.ctl[CTL_STATUS] = 1; done = 1; }
        d.ctl[CTL_ITER] = it;
        d.ctl[CTL_COUNTER] = 0;
        if (done) d.ctl[CTL_DONE] = 1;
        if (fa.use_cond) cudaGraphSetConditional(fa.hnd, done ? 0u : 1u);
    }
}

// Algorithm 3 stopping tests per independent component, each component with
// its own embedding (component mode; one block per component): the tests of
// finish_hsde_block on the component's own clique rows of the partial table,
// its own entries (|A^T u_y + H^T v_z - tau c|^2, <c, u_x>, per entry in t and
// q) and rows (|A u_x - tau b|^2, <b, u_y>, per row in g and hh), its own
// tau, kappa and norms of b and c.  A component that passes, proves
// infeasibility, reaches max_iter or meets a NaN is frozen from the next
// iteration on; the block that arrives last sets the global state.
__global__ void __launch_bounds__(256) k_finish_hsde_components(Dev d, FinishArgs fa) {
    __shared__ double sh[32 * 10];
    __shared__ int s_was_done;
    if (stopped(d)) return;
    const int c = blockIdx.x;
    const int it = d.ctl[CTL_ITER] + 1;
    if (threadIdx.x == 0) s_was_done = d.comp_done[c];
    __syncthreads();
    if (!s_was_done) {
        double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int j = d.ccl_ptr[c] + threadIdx.x; j < d.ccl_ptr[c + 1]; j += blockDim.x) {
            const double* pr = d.part + (size_t)d.ccl_idx[j] * PART_COLS;
#pragma unroll
            for (int q = 0; q < 6; ++q) v[q] += __ldcg(pr + q);
        }
        for (int j = d.cent_ptr[c] + threadIdx.x; j < d.cent_ptr[c + 1]; j += blockDim.x) {
            const int e = d.cent_idx[j];
            v[6] += __ldcg(d.t + e);
            v[7] += __ldcg(d.q + e);
        }
        for (int j = d.crow_ptr[c] + threadIdx.x; j < d.crow_ptr[c + 1]; j += blockDim.x) {
            const int i = d.crow_idx[j];
            v[8] += __ldcg(d.g + i);
            v[9] += __ldcg(d.hh + i);
        }
        block_sum<10>(v, sh);
        if (threadIdx.x == 0) {
            const double eps = fa.eps, tau = d.hs_tau[c], kappa = d.hs_kappa[c];
            const double rd2 = v[6], cux = v[7], rp2 = v[8], buy = v[9];
            const double nb = d.hs_nb[c], nc = d.hs_nc[c];
            double* r = d.comp_res + (size_t)c * HIST_COLS;
            r[6] = tau; r[7] = kappa;
            bool bad = !isfinite(tau) || !isfinite(kappa);
            int st = 1, done = 0;
            if (tau > 0) {
                const double pc = sqrt(v[0]) / fmax(fmax(sqrt(v[1]), sqrt(v[2])), 1e-300);
                const double dc = sqrt(v[3]) / fmax(fmax(sqrt(v[4]), sqrt(v[5])), 1e-300);
                const double ep = sqrt(rp2) / tau / (1.0 + nb);
                const double ed = sqrt(rd2) / tau / (1.0 + nc);
                const double cx = cux / tau, by = buy / tau;
                const double eg = fabs(cx - by) / (1.0 + fabs(cx) + fabs(by));
                const double ec = fmax(pc, dc);
                r[0] = ep; r[1] = ed; r[2] = eg; r[3] = ec; r[4] = cx; r[5] = by;
                bad = bad || !isfinite(ep) || !isfinite(ed) || !isfinite(eg) || !isfinite(ec);
                if (!bad && fmax(fmax(ep, ed), fmax(eg, ec)) <= eps) { st = 0; done = 1; }
            } else {
                const double rp = sqrt(rd2), rdd = sqrt(rp2);
                r[0] = rp; r[1] = rdd; r[2] = buy; r[3] = cux; r[4] = 0; r[5] = 0;
                bad = bad || !isfinite(rp) || !isfinite(rdd);
                if (!bad && buy > 0 && rp <= eps * buy / fmax(nb, 1e-300)) { st = 2; done = 1; }
                else if (!bad && cux < 0 && rdd <= -eps * cux / fmax(nc, 1e-300)) { st = 3; done = 1; }
            }
            if (bad) { st = -6; done = 1; }
            else if (!done && it >= d.max_iter) { st = 1; done = 1; }
            d.comp_iter[c] = it;
            if (done) {
                d.comp_status[c] = st;
                d.comp_done[c] = 1;
            }
        }
    }
    if (!last_block_single_writer(d)) return;
    components_global_state(d, fa, it);
}

// ---- set-up and result assembly --------------------------------------------

__global__ void k_init(Dev d, int form, double rho0) {
    for (int c = threadIdx.x; c < d.ncomp; c += blockDim.x) {
        d.rho[c] = rho0;
        d.hs_tau[c] = (form == 2) ? 1.0 : 0.0;
        d.hs_kappa[c] = (form == 2) ? 1.0 : 0.0;
        d.hs_gamma[c] = 0.0;
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        d.scal[SC_TAU] = (form == 2) ? 1.0 : 0.0;
        d.scal[SC_KAPPA] = (form == 2) ? 1.0 : 0.0;
        d.ctl[CTL_DONE] = 0;
        d.ctl[CTL_ITER] = 0;
        d.ctl[CTL_STATUS] = 1;
    }
}

// out_i = sign * rho_i * in_i, rho_i the penalty of entry i (rows = 0) or of
// constraint row i (rows = 1): the variables of Algorithms 1-2 scaled back by
// the penalty of their last iteration.
__global__ void k_scale_rho(Dev d, int n, const double* __restrict__ in, double sign, int rows,
                            double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = sign * (rows ? rho_row(d, i) : rho_entry(d, i)) * in[i];
}

// out = scale * in, or scale * in / *sptr: mode 1 divides only when *sptr > 0
// (the tau of Algorithm 3), mode 2 always divides (certificate normalisation).
__global__ void k_scale_out(int n, const double* __restrict__ in, double scale, const double* sptr,
                            double* __restrict__ out, int mode = 1) {
    double sc = scale;
    if (sptr && (mode == 2 || *sptr > 0)) sc = scale / *sptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = sc * in[i];
}

// out_i = in_i / tau_c for the component c of entry i (rows = 0) or of
// constraint row i (rows = 1), when tau_c > 0: Algorithm 3's X, y and Z in
// component mode.
__global__ void k_scale_hs_tau(Dev d, int n, const double* __restrict__ in, int rows, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double t = d.hs_tau[rows ? d.comp_of_row[i] : d.comp_of_entry[i]];
        out[i] = t > 0 ? in[i] / t : in[i];
    }
}

// dot product helper for certificates: out[0] = sum_i w_i a_i b_i (w may be null), one block
__global__ void k_dot(int n, const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ w,
                      double* out) {
    __shared__ double sh[32];
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += (w ? w[i] : 1.0) * a[i] * b[i];
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) *out = v[0];
}

}  // namespace cdsdp_dev
