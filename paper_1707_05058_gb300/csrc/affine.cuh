// Affine-projection and bookkeeping kernels of Algorithms 1-3 (arXiv 1707.05058):
// the scatter H^T (...) onto the pattern, the sparse products with A W and
// A^T, the solve with the cached inverse, and the deterministic reductions of
// the stopping tests.  All of this runs in float64.
//
// Work decomposition: pattern-entry kernels give each entry a group of G lanes
// (G = power of two <= 32, from the average A^T row length) that split its
// A^T row and reduce by shuffles; constraint-row kernels give each row a
// group of TPR threads (a multiple of 32, from the average A row length).
// Grids are sized to fill the GPU; every per-block partial sum is written by
// a fixed block in a fixed order, so reductions are reproducible.
#pragma once

#include "reduce.cuh"

namespace cdsdp_dev {

// ---- pattern-entry kernels ---------------------------------------------------

// out_e = (alpha c_e + beta sum_{j in H^T(e)} (P_j + gamma Q_j)) * scale_e, with
// alpha (gamma) divided by the entry's rho when alpha_rho (gamma_rho) is set.
// Algorithm 1: bhat / D with bhat = sum_k H_k^T (x_k + lambda_k/rho) - c/rho
// (Appendix A, Eq. bnflopsdef); Algorithm 2: (c - sum_k H_k^T (z_k + lambda_k/rho)) / D
// (right-hand side of Eq. OptCondMinYDual); output assembly: Z = sum_k H_k^T lambda_k.
template <typename T>
__global__ void __launch_bounds__(ETHREADS) k_scatter(Dev d, const T* __restrict__ P, const T* __restrict__ Q,
                                                      double alpha, double beta, double gamma, int alpha_rho,
                                                      int gamma_rho, const double* __restrict__ scale,
                                                      double* __restrict__ out, int check_stop, int G) {
    if (check_stop && stopped(d)) return;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, lig = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int nloop = (d.NE + ng - 1) / ng;
    for (int it = 0; it < nloop; ++it) {  // uniform trip count: every lane reaches the shuffles
        const int e = gid + it * ng;
        double acc = 0.0;
        const bool live = e < d.NE && !(check_stop && frozen_entry(d, e));
        double a = alpha, gm = gamma;
        if (live && (alpha_rho || gamma_rho)) {
            const double ir = 1.0 / rho_entry(d, e);
            if (alpha_rho) a *= ir;
            if (gamma_rho) gm *= ir;
        }
        if (live) {
            const int j1 = d.sc_ptr[e + 1];
            for (int j = d.sc_ptr[e] + lig; j < j1; j += G) {
                const int q = d.sc_idx[j];
                acc += Q ? double(P[q]) + gm * double(Q[q]) : double(P[q]);
            }
        }
        acc = group_sum(acc, G);
        if (live && lig == 0) {
            const double r = a * d.c[e] + beta * acc;
            out[e] = scale ? r * scale[e] : r;
        }
    }
}

// The same scatter walked in packed-position order, for problems whose
// entries mostly lie in one clique (Gs = 1): the thread of position q reads
// the clique values at q, and only the entry's first position (owner[q])
// writes out[e]; an entry in several cliques sums its positions in the order
// of the CSR row, as k_scatter with one lane per entry does (bit-identical).
// Clique values and the index map are read in order (coalesced); the entry
// data are read in the order the cliques list their entries.
template <typename T>
__global__ void __launch_bounds__(ETHREADS) k_scatter_owner(Dev d, const T* __restrict__ P, const T* __restrict__ Q,
                                                            double alpha, double beta, double gamma, int alpha_rho,
                                                            int gamma_rho, const double* __restrict__ scale,
                                                            double* __restrict__ out, int check_stop) {
    if (check_stop && stopped(d)) return;
    const int stride = gridDim.x * blockDim.x;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.nd; q += stride) {
        if (!d.owner[q]) continue;
        const int e = d.gmap[q];
        if (check_stop && frozen_entry(d, e)) continue;
        double a = alpha, gm = gamma;
        if (alpha_rho || gamma_rho) {
            const double ir = 1.0 / rho_entry(d, e);
            if (alpha_rho) a *= ir;
            if (gamma_rho) gm *= ir;
        }
        const int j0 = d.sc_ptr[e], j1 = d.sc_ptr[e + 1];
        double acc = 0.0;
        if (j1 - j0 == 1) {
            acc += Q ? double(P[q]) + gm * double(Q[q]) : double(P[q]);
        } else {
            for (int j = j0; j < j1; ++j) {
                const int qq = d.sc_idx[j];
                acc += Q ? double(P[qq]) + gm * double(Q[qq]) : double(P[qq]);
            }
        }
        const double r = a * d.c[e] + beta * acc;
        out[e] = scale ? r * scale[e] : r;
    }
}

// x_e = t_e - dinv_e (A^T y)_e  (Appendix A, Eq. KKTflops_s1), with the
// per-block partial sum of <c, x> (weighted) in parte[block][0].
__global__ void __launch_bounds__(ETHREADS) k_xupd(Dev d, const double* __restrict__ t, const double* __restrict__ y,
                                                   double* __restrict__ x, int G, int want_cx) {
    __shared__ double sh[32];
    if (stopped(d)) return;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, lig = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int nloop = (d.NE + ng - 1) / ng;
    double cx[1] = {0.0};
    for (int it = 0; it < nloop; ++it) {
        const int e = gid + it * ng;
        double s = 0.0;
        const bool live = e < d.NE && !frozen_entry(d, e);
        if (live) {
            const int q1 = d.at_ptr[e + 1];
            for (int q = d.at_ptr[e] + lig; q < q1; q += G) s += d.at_val[q] * y[d.at_col[q]];
        }
        s = group_sum(s, G);
        if (live && lig == 0) {
            const double xe = t[e] - d.dinv[e] * s;
            x[e] = xe;
            cx[0] += d.wgt[e] * d.c[e] * xe;
        }
    }
    if (!want_cx) return;  // block-uniform
    block_sum<1>(cx, sh);
    if (threadIdx.x == 0) d.parte[blockIdx.x * PART_COLS + 0] = cx[0];
}

// ---- constraint-row kernels ------------------------------------------------

// out_i = (A W v)_i + delta b_i (delta / rho_i when delta_rho); Appendix A
// item (ii): A D^-1 bhat - b.
__global__ void __launch_bounds__(RTHREADS) k_rows_aw(Dev d, const double* __restrict__ v, double delta,
                                                      int delta_rho, double* __restrict__ out, int TPR) {
    __shared__ double sh[RTHREADS / 32];
    if (stopped(d)) return;
    const int rpb = blockDim.x / TPR, gi = threadIdx.x / TPR, tig = threadIdx.x % TPR;
    const int nloop = (d.m + gridDim.x * rpb - 1) / (gridDim.x * rpb);
    for (int it = 0; it < nloop; ++it) {
        const int i = (it * gridDim.x + blockIdx.x) * rpb + gi;
        double s = 0.0;
        const bool live = i < d.m && !frozen_row(d, i);
        if (live) {
            const int q1 = d.a_ptr[i + 1];
            for (int q = d.a_ptr[i] + tig; q < q1; q += TPR) s += d.a_valw[q] * v[d.a_col[q]];
        }
        s = row_group_sum(s, TPR, sh);
        if (live && tig == 0) out[i] = s + (delta_rho ? delta / rho_row(d, i) : delta) * d.b[i];
    }
}

// y = Minv g, Minv the cached inverse (Appendix A item (iii); the paper
// allows a factorisation or the inverse), block diagonal over independent
// components.  Partial of <b, y> in partr[block][col].
__global__ void __launch_bounds__(RTHREADS) k_gemv(Dev d, const double* __restrict__ Minv, const double* __restrict__ g,
                                                   double* __restrict__ y, int col, int TPR) {
    __shared__ double sh[RTHREADS / 32];
    __shared__ double sh2[32];
    if (stopped(d)) return;
    const int rpb = blockDim.x / TPR, gi = threadIdx.x / TPR, tig = threadIdx.x % TPR;
    const int nloop = (d.m + gridDim.x * rpb - 1) / (gridDim.x * rpb);
    double by[1] = {0.0};
    for (int it = 0; it < nloop; ++it) {
        const int i = (it * gridDim.x + blockIdx.x) * rpb + gi;
        double s = 0.0;
        const bool live = i < d.m && !frozen_row(d, i);
        if (live) {
            if (d.diag_factor) {
                if (tig == 0) s = Minv[i] * g[i];
            } else {
                s = factor_row_dot(d, Minv, i, g, tig, TPR);
            }
        }
        s = row_group_sum(s, TPR, sh);
        if (live && tig == 0) {
            y[i] = s;
            by[0] += d.b[i] * s;
        }
    }
    block_sum<1>(by, sh2);
    if (threadIdx.x == 0 && col >= 0) d.partr[blockIdx.x * PART_COLS + col] = by[0];
}

}  // namespace cdsdp_dev
