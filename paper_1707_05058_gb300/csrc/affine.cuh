// Affine-projection and bookkeeping kernels of Algorithms 1-3 (arXiv 1707.05058):
// the scatter H^T (...) onto the pattern, the sparse products with A W and
// A^T, the solve with the cached inverse, and the deterministic reductions of
// the stopping tests.  All of this runs in float64.
#pragma once

#include "kernels.cuh"

namespace cdsdp_dev {

// ---- pattern-entry kernels (grid-stride, one thread per entry) -------------

// out_e = (alpha c_e + beta sum_{j in H^T(e)} (P_j + gamma Q_j)) * scale_e
// Algorithm 1: bhat / D with bhat = sum_k H_k^T (x_k + lambda_k/rho) - c/rho
// (Appendix A, Eq. bnflopsdef); Algorithm 2: (c - sum_k H_k^T (z_k + lambda_k/rho)) / D
// (right-hand side of Eq. OptCondMinYDual); output assembly: Z = sum_k H_k^T lambda_k.
template <typename T>
__global__ void __launch_bounds__(ETHREADS) k_scatter(Dev d, const T* __restrict__ P, const T* __restrict__ Q,
                                                      double alpha, double beta, double gamma,
                                                      const double* __restrict__ scale, double* __restrict__ out,
                                                      int check_stop) {
    if (check_stop && stopped(d)) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.NE; e += gridDim.x * blockDim.x) {
        double acc = 0.0;
        const int j0 = d.sc_ptr[e], j1 = d.sc_ptr[e + 1];
        if (Q) {
            for (int j = j0; j < j1; ++j) {
                const int q = d.sc_idx[j];
                acc += double(P[q]) + gamma * double(Q[q]);
            }
        } else {
            for (int j = j0; j < j1; ++j) acc += double(P[d.sc_idx[j]]);
        }
        double r = alpha * d.c[e] + beta * acc;
        out[e] = scale ? r * scale[e] : r;
    }
}

// x_e = t_e - dinv_e (A^T y)_e  (Appendix A, Eq. KKTflops_s1), with the
// per-block partial sum of <c, x> (weighted) in parte[block][0].
__global__ void __launch_bounds__(ETHREADS) k_xupd(Dev d, const double* __restrict__ t, const double* __restrict__ y,
                                                   double* __restrict__ x) {
    __shared__ double sh[32];
    if (stopped(d)) return;
    double cx[1] = {0.0};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.NE; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = d.at_ptr[e]; q < d.at_ptr[e + 1]; ++q) s += d.at_val[q] * y[d.at_col[q]];
        const double xe = t[e] - d.dinv[e] * s;
        x[e] = xe;
        cx[0] += d.wgt[e] * d.c[e] * xe;
    }
    block_sum<1>(cx, sh);
    if (threadIdx.x == 0) d.parte[blockIdx.x * PART_COLS + 0] = cx[0];
}

// ---- constraint-row kernels (one warp per row of A) ------------------------

// out_i = (A W v)_i + delta b_i ; Appendix A item (ii): A D^-1 bhat - b.
__global__ void __launch_bounds__(RTHREADS) k_rows_aw(Dev d, const double* __restrict__ v, double delta,
                                                      double* __restrict__ out) {
    if (stopped(d)) return;
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = w0; i < d.m; i += nw) {
        double s = 0.0;
        for (int q = d.a_ptr[i] + lane; q < d.a_ptr[i + 1]; q += 32) s += d.a_valw[q] * v[d.a_col[q]];
        s = warp_sum(s);
        if (lane == 0) out[i] = s + delta * d.b[i];
    }
}

// y = Minv g, Minv the cached inverse (Appendix A item (iii); the paper
// allows a factorisation or the inverse).  Partial of <b, y> in partr[block][col].
__global__ void __launch_bounds__(RTHREADS) k_gemv(Dev d, const double* __restrict__ Minv, const double* __restrict__ g,
                                                   double* __restrict__ y, int col) {
    __shared__ double sh[32];
    if (stopped(d)) return;
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    double by[1] = {0.0};
    for (int i = w0; i < d.m; i += nw) {
        double s;
        if (d.diag_factor) {
            s = Minv[i] * g[i];
        } else {
            s = 0.0;
            const double* row = Minv + (size_t)i * d.m;
            for (int j = lane; j < d.m; j += 32) s += row[j] * g[j];
            s = warp_sum(s);
        }
        if (lane == 0) {
            y[i] = s;
            by[0] += d.b[i] * s;
        }
    }
    block_sum<1>(by, sh);
    if (threadIdx.x == 0 && col >= 0) d.partr[blockIdx.x * PART_COLS + col] = by[0];
}

// ---- reductions of the stopping tests (one block, fixed order) -------------

__device__ __forceinline__ double sum_col(const double* part, int rows, int col, double* sh) {
    double v[1] = {0.0};
    for (int r = threadIdx.x; r < rows; r += blockDim.x) v[0] += part[(size_t)r * PART_COLS + col];
    block_sum<1>(v, sh);
    return v[0];  // valid in thread 0
}

__device__ __forceinline__ void finish_common(Dev d, bool nan_seen, bool converged, int it, int use_cond,
                                              cudaGraphConditionalHandle hnd) {
    int done = 0;
    if (nan_seen) { d.ctl[CTL_STATUS] = -6; done = 1; }
    else if (converged) { d.ctl[CTL_STATUS] = 0; done = 1; }
    else if (it >= d.max_iter) { d.ctl[CTL_STATUS] = 1; done = 1; }
    d.ctl[CTL_ITER] = it;
    if (done) d.ctl[CTL_DONE] = 1;
    if (use_cond) cudaGraphSetConditional(hnd, done ? 0u : 1u);
}

// Algorithm 1 stopping test (Eq. PrimalConsensusResidual, eps_lambda).
__global__ void k_finish_primal(Dev d, double rho, double eps, int nbe, int nbr, int use_cond,
                                cudaGraphConditionalHandle hnd) {
    __shared__ double sh[32];
    if (stopped(d)) { if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(hnd, 0u); return; }
    double s[5];
    for (int c = 0; c < 5; ++c) s[c] = sum_col(d.part, d.p, c, sh);
    const double cx = sum_col(d.parte, nbe, 0, sh);
    const double by = sum_col(d.partr, nbr, 0, sh);
    if (threadIdx.x == 0) {
        const int it = d.ctl[CTL_ITER] + 1;
        const double ec = sqrt(s[0]) / fmax(fmax(sqrt(s[1]), sqrt(s[2])), 1e-300);
        const double el = rho * sqrt(s[3]) / fmax(sqrt(s[4]), 1e-300);
        double* h = d.hist + (size_t)(it - 1) * HIST_COLS;
        h[0] = ec; h[1] = el; h[2] = 0; h[3] = 0; h[4] = cx; h[5] = -rho * by; h[6] = 0; h[7] = 0;
        const bool bad = !isfinite(ec) || !isfinite(el);
        finish_common(d, bad, it > 1 && fmax(ec, el) <= eps, it, use_cond, hnd);
    }
}

}  // namespace cdsdp_dev
