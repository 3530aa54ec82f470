// Conjugate-gradient solve of the affine step of Algorithms 1 and 2: the
// system (A D^-1 A^T) y = r of Eqs. OptCondMinYPrimal / OptCondMinYDual,
// the iterative alternative to the cached factor that Section 4.1.1 names.
// In the lower-packed storage the matrix is S = A W D^-1 A^T, applied as two
// sparse passes: u = D^-1 (A^T p) over the pattern entries, then S p = A W u
// over the constraint rows.  CG itself (Hestenes and Stiefel) runs in one
// thread block on the m-vectors, warm-started from the previous y, and stops
// once ||r - S y|| <= cg_tol ||r|| or after cg_max steps: a flag in cg_scal
// turns the remaining launches of the iteration into no-ops.
//   cg_scal[0] = rho_k = ||res||^2, [1] = cg_tol ||r||, [2] = steps, [3] = done
#pragma once

#include "kernels.cuh"
#include "reduce.cuh"

namespace cdsdp_dev {

constexpr int CG_THREADS = 1024;

__device__ __forceinline__ bool cg_done(const Dev& d) { return d.cg_scal[3] != 0.0; }

// Sum over the block in a fixed order, returned to every thread.
__device__ __forceinline__ double cg_block_total(double v, double* sh) {
    double a[1] = {v};
    block_sum<1>(a, sh);
    __shared__ double total;
    if (threadIdx.x == 0) total = a[0];
    __syncthreads();
    const double t = total;
    __syncthreads();
    return t;
}

// u_e = (A^T p)_e / D_e over the pattern entries (lanes of G per entry, as in
// k_xupd).  check = 0 for the product with the warm start, which comes before
// the done flag is reset.
__global__ void __launch_bounds__(ETHREADS) k_cg_atp(Dev d, const double* __restrict__ p, int G, int check) {
    if (stopped(d) || (check && cg_done(d))) return;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, lig = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int nloop = (d.NE + ng - 1) / ng;
    for (int it = 0; it < nloop; ++it) {
        const int e = gid + it * ng;
        double s = 0.0;
        if (e < d.NE) {
            const int q1 = d.at_ptr[e + 1];
            for (int q = d.at_ptr[e] + lig; q < q1; q += G) s += d.at_val[q] * p[d.at_col[q]];
        }
        s = group_sum(s, G);
        if (e < d.NE && lig == 0) d.cg_u[e] = d.dinv[e] * s;
    }
}

// cg_q_i = (A W u)_i over the constraint rows (TPR threads per row, as in k_rows_aw).
__global__ void __launch_bounds__(RTHREADS) k_cg_aw(Dev d, int TPR, int check) {
    __shared__ double sh[RTHREADS / 32];
    if (stopped(d) || (check && cg_done(d))) return;
    const int rpb = blockDim.x / TPR, gi = threadIdx.x / TPR, tig = threadIdx.x % TPR;
    const int nloop = (d.m + gridDim.x * rpb - 1) / (gridDim.x * rpb);
    for (int it = 0; it < nloop; ++it) {
        const int i = (it * gridDim.x + blockIdx.x) * rpb + gi;
        double s = 0.0;
        if (i < d.m) {
            const int q1 = d.a_ptr[i + 1];
            for (int q = d.a_ptr[i] + tig; q < q1; q += TPR) s += d.a_valw[q] * d.cg_u[d.a_col[q]];
        }
        s = row_group_sum(s, TPR, sh);
        if (i < d.m && tig == 0) d.cg_q[i] = s;
    }
}

// res = r - S y0 (cg_q holds S y0), p = res; the tolerance and the done flag.
__global__ void __launch_bounds__(CG_THREADS) k_cg_init(Dev d, const double* __restrict__ r) {
    __shared__ double sh[32];
    if (stopped(d)) return;
    double rr = 0.0, rn = 0.0;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
        const double ri = r[i], res = ri - d.cg_q[i];
        d.cg_res[i] = res;
        d.cg_p[i] = res;
        rr += res * res;
        rn += ri * ri;
    }
    rr = cg_block_total(rr, sh);
    rn = cg_block_total(rn, sh);
    if (threadIdx.x == 0) {
        const double target = d.cg_tol * sqrt(rn);
        d.cg_scal[0] = rr;
        d.cg_scal[1] = target;
        d.cg_scal[2] = 0.0;
        d.cg_scal[3] = (d.cg_max <= 0 || !(sqrt(rr) > target)) ? 1.0 : 0.0;
    }
}

// One CG step with q = S p: alpha = rho / <p, q>, y += alpha p,
// res -= alpha q, beta = rho' / rho, p = res + beta p.
__global__ void __launch_bounds__(CG_THREADS) k_cg_update(Dev d) {
    __shared__ double sh[32];
    if (stopped(d) || cg_done(d)) return;
    const double rr = d.cg_scal[0];
    double pq = 0.0;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) pq += d.cg_p[i] * d.cg_q[i];
    pq = cg_block_total(pq, sh);
    const double alpha = rr / pq;
    double rr2 = 0.0;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
        d.y[i] += alpha * d.cg_p[i];
        const double res = d.cg_res[i] - alpha * d.cg_q[i];
        d.cg_res[i] = res;
        rr2 += res * res;
    }
    rr2 = cg_block_total(rr2, sh);
    const double beta = rr2 / rr;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) d.cg_p[i] = d.cg_res[i] + beta * d.cg_p[i];
    if (threadIdx.x == 0) {
        const double steps = d.cg_scal[2] + 1.0;
        d.cg_scal[0] = rr2;
        d.cg_scal[2] = steps;
        d.cg_scal[3] = (steps >= (double)d.cg_max || !(sqrt(rr2) > d.cg_scal[1])) ? 1.0 : 0.0;
    }
}

// The partial of <b, y> that k_gemv leaves for the stopping test: the whole
// sum in row 0 of column `col`, zeros in rows 1..nrows-1.
__global__ void __launch_bounds__(CG_THREADS) k_cg_finish(Dev d, int col, int nrows) {
    __shared__ double sh[32];
    if (stopped(d)) return;
    double by = 0.0;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) by += d.b[i] * d.y[i];
    by = cg_block_total(by, sh);
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) d.partr[r * PART_COLS + col] = (r == 0) ? by : 0.0;
}

}  // namespace cdsdp_dev
