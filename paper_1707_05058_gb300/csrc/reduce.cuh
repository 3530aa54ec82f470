// Device-side reductions shared by several translation units (inline only):
// lane-group and row-group sums, the fixed-order sums of partial-sum tables,
// and the stopping test of Algorithm 1 (Eq. PrimalConsensusResidual and
// eps_lambda of Section 4.1.4).
#pragma once

#include "kernels.cuh"

namespace cdsdp_dev {

// Sum over the G lanes of an aligned lane group (result in every lane of it).
__device__ __forceinline__ double group_sum(double v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float group_sum(float v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduction over a row group of TPR threads (TPR a multiple of 32, the group
// is TPR/32 consecutive warps of the block); result valid in the group's
// first thread.  `sh` holds blockDim/32 doubles.
__device__ __forceinline__ double row_group_sum(double v, int TPR, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpg = TPR >> 5;
    if (wpg == 1) return v;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if ((warp % wpg) == 0 && lane == 0)
        for (int w = 0; w < wpg; ++w) s += sh[warp + w];
    return s;
}

// ---- reductions of the stopping tests (one block, fixed order) -------------

// Sums of NC columns of a partial-sum table, one pass; valid in thread 0.
template <int NC>
__device__ __forceinline__ void sum_cols(const double* part, int rows, const int (&cols)[NC], double (&out)[NC],
                                         double* sh) {
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = 0.0;
    const int stride = blockDim.x;
    int r = threadIdx.x;
    for (; r + 3 * stride < rows; r += 4 * stride) {  // four rows in flight per thread
        double v[4][NC];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < NC; ++c) v[u][c] = __ldcg(part + (size_t)(r + u * stride) * PART_COLS + cols[c]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < NC; ++c) out[c] += v[u][c];
    }
    for (; r < rows; r += stride)
#pragma unroll
        for (int c = 0; c < NC; ++c) out[c] += __ldcg(part + (size_t)r * PART_COLS + cols[c]);
    block_sum<NC>(out, sh);
}

__device__ __forceinline__ double sum_col(const double* part, int rows, int col, double* sh) {
    const int cols[1] = {col};
    double out[1];
    sum_cols<1>(part, rows, cols, out, sh);
    return out[0];
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

// Algorithm 1 stopping test (Eq. PrimalConsensusResidual, eps_lambda), run by
// every thread of the block that finishes the iteration.
__device__ __forceinline__ void finish_primal_block(const Dev& d, const FinishArgs& fa) {
    __shared__ double sh[32 * 6];
    const int cols[6] = {0, 1, 2, 3, 4, 5};
    double s[6];
    sum_cols<6>(d.part, fa.npart, cols, s, sh);
    const double cx = s[5];
    const double by = sum_col(d.partr, fa.nbr, 0, sh);
    if (threadIdx.x == 0) {
        const int it = d.ctl[CTL_ITER] + 1;
        const double rho = d.rho[0];
        const double ec = sqrt(s[0]) / fmax(fmax(sqrt(s[1]), sqrt(s[2])), 1e-300);
        const double el = rho * sqrt(s[3]) / fmax(sqrt(s[4]), 1e-300);
        double* h = d.hist + (size_t)(it - 1) * HIST_COLS;
        h[0] = ec; h[1] = el; h[2] = rho; h[3] = 0; h[4] = cx; h[5] = -rho * by; h[6] = 0; h[7] = 0;
        const bool bad = !isfinite(ec) || !isfinite(el);
        d.ctl[CTL_COUNTER] = 0;
        finish_common(d, bad, it > 1 && fmax(ec, el) <= fa.eps, it, fa.use_cond, fa.hnd);
        if (!d.ctl[CTL_DONE] && fa.adapt_every > 0 && it % fa.adapt_every == 0)
            d.rho[0] = adapt_rho(rho, ec, el, fa.mu, fa.nu);
    }
}

}  // namespace cdsdp_dev
