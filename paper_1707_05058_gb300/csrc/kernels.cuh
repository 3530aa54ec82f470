// Device kernels of the decomposed ADMM iteration (arXiv 1707.05058,
// Algorithms 1-3).  Storage convention (differs from the paper's full vec(),
// equivalently): every symmetric quantity is stored on the lower triangle of
// the extended pattern E*, and inner products weight off-diagonal entries by 2.
// A clique block is stored lower-packed, column-major:
//   entry (a, b), a >= b, of block k at pk_off[k] + b*(2s - b + 1)/2 + (a - b).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdsdp_dev {

enum { CTL_DONE = 0, CTL_ITER = 1, CTL_STATUS = 2, CTL_NAN = 3, CTL_COUNTER = 4, CTL_WORDS = 16 };
// iteration scalars of Algorithm 3
enum { SC_TAU = 0, SC_KAPPA = 1, SC_OMEGA2 = 2, SC_GAMMA = 3, SC_TAUHAT = 4, SC_WORDS = 32 };
enum { HIST_COLS = 8, PART_COLS = 8 };

// Device views of the workspace (all pointers into the caller's buffer).
struct Dev {
    int n, m, NE, p, nd;
    int diag_factor;
    // constants
    const double* c;      // [NE]
    const double* dinv;   // [NE]  1 / D
    const double* pinv;   // [NE]  1 / (1 + D/2)
    const double* wgt;    // [NE]  1 on the diagonal, 2 off it
    const int* a_ptr;     // [m+1]
    const int* a_col;     // [nnzA]
    const double* a_valw; // [nnzA] w_e * A_ie  (A W)
    const int* at_ptr;    // [NE+1]
    const int* at_col;    // [nnzA]
    const double* at_val; // [nnzA] A_ie     (A^T)
    const double* b;      // [m]
    const double* minv;   // [m*m] or [m]
    const double* kinv;   // [m*m] or [m]
    const int* gmap;      // [nd] packed position -> pattern entry
    const int* pk_off;    // [p+1]
    const int* csize;     // [p]
    const int* sc_ptr;    // [NE+1]
    const int* sc_idx;    // [nd]
    const double* zhx;    // [NE] zeta_hat, x part
    const double* zhy;    // [m]  zeta_hat, y part
    const double* atb;    // [NE] A^T b
    const double* azhx;   // [m]  A W zeta_hat_x
    double zeta_dot_zhat, norm_b, norm_c;
    // state
    double* x;            // [NE]
    double* t;            // [NE]
    double* q;            // [NE]
    double* s11;          // [NE]
    double* atuy;         // [NE]
    double* y;            // [m]
    double* g;            // [m]
    double* hh;           // [m]
    double* s21;          // [m]
    double* as11;         // [m]
    void* ck0;            // [nd] clique vectors (float or double)
    void* ck1;
    void* ck2;
    void* vcache;         // [sum_k s_k^2] eigenvectors of the previous iteration (warm start)
    const int* vv_off;    // [p+1] offsets into vcache
    const unsigned char* owner;  // [nd] 1 at the first packed position of each pattern entry
    const double* a_valu; // [nnzA] A_ie unweighted, CSR by rows (reverse pass)
    void* wstore;         // when set, primal projections record W of iteration n at wstore + n * nd
    int wstore_count;     // iterations that fit in wstore
    double* part;         // [p * PART_COLS] per-clique partial sums
    double* parte;        // [NBLK_E * PART_COLS] per-block partials, pattern-entry kernels
    double* partr;        // [NBLK_R * PART_COLS] per-block partials, constraint-row kernels
    double* scal;         // [SC_WORDS]
    int* ctl;             // [CTL_WORDS]
    double* hist;         // [max_iter * HIST_COLS]
    int max_iter;
    // independent components (summands of a direct sum).  The cached inverses
    // are block diagonal: row i of component c is the dense row lrow[i] of
    // the m_c x m_c block at minv_off[c], over the constraints crow_idx[crow_ptr[c] ..].
    int ncomp;
    int rows_contig;      // crow_idx is the identity
    int comp_mode;        // 1: each component stops and freezes on its own test
    const int* comp_of_entry;   // [NE]
    const int* comp_of_clique;  // [p]
    const int* comp_of_row;     // [m]
    const int* lrow;            // [m]
    const int* crow_ptr;        // [ncomp+1]
    const int* crow_idx;        // [m]
    const int* ccl_ptr;         // [ncomp+1]
    const int* ccl_idx;         // [p]
    const long long* minv_off;  // [ncomp]
    int* comp_done;             // [ncomp] 1 once the component has stopped
    int* comp_iter;             // [ncomp] iterations run by the component
    int* comp_status;           // [ncomp] cdsdp_status of the component
    double* comp_res;           // [ncomp * HIST_COLS] last stopping-test row of the component
    double* rho;                // [ncomp] penalty of Algorithms 1-2: one per component when
                                // components stop on their own, else entry 0 for the whole problem
    // Algorithm 3 with one embedding per independent component (component
    // mode): tau, kappa, gamma per component; zhx, zhy, azhx then point at the
    // per-component zeta_hat of each component's own embedding
    double* hs_tau;             // [ncomp]
    double* hs_kappa;           // [ncomp]
    double* hs_gamma;           // [ncomp]
    const double* hs_zdz;       // [ncomp] zeta_c^T zeta_hat_c
    const double* hs_nb;        // [ncomp] ||b_c||
    const double* hs_nc;        // [ncomp] ||c_c|| (weighted lower storage)
    const int* cent_ptr;        // [ncomp+1] pattern entries of each component
    const int* cent_idx;        // [NE]
    // conjugate-gradient affine step (opts.linear_solver = 1)
    double *cg_res, *cg_p, *cg_q;  // [m]
    double* cg_u;                  // [NE]
    double* cg_scal;               // [4]: ||res||^2, target, steps, done
    double cg_tol;
    int cg_max;
};

constexpr int NBLK_E = 1216;  // 152 SMs x 8
constexpr int NBLK_R = 1216;
constexpr int ETHREADS = 256;
constexpr int RTHREADS = 256;
constexpr int FTHREADS = 512;

// Stopping-test arguments handed to the kernel whose last block finishes an iteration.
struct FinishArgs {
    double eps;
    double mu, nu;       // adaptive penalty (Section 7.1.2): factor and balance ratio
    int adapt_every;     // 0: fixed rho; N: apply the rule after every N-th iteration
    int nbe, nbr;        // rows of the per-block partial tables to reduce
    int npart;           // rows of the clique partial table written this iteration
    int enabled;         // 0: this launch does not finish the iteration
    int use_cond;        // 1: inside the graph while loop (set its condition)
    cudaGraphConditionalHandle hnd;
};

// Eigensolver options of the projection kernels.
struct ProjArgs {
    double tolrel;
    int max_sweeps;
    int warm_start;      // reuse the previous iteration's eigenvectors
    int restart;         // cold start every `restart` iterations
    int row_off;         // first row of this launch in the per-block partial table
    int warps_div;       // warp-per-clique launches: warps per block = the maximum / warps_div
    int x_ready;         // Algorithm 1: x was computed by a separate kernel this
                         // iteration (read it) instead of inside the gather
    int cta_variant;     // thread-block projections, float32 orders 36..64: 0 = V in
                         // shared memory (CTAJacobiMid), 1 = V in registers (CTAJacobiReg)
};

__device__ __forceinline__ bool stopped(const Dev& d) {
    return *((volatile int*)d.ctl + CTL_DONE) != 0;
}

// Penalty of Algorithms 1-2 seen by a clique, pattern entry or constraint row.
__device__ __forceinline__ double rho_clique(const Dev& d, int k) {
    return d.rho[d.comp_mode ? d.comp_of_clique[k] : 0];
}
__device__ __forceinline__ double rho_entry(const Dev& d, int e) {
    return d.rho[d.comp_mode ? d.comp_of_entry[e] : 0];
}
__device__ __forceinline__ double rho_row(const Dev& d, int i) {
    return d.rho[d.comp_mode ? d.comp_of_row[i] : 0];
}
// Adaptive penalty rule (Section 7.1.2) on the residual pair (eps_c, eps_lambda).
__device__ __forceinline__ double adapt_rho(double rho, double ep, double ed, double mu, double nu) {
    if (ep >= nu * ed) return rho * mu;
    if (ed >= nu * ep) return rho / mu;
    return rho;
}

// tau, kappa and gamma of Algorithm 3 seen by a pattern entry, constraint row
// or clique: the component's own in component mode, else the single embedding's.
__device__ __forceinline__ double hs_tau_c(const Dev& d, int c) { return d.comp_mode ? d.hs_tau[c] : d.scal[SC_TAU]; }
__device__ __forceinline__ double hs_kappa_c(const Dev& d, int c) {
    return d.comp_mode ? d.hs_kappa[c] : d.scal[SC_KAPPA];
}
__device__ __forceinline__ double hs_gamma_c(const Dev& d, int c) {
    return d.comp_mode ? d.hs_gamma[c] : d.scal[SC_GAMMA];
}
__device__ __forceinline__ int comp_e(const Dev& d, int e) { return d.comp_mode ? d.comp_of_entry[e] : 0; }
__device__ __forceinline__ int comp_r(const Dev& d, int i) { return d.comp_mode ? d.comp_of_row[i] : 0; }
__device__ __forceinline__ int comp_k(const Dev& d, int k) { return d.comp_mode ? d.comp_of_clique[k] : 0; }

// Component freeze: a stopped component's entries, rows and cliques are left alone.
__device__ __forceinline__ bool frozen_clique(const Dev& d, int k) {
    return d.comp_mode && d.comp_done[d.comp_of_clique[k]];
}
__device__ __forceinline__ bool frozen_entry(const Dev& d, int e) {
    return d.comp_mode && d.comp_done[d.comp_of_entry[e]];
}
__device__ __forceinline__ bool frozen_row(const Dev& d, int i) {
    return d.comp_mode && d.comp_done[d.comp_of_row[i]];
}

// Partial dot product of row i of a cached inverse (dense m x m, or block
// diagonal over components) with g, over the row positions t0, t0+step, ...
__device__ __forceinline__ double factor_row_dot(const Dev& d, const double* __restrict__ M, int i,
                                                 const double* __restrict__ g, int t0, int step) {
    double s = 0.0;
    if (d.ncomp <= 1) {
        const double* row = M + (size_t)i * d.m;
        for (int j = t0; j < d.m; j += step) s += row[j] * g[j];
        return s;
    }
    const int c = d.comp_of_row[i], r0 = d.crow_ptr[c], mc = d.crow_ptr[c + 1] - r0;
    const double* row = M + d.minv_off[c] + (size_t)d.lrow[i] * mc;
    if (d.rows_contig) {
        const double* gc = g + r0;
        for (int j = t0; j < mc; j += step) s += row[j] * gc[j];
    } else {
        const int* idx = d.crow_idx + r0;
        for (int j = t0; j < mc; j += step) s += row[j] * g[idx[j]];
    }
    return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block reduction of NV doubles per thread; result valid in
// thread 0.  `sh` holds 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp * NV + k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = (lane < nw) ? sh[lane * NV + k] : 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    }
    __syncthreads();
}

// Called by every thread of a block after thread 0 (the only writer of the
// block's partial sums) has written them; returns true in the block that
// arrives last, which then sees every block's partials (read them through L2).
// The counter lives in ctl and is reset by the finishing block.
__device__ __forceinline__ bool last_block_single_writer(const Dev& d) {
    __shared__ int s_last1;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int ticket = atomicAdd(reinterpret_cast<unsigned int*>(d.ctl + CTL_COUNTER), 1u);
        s_last1 = (ticket == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    return s_last1 != 0;
}

// Per-block sum of NV per-warp values (each warp's value valid in its lane 0);
// thread 0 writes row `row` of the partial table at the listed columns.
template <int NV>
__device__ __forceinline__ void block_partial_row(const double (&v)[NV], double* part, int row, const int (&cols)[NV]) {
    __shared__ double wsum[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) wsum[warp][c] = v[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double* pr = part + (size_t)row * PART_COLS;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += wsum[w][c];
            pr[cols[c]] = s;
        }
    }
}

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }
template <typename T> __device__ __forceinline__ T div_t(T a, T b);
template <> __device__ __forceinline__ float div_t<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double div_t<double>(double a, double b) { return a / b; }

// Jacobi rotation threshold relative to ||W||_F: twice the unit roundoff (see jacobi.cuh).
__host__ __device__ constexpr double jacobi_tolrel(int S, bool fp32) {
    return (void)S, 2.0 * (fp32 ? 5.9604644775390625e-8 : 1.1102230246251565e-16);
}

}  // namespace cdsdp_dev
