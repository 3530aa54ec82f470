// Maximum-determinant positive definite completion (Section 7.1.1) of a
// partial matrix X given on the extended chordal pattern E*.
//
// The completion W is the unique positive definite matrix with W = X on E*
// and (W^-1)_ij = 0 off E* (Grone, Johnson, Sa and Wolkowicz 1984); on a
// chordal pattern it follows from a perfect elimination order v_1..v_n
// (Vandenberghe and Andersen, Chapter 10.2).  With N_k the neighbours of v_k
// eliminated after it (a clique),
//   t_k = X[N_k, N_k]^-1 X[N_k, v_k],   s_k = X[v_k, v_k] - X[v_k, N_k] t_k,
// all s_k > 0 exactly when every clique block of X is positive definite,
// log det W = sum_k log s_k, and, for k = n-1 down to 1, the free entries of
// column v_k are W[j, v_k] = W[j, N_k] t_k for every later j outside N_k.
//
// GPU design.
//   k_cmp_factor   one warp per vertex: gathers X[N, N] and X[N, v] from the
//                  pattern (binary search in the column-major lower pattern),
//                  Cholesky in shared memory, t_k and s_k.  Every vertex is
//                  independent, so this is one launch over all n vertices.
//   k_cmp_logdet   one thread block per component: sum of log s_k in a fixed
//                  order.
//   k_cmp_scatter  the given entries into the dense blocks.
//   k_cmp_step     one launch per step of the recurrence (the launches are
//                  captured once into a CUDA graph and replayed); within a step each
//                  thread owns one later vertex j of one component (all
//                  components advance together, aligned at their last
//                  vertex), reads rows N_k of the block at column j
//                  (coalesced) and writes W[v_k, j] and W[j, v_k].
// The dense output holds one row-major n_c x n_c block per component
// (independent components complete independently; entries between them are
// zero), vertices of a block in ascending order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cdsdp_internal.h"

namespace cdsdp_impl {
namespace {

constexpr size_t kCmpAlign = 256;
constexpr int kStepThreads = 256;
constexpr size_t kMaxWarpSmem = 200 * 1024;  // largest shared block per warp of the factor kernel

inline size_t align_up(size_t x) { return (x + kCmpAlign - 1) / kCmpAlign * kCmpAlign; }

// Scratch layout (byte offsets, all 256-aligned).  The index section [0, idx_end)
// is copied from the host image; the rest is written by the kernels.
struct CmpLayout {
    size_t lt_ptr, lt_idx, colptr, prow, pcol, comp, loc, posl, peo_cat, peo_off, woff, idx_end;
    size_t T, schur, logdet, flag, total;
    int smax = 0, ncomp = 0, maxnc = 0;
    long long welems = 0;
};

CmpLayout cmp_layout(const HostProblem& hp) {
    CmpLayout L;
    const size_t n = hp.n, NE = hp.prow.size(), nl = hp.lt_idx.size(), C = hp.ncomp;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + std::max<size_t>(bytes, 1)); return at; };
    L.lt_ptr = take((n + 1) * 4);
    L.lt_idx = take(nl * 4);
    L.colptr = take((n + 1) * 4);
    L.prow = take(NE * 4);
    L.pcol = take(NE * 4);
    L.comp = take(n * 4);
    L.loc = take(n * 4);
    L.posl = take(n * 4);
    L.peo_cat = take(n * 4);
    L.peo_off = take((C + 1) * 4);
    L.woff = take(C * 8);
    L.idx_end = o;
    L.T = take(nl * 8);
    L.schur = take(n * 8);
    L.logdet = take(C * 8);
    L.flag = take(16);
    L.total = o;
    L.ncomp = (int)C;
    for (int v = 0; v < hp.n; ++v) L.smax = std::max(L.smax, hp.lt_ptr[v + 1] - hp.lt_ptr[v]);
    return L;
}

// Host image of the index section, and the per-component block offsets.
void cmp_image(const HostProblem& hp, const CmpLayout& L, std::vector<unsigned char>& img,
               std::vector<long long>& woff_out, int& maxnc) {
    const int n = hp.n, C = hp.ncomp;
    img.assign(L.idx_end, 0);
    auto put = [&](size_t off, const void* src, size_t bytes) { if (bytes) std::memcpy(img.data() + off, src, bytes); };
    put(L.lt_ptr, hp.lt_ptr.data(), (n + 1) * 4);
    put(L.lt_idx, hp.lt_idx.data(), hp.lt_idx.size() * 4);
    put(L.colptr, hp.colptr.data(), (n + 1) * 4);
    put(L.prow, hp.prow.data(), hp.prow.size() * 4);
    put(L.pcol, hp.pcol.data(), hp.pcol.size() * 4);
    put(L.comp, hp.comp_of_vertex.data(), n * 4);
    // vertices of each component: ascending (local index) and in elimination order
    std::vector<int> cnt(C + 1, 0), loc(n), posl(n), peo_cat(n);
    for (int v = 0; v < n; ++v) loc[v] = cnt[hp.comp_of_vertex[v]]++;
    std::vector<int> peo_off(C + 1, 0);
    for (int c = 0; c < C; ++c) peo_off[c + 1] = peo_off[c] + cnt[c];
    std::vector<int> fill(peo_off.begin(), peo_off.end() - 1);
    for (int k = 0; k < n; ++k) {
        const int v = hp.peo[k], c = hp.comp_of_vertex[v];
        posl[v] = fill[c] - peo_off[c];
        peo_cat[fill[c]++] = v;
    }
    woff_out.assign(C + 1, 0);
    maxnc = 0;
    for (int c = 0; c < C; ++c) {
        woff_out[c + 1] = woff_out[c] + (long long)cnt[c] * cnt[c];
        maxnc = std::max(maxnc, cnt[c]);
    }
    put(L.loc, loc.data(), n * 4);
    put(L.posl, posl.data(), n * 4);
    put(L.peo_cat, peo_cat.data(), n * 4);
    put(L.peo_off, peo_off.data(), (C + 1) * 4);
    put(L.woff, woff_out.data(), C * 8);
}

// Pattern value of entry (i, j): binary search of max(i, j) among the rows of
// column min(i, j).  Sets bit 2 of *flag when the entry is not in the pattern.
__device__ __forceinline__ double pattern_value(int i, int j, const int* __restrict__ colptr,
                                                const int* __restrict__ prow, const double* __restrict__ X,
                                                int* flag) {
    const int r = max(i, j), c = min(i, j);
    int lo = colptr[c], hi = colptr[c + 1] - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int pr = prow[mid];
        if (pr == r) return X[mid];
        if (pr < r) lo = mid + 1;
        else hi = mid - 1;
    }
    atomicOr(flag, 2);
    return 0.0;
}

// One warp per vertex v: t = X[N,N]^-1 X[N,v] and s = X[v,v] - X[v,N] t by a
// Cholesky factorisation X[N,N] = R R^T in shared memory (ld x ld lower block
// plus two vectors per warp).  A pivot or Schur complement that is not
// positive sets bit 1 of *flag (no completion); the pivot is then replaced by
// 1 so that the warp finishes with finite values.
__global__ void k_cmp_factor(int n, int ld, int wpb, const int* __restrict__ lt_ptr, const int* __restrict__ lt_idx,
                             const int* __restrict__ colptr, const int* __restrict__ prow,
                             const double* __restrict__ X, double* __restrict__ T, double* __restrict__ schur,
                             int* flag) {
    extern __shared__ double cmp_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = blockIdx.x * wpb + warp;
    if (v >= n) return;  // warp-uniform
    double* M = cmp_smem + (size_t)warp * (ld * ld + 2 * ld);
    double* z = M + ld * ld;
    double* t = z + ld;
    const int beg = lt_ptr[v], s = lt_ptr[v + 1] - beg;
    const int* N = lt_idx + beg;
    for (int f = lane; f < s * s; f += 32) {
        const int a = f / s, b = f - a * s;
        if (b <= a) M[a * ld + b] = pattern_value(N[a], N[b], colptr, prow, X, flag);
    }
    for (int a = lane; a < s; a += 32) z[a] = pattern_value(N[a], v, colptr, prow, X, flag);
    __syncwarp();
    bool bad = false;
    // right-looking Cholesky, lower triangle
    for (int j = 0; j < s; ++j) {
        double d = M[j * ld + j];
        if (!(d > 0.0) || !isfinite(d)) { bad = true; d = 1.0; }
        const double rjj = sqrt(d);
        __syncwarp();
        if (lane == 0) M[j * ld + j] = rjj;
        for (int i = j + 1 + lane; i < s; i += 32) M[i * ld + j] /= rjj;
        __syncwarp();
        for (int i = j + 1 + lane; i < s; i += 32) {
            const double lij = M[i * ld + j];
            for (int k = j + 1; k <= i; ++k) M[i * ld + k] -= lij * M[k * ld + j];
        }
        __syncwarp();
    }
    // forward solve R w = r (in z), then s = x_vv - |w|^2
    for (int j = 0; j < s; ++j) {
        const double wj = z[j] / M[j * ld + j];
        __syncwarp();
        if (lane == 0) z[j] = wj;
        for (int i = j + 1 + lane; i < s; i += 32) z[i] -= M[i * ld + j] * wj;
        __syncwarp();
    }
    double q = 0.0;
    for (int a = lane; a < s; a += 32) q += z[a] * z[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    // back solve R^T t = w
    for (int a = lane; a < s; a += 32) t[a] = z[a];
    __syncwarp();
    for (int j = s - 1; j >= 0; --j) {
        const double tj = t[j] / M[j * ld + j];
        __syncwarp();
        if (lane == 0) t[j] = tj;
        for (int i = lane; i < j; i += 32) t[i] -= M[j * ld + i] * tj;
        __syncwarp();
    }
    for (int a = lane; a < s; a += 32) T[beg + a] = t[a];
    if (lane == 0) {
        const double sv = X[colptr[v]] - q;  // the first row of column v is v itself
        if (!(sv > 0.0) || !isfinite(sv)) bad = true;
        schur[v] = sv;
        if (bad) atomicOr(flag, 1);
    }
}

// log det of each component's completion: sum of log s over its vertices, in
// elimination order, strided partials then a fixed tree.
__global__ void k_cmp_logdet(const int* __restrict__ peo_cat, const int* __restrict__ peo_off,
                             const double* __restrict__ schur, double* __restrict__ logdet) {
    __shared__ double part[256];
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int q = peo_off[c] + threadIdx.x; q < peo_off[c + 1]; q += blockDim.x) acc += log(schur[peo_cat[q]]);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) logdet[c] = part[0];
}

// Given entries into the dense blocks (both triangles).
__global__ void k_cmp_scatter(int NE, const int* __restrict__ prow, const int* __restrict__ pcol,
                              const int* __restrict__ comp, const int* __restrict__ loc,
                              const int* __restrict__ peo_off, const long long* __restrict__ woff,
                              const double* __restrict__ X, double* __restrict__ W) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NE; e += gridDim.x * blockDim.x) {
        const int i = prow[e], j = pcol[e], c = comp[i];
        const size_t nc = peo_off[c + 1] - peo_off[c];
        double* Wc = W + woff[c];
        const size_t li = loc[i], lj = loc[j];
        Wc[li * nc + lj] = X[e];
        Wc[lj * nc + li] = X[e];
    }
}

// Step r of the recurrence: in every component with n_c > r, the vertex at
// elimination position k = n_c - 1 - r gets its free entries against every
// vertex eliminated after it.
__global__ void __launch_bounds__(kStepThreads) k_cmp_step(int n, int r, const int* __restrict__ lt_ptr,
                                                         const int* __restrict__ lt_idx, const int* __restrict__ comp,
                                                         const int* __restrict__ loc, const int* __restrict__ posl,
                                                         const int* __restrict__ peo_cat,
                                                         const int* __restrict__ peo_off,
                                                         const long long* __restrict__ woff,
                                                         const double* __restrict__ T, double* __restrict__ W) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = comp[j];
    const int nc = peo_off[c + 1] - peo_off[c];
    const int k = nc - 1 - r;
    if (k < 0 || posl[j] <= k) return;
    const int v = peo_cat[peo_off[c] + k];
    const int beg = lt_ptr[v], s = lt_ptr[v + 1] - beg;
    // j among the later neighbours of v: a given entry
    int lo = 0, hi = s - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int u = lt_idx[beg + mid];
        if (u == j) return;
        if (u < j) lo = mid + 1;
        else hi = mid - 1;
    }
    double* Wc = W + woff[c];
    const size_t lj = loc[j], ncz = nc;
    double acc = 0.0;
    for (int a = 0; a < s; ++a) acc += Wc[(size_t)loc[lt_idx[beg + a]] * ncz + lj] * T[beg + a];
    const size_t lv = loc[v];
    Wc[lv * ncz + lj] = acc;
    Wc[lj * ncz + lv] = acc;
}

int cuda_fail(std::string* err, cudaError_t e, const char* what) {
    if (err) *err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return CDSDP_ERR_CUDA;
}

}  // namespace

void completion_release(CmpGraph& g) {
    if (g.exec) cudaGraphExecDestroy((cudaGraphExec_t)g.exec);
    g.exec = nullptr;
    g.scratch = nullptr;
    g.W = nullptr;
}

int completion_sizes(const HostProblem& hp, size_t* scratch_bytes, long long* w_elems, long long* w_offsets) {
    const CmpLayout L = cmp_layout(hp);
    std::vector<unsigned char> img;
    std::vector<long long> woff;
    int maxnc = 0;
    cmp_image(hp, L, img, woff, maxnc);
    if (scratch_bytes) *scratch_bytes = L.total;
    if (w_elems) *w_elems = woff[hp.ncomp];
    if (w_offsets) std::copy(woff.begin(), woff.end(), w_offsets);
    return CDSDP_SOLVED;
}

int completion_run(const HostProblem& hp, const double* d_X, void* d_scratch, size_t scratch_bytes, double* d_W,
                   double* logdet, void* stream, std::string* err, CmpGraph* cache) {
    if (!d_X || !d_scratch) return CDSDP_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_scratch) % kCmpAlign) return CDSDP_ERR_ARG;
    const CmpLayout L = cmp_layout(hp);
    if (scratch_bytes < L.total) return CDSDP_ERR_NOMEM;
    const int ld = std::max(1, L.smax);
    const size_t per_warp = (size_t)(ld * ld + 2 * ld) * sizeof(double);
    if (per_warp > kMaxWarpSmem) return CDSDP_ERR_UNSUPPORTED;
    std::vector<unsigned char> img;
    std::vector<long long> woff;
    int maxnc = 0;
    cmp_image(hp, L, img, woff, maxnc);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* g = (unsigned char*)d_scratch;
    const int n = hp.n, NE = (int)hp.prow.size(), C = hp.ncomp;
    cudaError_t e;
#define CMP_CK(call)                                        \
    do {                                                    \
        e = (call);                                         \
        if (e != cudaSuccess) return cuda_fail(err, e, #call); \
    } while (0)
    CMP_CK(cudaMemcpyAsync(g, img.data(), img.size(), cudaMemcpyHostToDevice, st));
    CMP_CK(cudaMemsetAsync(g + L.flag, 0, 16, st));
    const int* lt_ptr = (const int*)(g + L.lt_ptr);
    const int* lt_idx = (const int*)(g + L.lt_idx);
    const int* colptr = (const int*)(g + L.colptr);
    const int* prow = (const int*)(g + L.prow);
    const int* pcol = (const int*)(g + L.pcol);
    const int* comp = (const int*)(g + L.comp);
    const int* loc = (const int*)(g + L.loc);
    const int* posl = (const int*)(g + L.posl);
    const int* peo_cat = (const int*)(g + L.peo_cat);
    const int* peo_off = (const int*)(g + L.peo_off);
    const long long* dwoff = (const long long*)(g + L.woff);
    double* T = (double*)(g + L.T);
    double* schur = (double*)(g + L.schur);
    double* dlog = (double*)(g + L.logdet);
    int* flag = (int*)(g + L.flag);
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / per_warp));
    const size_t smem = per_warp * wpb;
    if (smem > 48 * 1024) CMP_CK(cudaFuncSetAttribute(k_cmp_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_cmp_factor<<<(n + wpb - 1) / wpb, 32 * wpb, smem, st>>>(n, ld, wpb, lt_ptr, lt_idx, colptr, prow, d_X, T,
                                                               schur, flag);
    CMP_CK(cudaGetLastError());
    int hflag = 0;
    CMP_CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CMP_CK(cudaStreamSynchronize(st));
    if (hflag & 2) {
        if (err) *err = "completion: pattern inconsistent with the elimination order";
        return CDSDP_ERR_ARG;
    }
    if (hflag & 1) return CDSDP_NOT_PD;
    k_cmp_logdet<<<C, 256, 0, st>>>(peo_cat, peo_off, schur, dlog);
    CMP_CK(cudaGetLastError());
    if (d_W) {
        const int gs = std::max(1, std::min(4096, (NE + 255) / 256));
        k_cmp_scatter<<<gs, 256, 0, st>>>(NE, prow, pcol, comp, loc, peo_off, dwoff, d_X, d_W);
        CMP_CK(cudaGetLastError());
        const int gn = (n + kStepThreads - 1) / kStepThreads;
        auto steps = [&](cudaStream_t s2) {
            for (int r = 1; r < maxnc; ++r)
                k_cmp_step<<<gn, kStepThreads, 0, s2>>>(n, r, lt_ptr, lt_idx, comp, loc, posl, peo_cat, peo_off,
                                                        dwoff, T, d_W);
            return cudaGetLastError();
        };
        if (!cache || maxnc < 2) {
            CMP_CK(steps(st));
        } else {
            if (!cache->exec || cache->scratch != d_scratch || cache->W != d_W) {
                completion_release(*cache);
                cudaStream_t cs;
                CMP_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const cudaError_t e2 = steps(cs);
                    e = cudaStreamEndCapture(cs, &graph);
                    if (e2 != cudaSuccess) e = e2;
                }
                cudaStreamDestroy(cs);
                cudaGraphExec_t exec = nullptr;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(err, e, "completion graph");
                cache->exec = exec;
                cache->scratch = d_scratch;
                cache->W = d_W;
            }
            CMP_CK(cudaGraphLaunch((cudaGraphExec_t)cache->exec, st));
        }
    }
    if (logdet) {
        CMP_CK(cudaMemcpyAsync(logdet, dlog, C * sizeof(double), cudaMemcpyDeviceToHost, st));
        CMP_CK(cudaStreamSynchronize(st));
    }
#undef CMP_CK
    return CDSDP_SOLVED;
}

}  // namespace cdsdp_impl
