// Launchers of the batched projection kernels, spread over several
// translation units (by precision and order) so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace cdsdp_dev {

// Padded orders of the projection kernels: one warp per clique up to 32, one
// thread block per clique above (float32 up to 128, float64 up to 64).
constexpr int kProjClasses[] = {2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32, 36, 40, 44, 48, 52, 56, 60, 64, 96, 128};
constexpr int kNumProjClasses = 22;
constexpr int kMaxWarpOrder = 32;
constexpr int kMaxOrderF32 = 128;
constexpr int kMaxOrderF64 = 64;
// Lanes per clique of the warp projections: orders up to 8 share a warp four
// ways, up to 16 two ways (every lane then owns pair-blocks and a row of V),
// larger orders take the whole warp.
__host__ __device__ constexpr int proj_lanes(int S) { return S <= 8 ? 8 : (S <= 16 ? 16 : 32); }
// Warps per block allowed for a projection kernel of padded order S
// (registers: 16 warps only while a thread needs <= 128 registers).
__host__ __device__ constexpr int proj_max_warps(int S, bool fp32) { return S <= 16 ? 16 : (fp32 ? 8 : 4); }

// Launch shape of a projection over `nlist` cliques, one clique per warp:
// the grid is a multiple of the 152 SMs when it can be, and blocks are made as
// wide as allowed so that every SM receives the same number of warps.
struct ProjShape { int wpb, grid; };
inline int proj_cta_grid(int nlist) { return nlist < 1 ? 1 : (nlist < 152 * 32 ? nlist : 152 * 32); }
inline ProjShape proj_shape(int nlist, int max_warps) {
    constexpr int kSMs = 152;
    if (nlist < 1) return {1, 1};
    const int mult = (nlist + kSMs * max_warps - 1) / (kSMs * max_warps);
    int grid = kSMs * mult;
    const int wpb = (nlist + grid - 1) / grid;
    grid = (nlist + wpb - 1) / wpb;
    if (grid > kSMs * 32) grid = kSMs * 32;  // grid-stride beyond this
    return {wpb, grid};
}

inline int proj_class_of(int s) {
    for (int c = 0; c < kNumProjClasses; ++c)
        if (s <= kProjClasses[c]) return c;
    return -1;
}

// form 0/1/2: Algorithm 1/2/3 projection kernels over `list` (cliques of
// order <= kProjClasses[cls]).
// `fa` is used by the primal form only (its last block finishes the iteration).
// Instantiations live in proj_{f32,f64}_{small,large}.cu (orders 2..16 / 20..32).
#define CDSDP_DECLARE_PROJ(SUF)                                                                                 \
    cudaError_t launch_proj_##SUF(int form, int cls, const Dev& d, const int* list, int nlist,                 \
                                  const ProjArgs& pa, const FinishArgs& fa, cudaStream_t st);                    \
    cudaError_t launch_proj_standalone_##SUF(int cls, int p, const int* off, const int* size, const void* W,   \
                                             void* X, void* eig, const int* voff, void* V, const int* vvoff,  \
                                             double tolrel, int max_sweeps, cudaStream_t st);
CDSDP_DECLARE_PROJ(f32_small)
CDSDP_DECLARE_PROJ(f32_large)
CDSDP_DECLARE_PROJ(f64_small)
CDSDP_DECLARE_PROJ(f64_large)
#undef CDSDP_DECLARE_PROJ

// Thread-block-per-clique kernels, instantiated in proj_cta_{f32a,f32b,f32c,f64a,f64b}.cu
// (padded orders 36..48, 52..64, 96..128 in float; 36..48, 52..64 in double).
#define CDSDP_DECLARE_CTA(SUF)                                                                                  \
    cudaError_t launch_proj_cta_##SUF(int S, int form, const Dev& d, const int* list, int nlist,               \
                                      const ProjArgs& pa, const FinishArgs& fa, cudaStream_t st);                \
    cudaError_t launch_proj_cta_standalone_##SUF(int S, int p, const int* off, const int* size, const void* W, \
                                                 void* X, int max_sweeps, int variant, cudaStream_t st);
CDSDP_DECLARE_CTA(f32a)
CDSDP_DECLARE_CTA(f32b)
CDSDP_DECLARE_CTA(f32c)
CDSDP_DECLARE_CTA(f64a)
CDSDP_DECLARE_CTA(f64b)
#undef CDSDP_DECLARE_CTA

inline cudaError_t launch_proj_cta(bool fp32, int form, int cls, const Dev& d, const int* list, int nlist,
                                   const ProjArgs& pa, const FinishArgs& fa, cudaStream_t st) {
    const int S = kProjClasses[cls];
    if (fp32)
        return S <= 48 ? launch_proj_cta_f32a(S, form, d, list, nlist, pa, fa, st)
                       : (S <= 64 ? launch_proj_cta_f32b(S, form, d, list, nlist, pa, fa, st)
                                  : launch_proj_cta_f32c(S, form, d, list, nlist, pa, fa, st));
    return S <= 48 ? launch_proj_cta_f64a(S, form, d, list, nlist, pa, fa, st)
                   : launch_proj_cta_f64b(S, form, d, list, nlist, pa, fa, st);
}
inline cudaError_t launch_proj_cta_standalone(bool fp32, int cls, int p, const int* off, const int* size,
                                              const void* W, void* X, int max_sweeps, cudaStream_t st) {
    const int S = kProjClasses[cls];
    if (fp32)
        return S <= 48 ? launch_proj_cta_standalone_f32a(S, p, off, size, W, X, max_sweeps, 0, st)
                       : (S <= 64 ? launch_proj_cta_standalone_f32b(S, p, off, size, W, X, max_sweeps, 0, st)
                                  : launch_proj_cta_standalone_f32c(S, p, off, size, W, X, max_sweeps, 0, st));
    return S <= 48 ? launch_proj_cta_standalone_f64a(S, p, off, size, W, X, max_sweeps, 0, st)
                   : launch_proj_cta_standalone_f64b(S, p, off, size, W, X, max_sweeps, 0, st);
}

inline cudaError_t launch_proj_f32(int form, int cls, const Dev& d, const int* list, int nlist, const ProjArgs& pa,
                                   const FinishArgs& fa, cudaStream_t st) {
    if (kProjClasses[cls] > kMaxWarpOrder) return launch_proj_cta(true, form, cls, d, list, nlist, pa, fa, st);
    return kProjClasses[cls] <= 16 ? launch_proj_f32_small(form, cls, d, list, nlist, pa, fa, st)
                                   : launch_proj_f32_large(form, cls, d, list, nlist, pa, fa, st);
}
inline cudaError_t launch_proj_f64(int form, int cls, const Dev& d, const int* list, int nlist, const ProjArgs& pa,
                                   const FinishArgs& fa, cudaStream_t st) {
    if (kProjClasses[cls] > kMaxWarpOrder) return launch_proj_cta(false, form, cls, d, list, nlist, pa, fa, st);
    return kProjClasses[cls] <= 16 ? launch_proj_f64_small(form, cls, d, list, nlist, pa, fa, st)
                                   : launch_proj_f64_large(form, cls, d, list, nlist, pa, fa, st);
}
// grid of one projection launch (rows it writes in the partial table)
inline int proj_launch_grid(int cls, int nlist, bool fp32, int warps_div = 1) {
    const int S = kProjClasses[cls];
    if (S > kMaxWarpOrder) return proj_cta_grid(nlist);
    const int G = 32 / proj_lanes(S);
    return proj_shape((nlist + G - 1) / G, std::max(1, proj_max_warps(S, fp32) / std::max(1, warps_div))).grid;
}
inline cudaError_t launch_proj_standalone_f32(int cls, int p, const int* off, const int* size, const void* W, void* X,
                                              void* eig, const int* voff, void* V, const int* vvoff, double tolrel,
                                              int max_sweeps, cudaStream_t st) {
    if (kProjClasses[cls] > kMaxWarpOrder) return launch_proj_cta_standalone(true, cls, p, off, size, W, X, max_sweeps, st);
    return kProjClasses[cls] <= 16
               ? launch_proj_standalone_f32_small(cls, p, off, size, W, X, eig, voff, V, vvoff, tolrel, max_sweeps, st)
               : launch_proj_standalone_f32_large(cls, p, off, size, W, X, eig, voff, V, vvoff, tolrel, max_sweeps, st);
}
inline cudaError_t launch_proj_standalone_f64(int cls, int p, const int* off, const int* size, const void* W, void* X,
                                              void* eig, const int* voff, void* V, const int* vvoff, double tolrel,
                                              int max_sweeps, cudaStream_t st) {
    if (kProjClasses[cls] > kMaxWarpOrder) return launch_proj_cta_standalone(false, cls, p, off, size, W, X, max_sweeps, st);
    return kProjClasses[cls] <= 16
               ? launch_proj_standalone_f64_small(cls, p, off, size, W, X, eig, voff, V, vvoff, tolrel, max_sweeps, st)
               : launch_proj_standalone_f64_large(cls, p, off, size, W, X, eig, voff, V, vvoff, tolrel, max_sweeps, st);
}

}  // namespace cdsdp_dev
