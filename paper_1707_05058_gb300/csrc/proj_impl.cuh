// Dispatch from a size class to the projection kernel instantiations.
// Included once per precision with PROJ_T and PROJ_SUFFIX defined.
#include <algorithm>

#include "jacobi.cuh"
#include "proj_launch.h"

namespace cdsdp_dev {
namespace {

template <typename T, int S>
cudaError_t launch_form(int form, const Dev& d, const int* list, int nlist, const ProjArgs& pa_in,
                        const FinishArgs& fa, cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    constexpr int MW = proj_max_warps(S, sizeof(T) == 4);
    constexpr int LW = proj_lanes(S), G = 32 / LW;  // G cliques per warp
    using J = BLJacobi<T, S, LW>;
    const ProjShape sh = proj_shape((nlist + G - 1) / G, std::max(1, MW / std::max(1, pa_in.warps_div)));
    const size_t smem = (size_t)sh.wpb * G * J::bytes;
    const size_t smem_max = (size_t)MW * G * J::bytes;
    ProjArgs pa = pa_in;
    pa.tolrel = jacobi_tolrel(S, sizeof(T) == 4);
    static bool attr_done[3] = {false, false, false};  // per instantiation; setting twice is harmless
    cudaError_t e = cudaSuccess;
    if (form == 0) {
        if (!attr_done[0]) e = cudaFuncSetAttribute(k_project_primal<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e != cudaSuccess) return e;
        attr_done[0] = true;
        k_project_primal<T, S><<<sh.grid, 32 * sh.wpb, smem, st>>>(d, list, nlist, pa, fa);
    } else if (form == 1) {
        if (!attr_done[1]) e = cudaFuncSetAttribute(k_project_dual<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e != cudaSuccess) return e;
        attr_done[1] = true;
        k_project_dual<T, S><<<sh.grid, 32 * sh.wpb, smem, st>>>(d, list, nlist, pa);
    } else {
        if (!attr_done[2]) e = cudaFuncSetAttribute(k_project_hsde<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e != cudaSuccess) return e;
        attr_done[2] = true;
        k_project_hsde<T, S><<<sh.grid, 32 * sh.wpb, smem, st>>>(d, list, nlist, pa);
    }
    return cudaGetLastError();
}

template <typename T, int S>
cudaError_t launch_standalone(int p, const int* off, const int* size, const void* W, void* X, void* eig,
                              const int* voff, void* V, const int* vvoff, double tolrel, int max_sweeps,
                              cudaStream_t st) {
    const size_t smem = 4 * BLJacobi<T, S>::bytes;
    const int grid = std::max(1, std::min((p + 3) / 4, 152 * 64));
    cudaError_t e = cudaFuncSetAttribute(k_project_standalone<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_project_standalone<T, S><<<grid, 128, smem, st>>>(p, off, size, (const T*)W, (T*)X, (T*)eig, voff, (T*)V,
                                                        vvoff, jacobi_tolrel(S, sizeof(T) == 4), max_sweeps);
    return cudaGetLastError();
}

// PROJ_PART 0 instantiates orders 2..16, PROJ_PART 1 orders 20..32.
#if PROJ_PART == 0
#define CDSDP_CLASS_SWITCH(CALL)        \
    switch (kProjClasses[cls]) {        \
        case 2: return CALL(2);         \
        case 4: return CALL(4);         \
        case 6: return CALL(6);         \
        case 8: return CALL(8);         \
        case 10: return CALL(10);       \
        case 12: return CALL(12);       \
        case 14: return CALL(14);       \
        case 16: return CALL(16);       \
        default: return cudaErrorInvalidValue; \
    }
#else
#define CDSDP_CLASS_SWITCH(CALL)        \
    switch (kProjClasses[cls]) {        \
        case 20: return CALL(20);       \
        case 24: return CALL(24);       \
        case 28: return CALL(28);       \
        case 32: return CALL(32);       \
        default: return cudaErrorInvalidValue; \
    }
#endif

}  // namespace

cudaError_t PROJ_SUFFIX(launch_proj)(int form, int cls, const Dev& d, const int* list, int nlist, const ProjArgs& pa,
                                     const FinishArgs& fa, cudaStream_t st) {
#define CALL(S) launch_form<PROJ_T, S>(form, d, list, nlist, pa, fa, st)
    CDSDP_CLASS_SWITCH(CALL)
#undef CALL
}

cudaError_t PROJ_SUFFIX(launch_proj_standalone)(int cls, int p, const int* off, const int* size, const void* W,
                                                void* X, void* eig, const int* voff, void* V, const int* vvoff,
                                                double tolrel, int max_sweeps, cudaStream_t st) {
#define CALL(S) launch_standalone<PROJ_T, S>(p, off, size, W, X, eig, voff, V, vvoff, tolrel, max_sweeps, st)
    CDSDP_CLASS_SWITCH(CALL)
#undef CALL
}

}  // namespace cdsdp_dev
