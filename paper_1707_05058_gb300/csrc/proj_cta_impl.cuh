// CTA-per-clique projection kernels (orders 33..128 in float32, 33..64 in
// float64): instantiations and launchers.  Included once per translation unit
// with CTA_T (element type), CTA_SUFFIX (name suffix) and CTA_SIZES (X-macro
// list of the padded orders instantiated there) defined.
#include <algorithm>

#include "jacobi_cta.cuh"
#include "proj_launch.h"

namespace cdsdp_dev {
namespace {

template <typename T, int S, int FORM, int VARIANT>
cudaError_t launch_cta_v(const Dev& d, const int* list, int nlist, const ProjArgs& pa_in, const FinishArgs& fa,
                         const int* off, const int* size, const void* W, void* X, int max_sweeps, cudaStream_t st) {
    using Pick = CTAPick<T, S, VARIANT>;
    const size_t smem = Pick::type::bytes;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_project_cta<T, S, FORM, VARIANT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // as much shared memory as the SM offers, so that the register limit
        // decides how many cliques share an SM
        e = cudaFuncSetAttribute(k_project_cta<T, S, FORM, VARIANT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    ProjArgs pa = pa_in;
    pa.tolrel = jacobi_tolrel(S, sizeof(T) == 4);
    if (FORM == 3) pa.max_sweeps = max_sweeps;
    k_project_cta<T, S, FORM, VARIANT><<<proj_cta_grid(nlist), Pick::threads, smem, st>>>(d, list, nlist, pa, fa, off,
                                                                                         size, (const T*)W, (T*)X);
    return cudaGetLastError();
}

// pa.cta_variant = 1 selects variant 1 (V in registers) for float32 orders 36..64.
template <typename T, int S, int FORM>
cudaError_t launch_cta(const Dev& d, const int* list, int nlist, const ProjArgs& pa, const FinishArgs& fa,
                       const int* off, const int* size, const void* W, void* X, int max_sweeps, cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4 && S >= 36 && S <= 64) {
        if (pa.cta_variant == 1)
            return launch_cta_v<T, S, FORM, 1>(d, list, nlist, pa, fa, off, size, W, X, max_sweeps, st);
    }
    return launch_cta_v<T, S, FORM, 0>(d, list, nlist, pa, fa, off, size, W, X, max_sweeps, st);
}

template <typename T, int S>
cudaError_t launch_cta_form(int form, const Dev& d, const int* list, int nlist, const ProjArgs& pa,
                            const FinishArgs& fa, cudaStream_t st) {
    switch (form) {
        case 0: return launch_cta<T, S, 0>(d, list, nlist, pa, fa, nullptr, nullptr, nullptr, nullptr, 0, st);
        case 1: return launch_cta<T, S, 1>(d, list, nlist, pa, fa, nullptr, nullptr, nullptr, nullptr, 0, st);
        default: return launch_cta<T, S, 2>(d, list, nlist, pa, fa, nullptr, nullptr, nullptr, nullptr, 0, st);
    }
}

}  // namespace

cudaError_t CTA_SUFFIX(launch_proj_cta)(int S, int form, const Dev& d, const int* list, int nlist,
                                        const ProjArgs& pa, const FinishArgs& fa, cudaStream_t st) {
    switch (S) {
#define CTA_CASE(N) \
    case N: return launch_cta_form<CTA_T, N>(form, d, list, nlist, pa, fa, st);
        CTA_SIZES(CTA_CASE)
#undef CTA_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t CTA_SUFFIX(launch_proj_cta_standalone)(int S, int p, const int* off, const int* size, const void* W,
                                                   void* X, int max_sweeps, int variant, cudaStream_t st) {
    Dev d{};
    ProjArgs pa{};
    FinishArgs fa{};
    pa.restart = 1;
    pa.cta_variant = variant;
    switch (S) {
#define CTA_CASE(N) \
    case N: return launch_cta<CTA_T, N, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
        CTA_SIZES(CTA_CASE)
#undef CTA_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace cdsdp_dev
