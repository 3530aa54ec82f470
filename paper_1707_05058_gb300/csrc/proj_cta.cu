// CTA-per-clique projection kernels (orders 33..128 in float32, 33..64 in
// float64): instantiations and launchers.
#include <algorithm>

#include "jacobi_cta.cuh"
#include "proj_launch.h"

namespace cdsdp_dev {
namespace {

template <typename T, int S, int FORM>
cudaError_t launch_cta(const Dev& d, const int* list, int nlist, const ProjArgs& pa_in, const FinishArgs& fa,
                       const int* off, const int* size, const void* W, void* X, int max_sweeps, cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    const size_t smem = CTAJacobi<T, S>::bytes;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_project_cta<T, S, FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    ProjArgs pa = pa_in;
    pa.tolrel = jacobi_tolrel(S, sizeof(T) == 4);
    if (FORM == 3) pa.max_sweeps = max_sweeps;
    k_project_cta<T, S, FORM><<<proj_cta_grid(nlist), kCtaThreads, smem, st>>>(d, list, nlist, pa, fa, off, size,
                                                                               (const T*)W, (T*)X);
    return cudaGetLastError();
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

cudaError_t launch_proj_cta(bool fp32, int form, int cls, const Dev& d, const int* list, int nlist,
                            const ProjArgs& pa, const FinishArgs& fa, cudaStream_t st) {
    const int S = kProjClasses[cls];
    if (fp32) {
        switch (S) {
            case 48: return launch_cta_form<float, 48>(form, d, list, nlist, pa, fa, st);
            case 64: return launch_cta_form<float, 64>(form, d, list, nlist, pa, fa, st);
            case 96: return launch_cta_form<float, 96>(form, d, list, nlist, pa, fa, st);
            case 128: return launch_cta_form<float, 128>(form, d, list, nlist, pa, fa, st);
        }
    } else {
        switch (S) {
            case 48: return launch_cta_form<double, 48>(form, d, list, nlist, pa, fa, st);
            case 64: return launch_cta_form<double, 64>(form, d, list, nlist, pa, fa, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_proj_cta_standalone(bool fp32, int cls, int p, const int* off, const int* size, const void* W,
                                       void* X, int max_sweeps, cudaStream_t st) {
    const int S = kProjClasses[cls];
    Dev d{};
    ProjArgs pa{};
    FinishArgs fa{};
    pa.restart = 1;
    if (fp32) {
        switch (S) {
            case 48: return launch_cta<float, 48, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
            case 64: return launch_cta<float, 64, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
            case 96: return launch_cta<float, 96, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
            case 128: return launch_cta<float, 128, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
        }
    } else {
        switch (S) {
            case 48: return launch_cta<double, 48, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
            case 64: return launch_cta<double, 64, 3>(d, nullptr, p, pa, fa, off, size, W, X, max_sweeps, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace cdsdp_dev
