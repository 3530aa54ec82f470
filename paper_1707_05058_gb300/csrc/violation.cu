// PSD-violation measure of Section 7.2 (Eq. PSD-violation) of arXiv 1707.05058:
//   alpha = -min{0, lambda_min[mat(H_1 x)], ..., lambda_min[mat(H_p x)]}
// over a batch of lower-packed blocks, in one kernel: one warp per block runs
// the Jacobi eigensolver of jacobi.cuh, each thread block writes its minimum
// eigenvalue to scratch, and the last thread block to finish (an atomic
// counter in scratch) reduces those partials in a fixed order and writes alpha.
// A block whose order lies outside 1..max_size is not a valid input: its
// thread block writes NaN as its partial, so alpha comes out NaN.
#include <cuda_runtime.h>

#include <algorithm>

#include "cdsdp_internal.h"
#include "jacobi.cuh"
#include "proj_launch.h"

using namespace cdsdp_dev;

namespace {

constexpr int kViolWarps = 4;  // warps (blocks of the batch) per thread block

// Scratch layout: [0, 256) counter (unsigned int), then one double per thread block.
inline size_t violation_scratch_bytes(int p) {
    const size_t grid = (size_t)std::max(1, (p + kViolWarps - 1) / kViolWarps);
    return 256 + grid * sizeof(double);
}

template <typename T, int S>
__global__ void __launch_bounds__(32 * kViolWarps) k_psd_violation(int p, const int* __restrict__ off_arr,
                                                                    const int* __restrict__ size_arr,
                                                                    const T* __restrict__ W, int max_size,
                                                                    double tolrel, int max_sweeps, unsigned char* scratch,
                                                                    double* alpha_out) {
    using J = BLJacobi<T, S>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double wmin[kViolWarps];
    __shared__ bool last;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
    double* partial = reinterpret_cast<double*>(scratch + 256);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    J jac;
    jac.bind(smem + warp * J::bytes, lane);
    double lmin = 0.0;  // min{0, ...}: start from 0
    bool bad = false;   // an order outside 1..max_size (max_size <= S)
    const int k = blockIdx.x * kViolWarps + warp;
    if (k < p) {
        const int s = size_arr[k];
        bad = s < 1 || s > max_size;
        if (!bad) {  // warp-uniform
            const int off = off_arr[k], npk = s * (s + 1) / 2;
            jac.clear(lane);
            T nrm = T(0);
            for (int f = lane; f < npk; f += 32) {
                const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
                const T w = W[off + f];
                jac.put(a, b, w);
                nrm += (a == b ? T(1) : T(2)) * w * w;
            }
            nrm = warp_sum(nrm);
            __syncwarp();
            jac.run(T(tolrel) * sqrt(nrm), max_sweeps, lane);
            double l = (lane < s) ? double(jac.X[lane * J::LDA + lane]) : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
            lmin = fmin(0.0, l);
        }
    }
    if (lane == 0) wmin[warp] = bad ? __longlong_as_double(0x7ff8000000000000LL) : lmin;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        bool nan = false;
        for (int w = 0; w < kViolWarps; ++w) {
            nan = nan || isnan(wmin[w]);
            m = fmin(m, wmin[w]);
        }
        partial[blockIdx.x] = nan ? __longlong_as_double(0x7ff8000000000000LL) : m;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {  // the final reduction, in a fixed order (fmin drops NaN, so it is counted apart)
        __threadfence();
        double m = 0.0;
        int nan = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            const double v = ((volatile double*)partial)[b];
            nan |= isnan(v) ? 1 : 0;
            m = fmin(m, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
            nan |= __shfl_xor_sync(0xffffffffu, nan, o);
        }
        if (lane == 0) wmin[warp] = nan ? __longlong_as_double(0x7ff8000000000000LL) : m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double mm = 0.0;
            bool any_nan = false;
            for (int w = 0; w < kViolWarps; ++w) {
                any_nan = any_nan || isnan(wmin[w]);
                mm = fmin(mm, wmin[w]);
            }
            *alpha_out = any_nan ? __longlong_as_double(0x7ff8000000000000LL) : -mm;
            *counter = 0u;
        }
    }
}

// Jacobi threshold: jacobi_tolrel, the same as the projection kernels'.
template <typename T, int S>
cudaError_t launch_violation(int p, const int* off, const int* size, int max_size, const void* W, int max_sweeps,
                             unsigned char* scratch, double* alpha, cudaStream_t st) {
    const size_t smem = kViolWarps * BLJacobi<T, S>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k_psd_violation<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, (p + kViolWarps - 1) / kViolWarps);
    k_psd_violation<T, S><<<grid, 32 * kViolWarps, smem, st>>>(p, off, size, (const T*)W, max_size,
                                                              jacobi_tolrel(S, sizeof(T) == 4), max_sweeps, scratch,
                                                              alpha);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_violation(int cls, int p, const int* off, const int* size, int max_size, const void* W,
                               int max_sweeps, unsigned char* scratch, double* alpha, cudaStream_t st) {
    switch (kProjClasses[cls]) {
        case 2: return launch_violation<T, 2>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 4: return launch_violation<T, 4>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 6: return launch_violation<T, 6>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 8: return launch_violation<T, 8>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 10: return launch_violation<T, 10>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 12: return launch_violation<T, 12>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 14: return launch_violation<T, 14>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 16: return launch_violation<T, 16>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 20: return launch_violation<T, 20>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 24: return launch_violation<T, 24>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 28: return launch_violation<T, 28>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        case 32: return launch_violation<T, 32>(p, off, size, max_size, W, max_sweeps, scratch, alpha, st);
        default: return cudaErrorInvalidValue;  // orders above 32 are not served by this entry point
    }
}

// Shared body of the entry points: validate, clear the counter, launch.
int run_violation(int p, const int* d_off, const int* d_size, int max_size, const void* d_W, int precision,
                  int max_sweeps, unsigned char* scratch, double* d_alpha, cudaStream_t st) {
    const int cls = proj_class_of(max_size);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) { cudaGetLastError(); return CDSDP_ERR_CUDA; }
    if (precision == CDSDP_FP64)
        e = dispatch_violation<double>(cls, p, d_off, d_size, max_size, d_W, max_sweeps, scratch, d_alpha, st);
    else
        e = dispatch_violation<float>(cls, p, d_off, d_size, max_size, d_W, max_sweeps, scratch, d_alpha, st);
    if (e != cudaSuccess) { cudaGetLastError(); return CDSDP_ERR_CUDA; }
    return CDSDP_SOLVED;
}

int check_violation_args(int p, const int* d_off, const int* d_size, int max_size, const void* d_W, int precision,
                         int max_sweeps, const double* d_alpha) {
    if (p < 1 || max_size < 1 || max_size > 32 || max_sweeps < 1) return CDSDP_ERR_ARG;
    if (!d_off || !d_size || !d_W || !d_alpha) return CDSDP_ERR_ARG;
    if (precision != CDSDP_FP32_PROJECTION && precision != CDSDP_FP64) return CDSDP_ERR_ARG;
    return CDSDP_SOLVED;
}

}  // namespace

extern "C" {

size_t cdsdp_psd_violation_scratch_bytes(int p) { return violation_scratch_bytes(p); }

int cdsdp_psd_violation(int p, const int* d_off, const int* d_size, int max_size, const void* d_W, int precision,
                        int max_sweeps, void* d_scratch, size_t scratch_bytes, double* d_alpha, void* stream) {
    int rc = check_violation_args(p, d_off, d_size, max_size, d_W, precision, max_sweeps, d_alpha);
    if (rc != CDSDP_SOLVED) return rc;
    if (!d_scratch || reinterpret_cast<uintptr_t>(d_scratch) % 256) return CDSDP_ERR_ARG;
    if (scratch_bytes < violation_scratch_bytes(p)) return CDSDP_ERR_NOMEM;
    return run_violation(p, d_off, d_size, max_size, d_W, precision, max_sweeps, (unsigned char*)d_scratch, d_alpha,
                         (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Variant for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need this measure:
// code running inside a framework whose caching allocator owns the device
// memory (a raw cudaMalloc there fragments or overcommits the pool it
// manages), a plugin whose host hands it only input and output buffers, or a
// real-time loop that forbids the latency and possible failure of an
// allocation.  For them the scratch lives in a fixed array in the library's
// device image, held on every GPU that loads the library until the process
// exits.  Its device address is looked up once per device and kept for the
// life of the process, so the entry point must not be used on a device after
// cudaDeviceReset (the module is loaded again there, at a new address).
#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;  // 1 MiB: counter + 131040 per-block minima
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_violation_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_violation_scratch on the current device (the host-side
// name is only a stand-in, never a device pointer).  Looked up once per device.
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CDSDP_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return CDSDP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_violation_scratch);
        if (e != cudaSuccess || !ptr) { cudaGetLastError(); return CDSDP_ERR_CUDA; }
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return CDSDP_SOLVED;
}

}  // namespace

extern "C" int cdsdp_psd_violation_noalloc(int p, const int* d_off, const int* d_size, int max_size, const void* d_W,
                                           int precision, int max_sweeps, double* d_alpha, void* stream) {
    int rc = check_violation_args(p, d_off, d_size, max_size, d_W, precision, max_sweeps, d_alpha);
    if (rc != CDSDP_SOLVED) return rc;
    if (violation_scratch_bytes(p) > kNoAllocScratchBytes) return CDSDP_ERR_UNSUPPORTED;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != CDSDP_SOLVED) return rc;
    return run_violation(p, d_off, d_size, max_size, d_W, precision, max_sweeps, (unsigned char*)scratch, d_alpha,
                         (cudaStream_t)stream);
}
