// Large-order PSD projection (order 129 and above) by the Newton-Schulz sign
// iteration on the tensor cores (see large.cuh for the method), and the C ABI
// entry point that projects a batch of packed blocks this way.
//
// Product kernel (one CTA per 128 x 128 output tile, 128 threads):
//  * thread 0 of warp 0 streams 128 x 32 float tiles of A_hi, A_lo, B_hi, B_lo
//    into a 3-stage shared-memory ring with TMA (cp.async.bulk.tensor, 128-byte
//    swizzle), one mbarrier per stage with the transaction byte count;
//  * thread 0 of warp 1 issues tcgen05.mma kind::tf32 (M = N = 128, K = 8):
//    three products per K step into one float32 accumulator in tensor memory,
//    and frees a stage with tcgen05.commit on that stage's "empty" mbarrier;
//  * all four warps read the accumulator back (tcgen05.ld 32x32b, one row per
//    thread), apply D = alpha acc + beta C, split D into (tf32(D), D - tf32(D))
//    and store the tile and its mirror (the products are symmetric).
// Every wait is bounded (about a second of clock cycles): on a timeout the
// kernel records an error code, lets its in-flight copies land (bounded
// again), frees its tensor memory and returns; the host reports
// CDSDP_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "cdsdp_internal.h"
#include "large.cuh"
#include "large_launch.h"

namespace cdsdp_large {
namespace {

constexpr long long kSpinCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity` to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kSpinCycles) return false;
    return true;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    // leading byte offset 0: one swizzle atom spans the whole K extent of a tile
    d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1u << 46;             // descriptor version of the tcgen05 family
    d |= (uint64_t)2u << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor: D float32, A and B tf32, both K-major, N = M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTile >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kGemmThreads, 1) k_tf32x3_sym(GemmArgs g) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);  // full[3], empty[3], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* issued_slot = reinterpret_cast<int*>(tmem_slot + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Tile t = g.tiles[blockIdx.x];
    const Block B = g.blocks[t.blk];
    const int nk = B.S / kChunk;
    const CUtensorMap* mAh = reinterpret_cast<const CUtensorMap*>(g.mapA_hi) + t.blk;
    const CUtensorMap* mAl = reinterpret_cast<const CUtensorMap*>(g.mapA_lo) + t.blk;
    const CUtensorMap* mBh = reinterpret_cast<const CUtensorMap*>(g.mapB_hi) + t.blk;
    const CUtensorMap* mBl = reinterpret_cast<const CUtensorMap*>(g.mapB_lo) + t.blk;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), done = smem_u32(bars + 2 * kStages);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *issued_slot = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {  // TMA producer
        int issued = 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages;
            if (kc >= kStages && !mbar_wait(empty0 + 8 * s, ((kc / kStages) - 1) & 1)) {
                *abort_flag = 1;
                atomicExch(g.err, 1);
                break;
            }
            if (*abort_flag) break;
            const uint32_t base = smem_u32(smem + s * kStageBytes);
            mbar_expect_tx(full0 + 8 * s, kStageBytes);
            const int x = kc * kChunk;
            tma_load_2d(base, mAh, x, t.ti * kTile, full0 + 8 * s);
            tma_load_2d(base + kTileBytes, mAl, x, t.ti * kTile, full0 + 8 * s);
            tma_load_2d(base + 2 * kTileBytes, mBh, x, t.tj * kTile, full0 + 8 * s);
            tma_load_2d(base + 3 * kTileBytes, mBl, x, t.tj * kTile, full0 + 8 * s);
            ++issued;
        }
        *issued_slot = issued;
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages;
            if (!mbar_wait(full0 + 8 * s, (kc / kStages) & 1)) {
                *abort_flag = 1;
                atomicExch(g.err, 2);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
            for (int k = 0; k < kChunk / 8; ++k) {
                const uint64_t ah = sdesc(base + 32 * k), al = sdesc(base + kTileBytes + 32 * k);
                const uint64_t bh = sdesc(base + 2 * kTileBytes + 32 * k), bl = sdesc(base + 3 * kTileBytes + 32 * k);
                mma_tf32(tmem, ah, bh, (kc | k) != 0 ? 1u : 0u);
                mma_tf32(tmem, ah, bl, 1u);
                mma_tf32(tmem, al, bh, 1u);
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);  // completes once every MMA issued above has finished
    }
    __syncwarp();

    // epilogue: thread (warp w, lane l) owns row 32 w + l of the tile
    bool ok = mbar_wait(done, 0);
    if (!ok) atomicExch(g.err, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    if (ok && !*abort_flag) {
        // Every stored matrix is kept exactly symmetric: an off-diagonal tile is
        // stored with its mirror, a diagonal tile only from its lower triangle
        // (mirrored).  The products are symmetric only up to rounding, and the
        // B operand enters transposed, so an antisymmetric remainder left in an
        // iterate would be amplified by the sign iteration near eigenvalue 0.
        const int S = B.S;
        const int r = 32 * warp + lane;
        const bool diag = t.ti == t.tj;
        const long long gr = (long long)t.ti * kTile + r;
        const float* Ch = g.C_hi ? g.C_hi + B.off : nullptr;
        const float* Cl = g.C_lo ? g.C_lo + B.off : nullptr;
        float* Dh = g.D_hi + B.off;
        float* Dl = g.D_lo ? g.D_lo + B.off : nullptr;
#pragma unroll 1
        for (int cc = 0; cc < kTile / 32; ++cc) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * cc), v);
            const long long gc0 = (long long)t.tj * kTile + 32 * cc;
            float hi[32], lo[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                // C is symmetric: read its entry (gc, gr), consecutive over the warp's rows
                float c = 0.f;
                if (Ch) c = Ch[(gc0 + j) * S + gr] + Cl[(gc0 + j) * S + gr];
                const float d = g.alpha * __uint_as_float(v[j]) + g.beta * c;
                hi[j] = Dl ? tf32_round(d) : d;
                lo[j] = d - hi[j];
            }
            if (!diag) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {  // mirror (gc, gr): coalesced over the warp
                    const long long mi = (gc0 + j) * S + gr;
                    Dh[mi] = hi[j];
                    if (Dl) Dl[mi] = lo[j];
                }
                float4* dh4 = reinterpret_cast<float4*>(Dh + gr * S + gc0);
#pragma unroll
                for (int q = 0; q < 8; ++q) dh4[q] = make_float4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
                if (Dl) {
                    float4* dl4 = reinterpret_cast<float4*>(Dl + gr * S + gc0);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dl4[q] = make_float4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int lc = 32 * cc + j;  // column within the tile
                    if (lc > r) continue;        // upper triangle: written as the mirror of (lc, r)
                    Dh[gr * S + gc0 + j] = hi[j];
                    if (Dl) Dl[gr * S + gc0 + j] = lo[j];
                    if (lc < r) {
                        Dh[(gc0 + j) * S + gr] = hi[j];
                        if (Dl) Dl[(gc0 + j) * S + gr] = lo[j];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // after an abort, let the copies already issued land before the CTA exits
    if (*abort_flag && warp == 0 && lane == 0) {
        const int issued = *issued_slot;
        for (int kc = max(0, issued - kStages); kc < issued; ++kc)
            (void)mbar_wait(full0 + 8 * (kc % kStages), (kc / kStages) & 1);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTile) : "memory");
    }
}

// ---- element-wise kernels ---------------------------------------------------

// (a, b), a >= b, of packed (lower, column-major) element f of an s x s block.
__device__ __forceinline__ void packed_rc(long long f, int s, int& a, int& b) {
    const double t = 2.0 * s + 1.0;
    int bb = (int)((t - sqrt(t * t - 8.0 * (double)f)) * 0.5);
    bb = max(0, min(bb, s - 1));
    while (bb > 0 && (long long)bb * (2 * s - bb + 1) / 2 > f) --bb;
    while (bb + 1 < s && (long long)(bb + 1) * (2 * s - bb) / 2 <= f) ++bb;
    b = bb;
    a = bb + (int)(f - (long long)bb * (2 * s - bb + 1) / 2);
}

// Dense symmetric W (hi, lo) of block k from its packed lower values (grid.y = block).
__global__ void k_dense_from_packed(const Block* __restrict__ blocks, const long long* __restrict__ poff,
                                    const float* __restrict__ Wp, float* Wh, float* Wl) {
    const int k = blockIdx.y;
    const Block B = blocks[k];
    const long long npk = (long long)B.s * (B.s + 1) / 2;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npk; f += (long long)gridDim.x * blockDim.x) {
        int a, b;
        packed_rc(f, B.s, a, b);
        const float w = Wp[poff[k] + f];
        const float h = tf32_round(w), l = w - h;
        Wh[B.off + (long long)a * B.S + b] = h;
        Wl[B.off + (long long)a * B.S + b] = l;
        Wh[B.off + (long long)b * B.S + a] = h;
        Wl[B.off + (long long)b * B.S + a] = l;
    }
}

// Partial sums of ||W||_F^2 over fixed chunks of each block's dense rows
// (deterministic: one partial per (block, chunk), summed in order below).
constexpr int kNormChunkRows = 32;
__global__ void k_norm_partials(const Block* __restrict__ blocks, const int* __restrict__ chunk_off,
                                const float* __restrict__ Wh, const float* __restrict__ Wl, double* partial) {
    const int k = blockIdx.y;
    const Block B = blocks[k];
    const int nchunk = chunk_off[k + 1] - chunk_off[k];
    if ((int)blockIdx.x >= nchunk) return;
    const long long r0 = (long long)blockIdx.x * kNormChunkRows;
    const long long e0 = B.off + r0 * B.S;
    const long long ne = (long long)min((long long)kNormChunkRows, B.S - r0) * B.S;
    double acc = 0.0;
    for (long long e = threadIdx.x; e < ne; e += blockDim.x) {
        const double w = (double)Wh[e0 + e] + (double)Wl[e0 + e];
        acc += w * w;
    }
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        partial[chunk_off[k] + blockIdx.x] = s;
    }
}

// X_0 = W / ||W||_F as (hi, lo); scale[k] = ||W||_F (grid.y = block).
__global__ void k_scale_start(const Block* __restrict__ blocks, const int* __restrict__ chunk_off,
                              const double* __restrict__ partial, const float* __restrict__ Wh,
                              const float* __restrict__ Wl, float* Xh, float* Xl, double* scale) {
    const int k = blockIdx.y;
    const Block B = blocks[k];
    double s2 = 0.0;
    for (int c = chunk_off[k]; c < chunk_off[k + 1]; ++c) s2 += partial[c];
    const double nrm = sqrt(s2);
    if (blockIdx.x == 0 && threadIdx.x == 0) scale[k] = nrm;
    const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
    const long long ne = (long long)B.S * B.S;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const float x = (Wh[B.off + e] + Wl[B.off + e]) * inv;
        const float h = tf32_round(x);
        Xh[B.off + e] = h;
        Xl[B.off + e] = x - h;
    }
}

// Packed lower values of the dense P (grid.y = block).
__global__ void k_packed_from_dense(const Block* __restrict__ blocks, const long long* __restrict__ poff,
                                    const float* __restrict__ P, float* Xp) {
    const int k = blockIdx.y;
    const Block B = blocks[k];
    const long long npk = (long long)B.s * (B.s + 1) / 2;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npk; f += (long long)gridDim.x * blockDim.x) {
        int a, b;
        packed_rc(f, B.s, a, b);
        Xp[poff[k] + f] = P[B.off + (long long)a * B.S + b];
    }
}

// ---- host side ----------------------------------------------------------------

std::mutex g_encode_mutex;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool get_encode() {
    std::lock_guard<std::mutex> lock(g_encode_mutex);
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return true;
}

bool encode_map(CUtensorMap* m, const float* base, int S) {
    const cuuint64_t dims[2] = {(cuuint64_t)S, (cuuint64_t)S};
    const cuuint64_t strides[1] = {(cuuint64_t)S * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)kTile};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// ---- layout of the iteration's device memory ------------------------------------

NsLayout ns_layout(const std::vector<int>& sizes) {
    NsLayout L;
    L.nb = (int)sizes.size();
    long long off = 0;
    int chunks = 0;
    L.chunk_off.push_back(0);
    for (int s : sizes) {
        Block b;
        b.s = s;
        b.S = (s + kTile - 1) / kTile * kTile;
        b.off = off;
        off += (long long)b.S * b.S;
        L.blocks.push_back(b);
        const int nt = b.S / kTile;
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j <= i; ++j) L.tiles.push_back(Tile{(int)L.blocks.size() - 1, i, j, 0});
        chunks += (b.S + kNormChunkRows - 1) / kNormChunkRows;
        L.chunk_off.push_back(chunks);
        L.max_S = std::max(L.max_S, b.S);
        const int nu = (int)(((long long)s * (s + 1) / 2 + kUpdChunk - 1) / kUpdChunk);
        if (L.upd_off.empty()) L.upd_off.push_back(0);
        L.upd_off.push_back(L.upd_off.back() + nu);
        L.max_upd = std::max(L.max_upd, nu);
    }
    if (L.upd_off.empty()) L.upd_off.push_back(0);
    L.elems = off;
    size_t o = 0;
    L.o_err = o; o = up256(o + 16);
    L.o_maps = o; o = up256(o + sizeof(CUtensorMap) * 2 * NBUF * (size_t)std::max(1, L.nb));
    L.o_tiles = o; o = up256(o + sizeof(Tile) * std::max<size_t>(1, L.tiles.size()));
    L.o_blocks = o; o = up256(o + sizeof(Block) * std::max(1, L.nb));
    L.o_chunk = o; o = up256(o + sizeof(int) * (L.nb + 1));
    L.o_partial = o; o = up256(o + sizeof(double) * std::max(1, chunks));
    L.o_scale = o; o = up256(o + sizeof(double) * std::max(1, L.nb));
    L.o_poff = o; o = up256(o + sizeof(long long) * std::max(1, L.nb));
    L.o_list = o; o = up256(o + sizeof(int) * std::max(1, L.nb));
    L.o_upd = o; o = up256(o + sizeof(int) * (L.nb + 1));
    L.o_updpart = o; o = up256(o + sizeof(double) * 8 * std::max(1, L.upd_off.back()));
    for (int b = 0; b < 2 * NBUF; ++b) {
        L.o_buf[b] = o;
        o = up256(o + (size_t)off * sizeof(float));
    }
    L.bytes = o;
    return L;
}

// Host image of the tables (tensor maps, tiles, blocks, chunk offsets, packed
// offsets) for device memory at `base`; false when the tensor-map encoder is
// unavailable or refuses a map.
bool ns_tables(const NsLayout& L, unsigned char* base, const std::vector<long long>& poff,
               const std::vector<int>& list, std::vector<unsigned char>& img) {
    if (!get_encode()) return false;
    img.assign(L.o_buf[0], 0);
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(img.data() + L.o_maps);
    for (int buf = 0; buf < 2 * NBUF; ++buf)
        for (int k = 0; k < L.nb; ++k) {
            const float* p = reinterpret_cast<const float*>(base + L.o_buf[buf]) + L.blocks[k].off;
            if (!encode_map(&maps[buf * L.nb + k], p, L.blocks[k].S)) return false;
        }
    std::memcpy(img.data() + L.o_tiles, L.tiles.data(), sizeof(Tile) * L.tiles.size());
    std::memcpy(img.data() + L.o_blocks, L.blocks.data(), sizeof(Block) * L.blocks.size());
    std::memcpy(img.data() + L.o_chunk, L.chunk_off.data(), sizeof(int) * L.chunk_off.size());
    std::memcpy(img.data() + L.o_poff, poff.data(), sizeof(long long) * poff.size());
    std::memcpy(img.data() + L.o_list, list.data(), sizeof(int) * list.size());
    std::memcpy(img.data() + L.o_upd, L.upd_off.data(), sizeof(int) * L.upd_off.size());
    return true;
}

namespace {

cudaError_t gemm(const NsLayout& L, unsigned char* base, int a, int bsrc, int c, int d, float alpha, float beta,
                 bool split, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tf32x3_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(base + L.o_maps);
    GemmArgs g;
    g.mapA_hi = maps + (2 * a) * L.nb;
    g.mapA_lo = maps + (2 * a + 1) * L.nb;
    g.mapB_hi = maps + (2 * bsrc) * L.nb;
    g.mapB_lo = maps + (2 * bsrc + 1) * L.nb;
    g.C_hi = c >= 0 ? reinterpret_cast<const float*>(base + L.o_buf[2 * c]) : nullptr;
    g.C_lo = c >= 0 ? reinterpret_cast<const float*>(base + L.o_buf[2 * c + 1]) : nullptr;
    g.D_hi = reinterpret_cast<float*>(base + L.o_buf[2 * d]);
    g.D_lo = split ? reinterpret_cast<float*>(base + L.o_buf[2 * d + 1]) : nullptr;
    g.blocks = reinterpret_cast<const Block*>(base + L.o_blocks);
    g.tiles = reinterpret_cast<const Tile*>(base + L.o_tiles);
    g.ntiles = (int)L.tiles.size();
    g.alpha = alpha;
    g.beta = beta;
    g.err = reinterpret_cast<int*>(base + L.o_err);
    k_tf32x3_sym<<<g.ntiles, kGemmThreads, kGemmSmem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace

// The sign iteration and P = (W + W X) / 2 on buffers already holding W
// (hi, lo) and X_0 (BUF_XA); P goes to BUF_X2 hi.
cudaError_t ns_iterate(const NsLayout& L, unsigned char* base, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    int x = BUF_XA, xn = BUF_XB;
    for (int i = 0; i < kPhase1 && e == cudaSuccess; ++i) {  // X <- a X + b X^3 + c X^5
        e = gemm(L, base, x, x, -1, BUF_X2, 1.f, 0.f, true, st);                          // X2 = X X
        if (e == cudaSuccess) e = gemm(L, base, BUF_X2, BUF_X2, BUF_X2, BUF_B, kPc, kPb, true, st);  // c X2 X2 + b X2
        if (e == cudaSuccess) e = gemm(L, base, x, BUF_B, x, xn, 1.f, kPa, true, st);     // X B + a X
        std::swap(x, xn);
    }
    for (int i = 0; i < kPhase2 && e == cudaSuccess; ++i) {  // X <- 1.5 X - 0.5 X^3
        e = gemm(L, base, x, x, -1, BUF_X2, 1.f, 0.f, true, st);
        if (e == cudaSuccess) e = gemm(L, base, x, BUF_X2, x, xn, -0.5f, 1.5f, true, st);
        std::swap(x, xn);
    }
    if (e == cudaSuccess) e = gemm(L, base, BUF_W, x, BUF_W, BUF_X2, 0.5f, 0.5f, false, st);  // P
    return e;
}

cudaError_t ns_scale_and_iterate(const NsLayout& L, unsigned char* base, cudaStream_t st) {
    const Block* blocks = reinterpret_cast<const Block*>(base + L.o_blocks);
    const int* chunk = reinterpret_cast<const int*>(base + L.o_chunk);
    const float* Wh = reinterpret_cast<const float*>(base + L.o_buf[2 * BUF_W]);
    const float* Wl = reinterpret_cast<const float*>(base + L.o_buf[2 * BUF_W + 1]);
    float* Xh = reinterpret_cast<float*>(base + L.o_buf[2 * BUF_XA]);
    float* Xl = reinterpret_cast<float*>(base + L.o_buf[2 * BUF_XA + 1]);
    const int gx = std::min(1024, std::max(1, (int)(((long long)L.max_S * L.max_S / 2 + 255) / 256)));
    const int maxchunk = (L.max_S + kNormChunkRows - 1) / kNormChunkRows;
    k_norm_partials<<<dim3(maxchunk, L.nb), 256, 0, st>>>(blocks, chunk, Wh, Wl,
                                                         reinterpret_cast<double*>(base + L.o_partial));
    k_scale_start<<<dim3(gx, L.nb), 256, 0, st>>>(blocks, chunk, reinterpret_cast<const double*>(base + L.o_partial),
                                                  Wh, Wl, Xh, Xl, reinterpret_cast<double*>(base + L.o_scale));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = ns_iterate(L, base, st);
    return e;
}

cudaError_t ns_from_packed(const NsLayout& L, unsigned char* base, const float* Wp, cudaStream_t st) {
    const Block* blocks = reinterpret_cast<const Block*>(base + L.o_blocks);
    const long long* poff = reinterpret_cast<const long long*>(base + L.o_poff);
    float* Wh = reinterpret_cast<float*>(base + L.o_buf[2 * BUF_W]);
    float* Wl = reinterpret_cast<float*>(base + L.o_buf[2 * BUF_W + 1]);
    cudaError_t e = cudaMemsetAsync(base + L.o_buf[2 * BUF_W], 0, 2 * (size_t)L.elems * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const int gx = std::min(1024, std::max(1, (int)(((long long)L.max_S * L.max_S / 2 + 255) / 256)));
    k_dense_from_packed<<<dim3(gx, L.nb), 256, 0, st>>>(blocks, poff, Wp, Wh, Wl);
    return cudaGetLastError();
}

cudaError_t ns_to_packed(const NsLayout& L, unsigned char* base, float* Xp, cudaStream_t st) {
    const int gx = std::min(1024, std::max(1, (int)(((long long)L.max_S * L.max_S / 2 + 255) / 256)));
    k_packed_from_dense<<<dim3(gx, L.nb), 256, 0, st>>>(reinterpret_cast<const Block*>(base + L.o_blocks),
                                                        reinterpret_cast<const long long*>(base + L.o_poff),
                                                        reinterpret_cast<const float*>(base + L.o_buf[2 * BUF_X2]),
                                                        Xp);
    return cudaGetLastError();
}

}  // namespace cdsdp_large

using namespace cdsdp_large;

extern "C" {

int cdsdp_psd_project_large_bytes(int p, const int* h_size, size_t* bytes) {
    if (p < 1 || !h_size || !bytes) return CDSDP_ERR_ARG;
    std::vector<int> sizes(h_size, h_size + p);
    for (int s : sizes)
        if (s < 1 || s > kMaxLargeOrder) return CDSDP_ERR_ARG;
    *bytes = ns_layout(sizes).bytes;
    return CDSDP_SOLVED;
}

int cdsdp_psd_project_large(int p, const int* h_size, const long long* h_off, const float* d_W, float* d_X,
                            void* d_scratch, size_t scratch_bytes, void* stream) {
    if (p < 1 || !h_size || !h_off || !d_W || !d_X || !d_scratch) return CDSDP_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_scratch) % 256) return CDSDP_ERR_ARG;
    std::vector<int> sizes(h_size, h_size + p);
    for (int s : sizes)
        if (s < 1 || s > kMaxLargeOrder) return CDSDP_ERR_ARG;
    for (int k = 0; k < p; ++k)
        if (h_off[k] < 0) return CDSDP_ERR_ARG;
    try {
        const NsLayout L = ns_layout(sizes);
        if (scratch_bytes < L.bytes) return CDSDP_ERR_NOMEM;
        unsigned char* base = static_cast<unsigned char*>(d_scratch);
        std::vector<long long> poff(h_off, h_off + p);
        std::vector<int> list(p);
        for (int k = 0; k < p; ++k) list[k] = k;
        std::vector<unsigned char> img;
        if (!ns_tables(L, base, poff, list, img)) return CDSDP_ERR_CUDA;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (cudaMemcpyAsync(base, img.data(), img.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return CDSDP_ERR_CUDA;
        }
        cudaError_t e = ns_from_packed(L, base, d_W, st);
        if (e == cudaSuccess) e = ns_scale_and_iterate(L, base, st);
        if (e == cudaSuccess) e = ns_to_packed(L, base, d_X, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return CDSDP_ERR_CUDA;
        }
        int err = 0;
        if (cudaMemcpyAsync(&err, base + L.o_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return CDSDP_ERR_CUDA;
        }
        return err ? CDSDP_ERR_TIMEOUT : CDSDP_SOLVED;
    } catch (const std::exception&) {
        return CDSDP_ERR_NOMEM;
    }
}

}  // extern "C"
