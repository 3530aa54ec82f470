// Host interface of the large-order projection (large.cu): layout of its
// device memory and the launch sequence.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "large.cuh"

namespace cdsdp_large {

// Largest clique order served (dense blocks of up to 8192 x 8192 floats).
constexpr int kMaxLargeOrder = 8192;
// Orders above this go to the sign iteration (the thread-block Jacobi serves up to it).
constexpr int kLargeFrom = 129;

// Packed entries per thread block of the gather and update kernels.
constexpr int kUpdChunk = 8192;

// Device memory of one batch of large blocks: tables, then 2 * NBUF dense
// float buffers (the (hi, lo) pairs of W, X_a, X_b, X^2, B), each holding
// every block at Block::off with row pitch Block::S.
struct NsLayout {
    int nb = 0;
    int max_S = 0;
    long long elems = 0;            // floats per buffer
    std::vector<Block> blocks;
    std::vector<Tile> tiles;        // lower output tiles of every block
    std::vector<int> chunk_off;     // row chunks of the norm reduction, per block
    std::vector<int> upd_off;       // packed-entry chunks of the gather / update, per block
    int max_upd = 0;                // most packed-entry chunks of one block
    size_t o_err = 0, o_maps = 0, o_tiles = 0, o_blocks = 0, o_chunk = 0, o_partial = 0, o_scale = 0, o_poff = 0;
    size_t o_list = 0, o_upd = 0, o_updpart = 0;
    size_t o_buf[2 * NBUF] = {0};
    size_t bytes = 0;
};

NsLayout ns_layout(const std::vector<int>& sizes);
// Host image of bytes [0, o_buf[0]) for device memory at `base`: tensor maps
// of every (buffer, block), tiles, blocks, chunk offsets, packed offsets and
// the block's clique index (list).
bool ns_tables(const NsLayout& L, unsigned char* base, const std::vector<long long>& poff,
               const std::vector<int>& list, std::vector<unsigned char>& img);
// ||W||_F per block, X_0 = W / ||W||_F, then ns_iterate.
cudaError_t ns_scale_and_iterate(const NsLayout& L, unsigned char* base, cudaStream_t st);
// W (hi, lo) from packed lower float blocks at poff (device table).
cudaError_t ns_from_packed(const NsLayout& L, unsigned char* base, const float* Wp, cudaStream_t st);
// sign iteration, then P = (W + W sign(W)) / 2 into BUF_X2 (hi, plain float)
cudaError_t ns_iterate(const NsLayout& L, unsigned char* base, cudaStream_t st);
// packed lower values of P
cudaError_t ns_to_packed(const NsLayout& L, unsigned char* base, float* Xp, cudaStream_t st);

// One projection step of the ADMM iteration for the large cliques (FP32
// clique state; large_step.cu): gather W of `form` (0/1/2: Algorithm 1/2/3)
// into the dense buffers, the sign iteration, then the state updates of that
// form and the per-clique stopping sums (row `row_off + i` of the partial
// table, or row k in component mode); with fa.enabled (Algorithm 1) the last
// block runs the stopping test.
}  // namespace cdsdp_large
namespace cdsdp_dev { struct Dev; struct FinishArgs; }
namespace cdsdp_large {
cudaError_t large_step(int form, const cdsdp_dev::Dev& d, const NsLayout& L, unsigned char* base, int row_off,
                       const cdsdp_dev::FinishArgs& fa, cudaStream_t st);

}  // namespace cdsdp_large
