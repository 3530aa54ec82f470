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
    size_t o_err = 0, o_maps = 0, o_tiles = 0, o_blocks = 0, o_chunk = 0, o_partial = 0, o_scale = 0, o_poff = 0;
    size_t o_buf[2 * NBUF] = {0};
    size_t bytes = 0;
};

NsLayout ns_layout(const std::vector<int>& sizes);
// Host image of bytes [0, o_buf[0]) for device memory at `base`: tensor maps
// of every (buffer, block), tiles, blocks, chunk offsets, packed offsets.
bool ns_tables(const NsLayout& L, unsigned char* base, const std::vector<long long>& poff,
               std::vector<unsigned char>& img);
// W (hi, lo) and X_0 from packed lower float blocks at poff (device table).
cudaError_t ns_from_packed(const NsLayout& L, unsigned char* base, const float* Wp, cudaStream_t st);
// sign iteration, then P = (W + W sign(W)) / 2 into BUF_X2 (hi, plain float)
cudaError_t ns_iterate(const NsLayout& L, unsigned char* base, cudaStream_t st);
// packed lower values of P
cudaError_t ns_to_packed(const NsLayout& L, unsigned char* base, float* Xp, cudaStream_t st);

}  // namespace cdsdp_large
