// PSD projection of large clique blocks (order > 128) on the tensor cores.
//
// The projection of Section 4.1.2 (Eq. XkUpdate) needs only
//   P(W) = V max(Lambda, 0) V^T = (W + W sign(W)) / 2,
// where sign(W) = V sign(Lambda) V^T.  For blocks of order 129 .. a few
// thousand (the cliques of a minimum-degree extension of a sparse random
// graph) the sign is computed by an odd polynomial (Newton-Schulz) iteration
// on X_0 = W / ||W||_F, whose eigenvalues lie in [-1, 1]:
//   phase 1 (range growth), N1 steps of  X <- a X + b X^3 + c X^5,
//            a = 3.30, b = -3.66, c = 1.36: p(1) = 1, p maps [0, 1.3] into
//            itself, every x >= 0.22 into [0.7, 1.3], and small x grow by
//            3.3 per step (coefficients found by a grid search under those
//            constraints);
//   phase 2 (convergence), N2 steps of  X <- 1.5 X - 0.5 X^3  (Newton-Schulz;
//            quadratic convergence from [0.7, 1.3]);
// then P = (W + W X) / 2.  With N1 = 16 and N2 = 5 every eigenvalue with
// |lambda| >= 1e-8 ||W||_F reaches |sign| within float32 rounding of 1; an
// eigenvalue below that contributes at most |lambda| / 2 to the error of P.
// Every step is a product of two symmetric matrices that commute (powers of
// W), so only the lower tiles of each product are computed and mirrored.
//
// Products run in float32 accuracy as three TF32 products (Ootomo and
// Yokota, 2022): x = x_hi + x_lo with x_hi = tf32(x) (round to nearest) and
// x_lo = x - x_hi; A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, all accumulated in
// float32 in tensor memory.  Every matrix of the iteration is stored as its
// (hi, lo) pair, row-major, block k at a 256-byte aligned offset with row
// pitch S_k = ceil(s_k / 128) * 128 floats (zero padding stays zero under odd
// polynomials).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdsdp_large {

constexpr int kTile = 128;         // output tile (M = N = 128), one CTA each
constexpr int kChunk = 32;         // K floats per stage: one 128-byte swizzle row
constexpr int kStages = 3;
constexpr int kTileBytes = kTile * kChunk * 4;       // 16 KB per operand tile
constexpr int kStageBytes = 4 * kTileBytes;          // A_hi, A_lo, B_hi, B_lo
constexpr int kGemmSmem = kStages * kStageBytes + 1024 + 256;
constexpr int kGemmThreads = 128;

// Phase-1 polynomial and the iteration counts.
constexpr float kPa = 3.30f, kPb = -3.66f, kPc = 1.36f;
constexpr int kPhase1 = 16, kPhase2 = 5;

// One output tile (ti, tj), ti >= tj, of block `blk`.
struct Tile { int blk, ti, tj, pad; };

// Dense layout of one block in every buffer: float offset and padded order.
struct Block { long long off; int S, s; };

// The (hi, lo) buffers of the iteration.
enum { BUF_W = 0, BUF_XA = 1, BUF_XB = 2, BUF_X2 = 3, BUF_B = 4, NBUF = 5 };

// Epilogue of one product D = alpha A B + beta C over the lower tiles, C and
// D given as (hi, lo) pairs; D_lo == nullptr writes D in plain float32 to D_hi.
struct GemmArgs {
    const void* mapA_hi; const void* mapA_lo;   // tensor maps, one per block (CUtensorMap arrays)
    const void* mapB_hi; const void* mapB_lo;
    const float* C_hi; const float* C_lo;
    float* D_hi; float* D_lo;
    const Block* blocks;
    const Tile* tiles;
    int ntiles;
    float alpha, beta;
    int* err;                                   // set on a timed-out wait (kernel returns early)
};

}  // namespace cdsdp_large
