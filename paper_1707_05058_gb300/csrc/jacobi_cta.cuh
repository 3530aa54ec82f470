// Batched PSD projection of clique blocks of order 33..128: one thread block
// (CTA) per clique.  Same method as jacobi.cuh (two-sided Jacobi in the
// Brent-Luk parallel ordering, 2x2 symmetric Schur step and rotations in
// Rutishauser's form (tau = s / (1 + c), no norm bias at small angles),
// warm start from the clique's previous eigenvectors, stagnation stop at the
// rounding-noise floor), laid out for a CTA.
//
// Orders up to 64 (CTAJacobiMid, padded orders in steps of 4):
//  * A (lower triangle) and V live in shared memory, each double-buffered;
//    V is kept in the same storage order as A, so a round is one uniform pass
//    over pair-blocks: lower blocks (I, J) of A get J_I^T B J_J, blocks of V
//    get the column rotation B J_J, and every result is stored at its
//    position permuted by sigma in the other buffer;
//  * each thread owns a fixed list of pair-blocks whose source and permuted
//    destination offsets it computes once per launch (registers);
//  * V^T W V (warm start) and V max(Lambda, 0) V^T are 4x4-tiled products;
//  * two barriers per round (rotations ready; buffers swapped).
// Orders 65..128 (CTAJacobi): A double-buffered as above, V single-buffered
// and rotated in place at the round's logical column pair (L[2k], L[2k+1]),
// L following sigma.
// Float32 orders 36..64 can also run CTAJacobiReg (jacobi_reg.cuh: V in
// registers, one barrier per round); k_project_cta's VARIANT selects it.
#pragma once

#include <type_traits>

#include "jacobi.cuh"
#include "jacobi_reg.cuh"

namespace cdsdp_dev {

constexpr int kCtaThreads = 256;
// Threads per clique block: float32 orders up to 48 use 128 threads, so that
// six independent cliques share an SM (more latency hidden per round);
// larger orders and float64 use 256.
template <typename T, int S>
__host__ __device__ constexpr int cta_threads() { return (sizeof(T) == 4 && S <= 48) ? 128 : kCtaThreads; }
template <typename T, int S>
__host__ __device__ constexpr int cta_min_blocks() {
    return (sizeof(T) == 4 && S <= 48) ? 6 : ((sizeof(T) == 4 && S <= 64) ? 3 : 1);
}

template <typename T, int S>
struct CTAJacobi {
    using RR = RoundRobin<S>;
    static constexpr int K = S / 2;
    static constexpr int R = S - 1;
    static constexpr int LDA = S + 1;
    static constexpr int BUF = S * LDA;
    static constexpr int NB = K * (K + 1) / 2;
    static constexpr size_t bytes =
        ((3 * (size_t)BUF + 3 * K) * sizeof(T) + 4 * (size_t)S * sizeof(int) + 64 * sizeof(T) + 15) & ~size_t(15);

    T* X;    // current A
    T* Y;    // next A
    T* V;    // eigenvectors, row-major, logical columns
    T* cs;   // [K] tau = s / (1 + c), [K] sin, [K] t * a_pq
    int* L;  // logical index at each storage position (current)
    int* Ln; // next
    T* red;  // [32] reduction scratch

    __device__ __forceinline__ void bind(unsigned char* base) {
        X = reinterpret_cast<T*>(base);
        Y = X + BUF;
        V = Y + BUF;
        cs = V + BUF;
        red = cs + 3 * K;
        L = reinterpret_cast<int*>(red + 64);
        Ln = L + 2 * S;
    }

    __device__ __forceinline__ static void block_coords(int b, int& I, int& J) {
        if (b < K) { I = J = b; return; }
        const int o = b - K;  // off-diagonal blocks I > J, o = I (I - 1) / 2 + J
        int i = int((1.0f + sqrtf(1.0f + 8.0f * float(o))) * 0.5f);
        while (i * (i - 1) / 2 > o) --i;
        while ((i + 1) * i / 2 <= o) ++i;
        I = i;
        J = o - i * (i - 1) / 2;
    }

    __device__ __forceinline__ void clear() {
        for (int i = threadIdx.x; i < BUF; i += blockDim.x) X[i] = T(0);
        __syncthreads();
    }
    __device__ __forceinline__ void put(int a, int b, T w) {
        X[a * LDA + b] = w;
        X[b * LDA + a] = w;
    }

    // block-wide max of |off-diagonal| of the lower triangle of X
    __device__ T off_max() {
        T m = T(0);
        for (int idx = threadIdx.x; idx < S * S; idx += blockDim.x) {
            const int i = idx / S, j = idx - i * S;
            if (i > j) m = fmax(m, fabs(X[i * LDA + j]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) red[warp] = m;
        __syncthreads();
        T r = T(0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
        __syncthreads();
        return r;
    }

    __device__ void round(T tol) {
        const int tid = threadIdx.x, nt = blockDim.x;
        if (tid < K) {  // rotation of pair tid (Rutishauser form)
            const T app = X[(2 * tid) * LDA + 2 * tid], aqq = X[(2 * tid + 1) * LDA + 2 * tid + 1];
            const T apq = X[(2 * tid + 1) * LDA + 2 * tid];
            T tau = T(0), sn = T(0), ta = T(0);
            if (fabs(apq) > tol) {
                const T zeta = T(0.5) * (aqq - app);
                const T r2 = zeta * zeta + apq * apq;
                const T r = r2 * rsqrt_t<T>(r2);
                const T tt = copysign(T(1), zeta) * div_t<T>(apq, fabs(zeta) + r);
                const T c = rsqrt_t<T>(T(1) + tt * tt);
                sn = tt * c;
                tau = div_t<T>(sn, T(1) + c);
                ta = tt * apq;
            }
            cs[tid] = tau;
            cs[K + tid] = sn;
            cs[2 * K + tid] = ta;
        }
        if (tid < S) Ln[RR::sigma(tid)] = L[tid];
        __syncthreads();
        for (int b = tid; b < NB; b += nt) {  // pair-blocks of A, into Y at permuted positions
            int I, J;
            block_coords(b, I, J);
            const int r0 = 2 * I, r1 = r0 + 1, c0 = 2 * J, c1 = c0 + 1;
            const int sr0 = RR::sigma(r0), sr1 = RR::sigma(r1), sc0 = RR::sigma(c0), sc1 = RR::sigma(c1);
            if (I == J) {
                const T ta = cs[2 * K + I];
                const bool rot = ta != T(0) || cs[K + I] != T(0);
                Y[max(sr0, sc0) * LDA + min(sr0, sc0)] = X[r0 * LDA + c0] - ta;
                Y[max(sr1, sc0) * LDA + min(sr1, sc0)] = rot ? T(0) : X[r1 * LDA + c0];
                Y[max(sr1, sc1) * LDA + min(sr1, sc1)] = X[r1 * LDA + c1] + ta;
            } else {
                const T uI = cs[I], sI = cs[K + I], uJ = cs[J], sJ = cs[K + J];
                const T b00 = X[r0 * LDA + c0], b10 = X[r1 * LDA + c0], b01 = X[r0 * LDA + c1], b11 = X[r1 * LDA + c1];
                const T q00 = b00 - sI * (b10 + uI * b00), q10 = b10 + sI * (b00 - uI * b10);
                const T q01 = b01 - sI * (b11 + uI * b01), q11 = b11 + sI * (b01 - uI * b11);
                Y[max(sr0, sc0) * LDA + min(sr0, sc0)] = q00 - sJ * (q01 + uJ * q00);
                Y[max(sr0, sc1) * LDA + min(sr0, sc1)] = q01 + sJ * (q00 - uJ * q01);
                Y[max(sr1, sc0) * LDA + min(sr1, sc0)] = q10 - sJ * (q11 + uJ * q10);
                Y[max(sr1, sc1) * LDA + min(sr1, sc1)] = q11 + sJ * (q10 - uJ * q11);
            }
        }
        for (int task = tid; task < S * K; task += nt) {  // V <- V J at the logical column pairs
            const int i = task / K, k = task - i * K;
            const T u = cs[k], sn = cs[K + k];
            if (sn == T(0)) continue;
            const int p = L[2 * k], q = L[2 * k + 1];
            T* vr = V + i * LDA;
            const T vp = vr[p], vq = vr[q];
            vr[p] = vp - sn * (vq + u * vp);
            vr[q] = vq + sn * (vp - u * vq);
        }
        __syncthreads();
        T* t = X; X = Y; Y = t;
        int* u = L; L = Ln; Ln = u;
    }

    // V <- identity (cold) or keep the loaded basis (warm), then sweep.
    __device__ int run(T tol, int max_sweeps, bool v_preset) {
        if (!v_preset)
            for (int i = threadIdx.x; i < BUF; i += blockDim.x) V[i] = ((i / LDA) == (i % LDA)) ? T(1) : T(0);
        if (threadIdx.x < S) L[threadIdx.x] = threadIdx.x;
        __syncthreads();
        const T noise = tol * T(2 * S);
        T prev = T(3.0e38);
        int sw = 0;
        while (sw < max_sweeps) {
            const T off = off_max();
            if (off <= tol) break;
            if (off <= noise && off > T(0.5) * prev) break;
            prev = off;
            ++sw;
            for (int r = 0; r < R; ++r) round(tol);
        }
        return sw;
    }

    // X <- V^T X V (X holds the symmetric W in both triangles, V the basis).
    __device__ void rotate_into_basis() {
        const int tid = threadIdx.x, nt = blockDim.x;
        for (int idx = tid; idx < S * S; idx += nt) {  // Y = W V
            const int r = idx / S, j = idx - r * S;
            T a = T(0);
#pragma unroll 8
            for (int i = 0; i < S; ++i) a += X[r * LDA + i] * V[i * LDA + j];
            Y[r * LDA + j] = a;
        }
        __syncthreads();
        for (int idx = tid; idx < S * S; idx += nt) {  // X = V^T Y
            const int i = idx / S, j = idx - i * S;
            T a = T(0);
#pragma unroll 8
            for (int r = 0; r < S; ++r) a += V[r * LDA + i] * Y[r * LDA + j];
            X[i * LDA + j] = a;
        }
        __syncthreads();
    }

    __device__ void load_basis(const T* __restrict__ Vc, int s) {
        for (int i = threadIdx.x; i < BUF; i += blockDim.x) {
            const int r = i / LDA, c = i - r * LDA;
            V[i] = (r < s && c < s) ? Vc[r * s + c] : (r == c ? T(1) : T(0));
        }
        __syncthreads();
    }
    __device__ void store_basis(T* __restrict__ Vc, int s) const {
        for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
            const int r = i / s, c = i - r * s;
            Vc[i] = V[r * LDA + c];
        }
    }
    // Y row a <- V row a scaled by max(lambda, 0) (lambda on X's diagonal).
    __device__ void prepare_rebuild() {
        for (int i = threadIdx.x; i < BUF; i += blockDim.x) {
            const int r = i / LDA, c = i - r * LDA;
            if (c < S) {
                const T l = X[c * LDA + c];
                Y[i] = V[i] * (l > T(0) ? l : T(0));
            }
        }
        __syncthreads();
    }
    __device__ __forceinline__ T rebuild(int a, int b, int s) const {
        const T* ya = Y + a * LDA;
        const T* vb = V + b * LDA;
        T acc = T(0);
        for (int i = 0; i < s; ++i) acc += ya[i] * vb[i];
        return acc;
    }
};

// Vector views of shared memory (the dynamic buffer is only 16-byte aligned,
// so a 4-vector of doubles is read as two 16-byte halves).
template <typename T> struct alignas(2 * sizeof(T)) Vec2 { T x, y; };
template <typename T> struct alignas(16) Vec4 { T x, y, z, w; };

template <typename T, int S>
struct CTAJacobiMid {
    static_assert(S % 4 == 0 && S <= 64, "padded orders 36..64 in steps of 4");
    using RR = RoundRobin<S>;
    using T2 = Vec2<T>;
    using T4 = Vec4<T>;
    static constexpr int K = S / 2;
    static constexpr int R = S - 1;
    static constexpr int LDA = S + 4;          // rows stay 16-byte aligned
    static constexpr int BUF = S * LDA;
    static constexpr int NB = K * (K + 1) / 2; // lower pair-blocks of A
    static constexpr int NBLK = NB + K * K;    // plus the pair-blocks of V
    static constexpr int NT = cta_threads<T, S>();
    static constexpr int NPT = (NBLK + NT - 1) / NT;
    static constexpr int S4 = S / 4;
    static constexpr size_t bytes = ((4 * (size_t)BUF + 3 * K + 32 + S) * sizeof(T) + 15) & ~size_t(15);
    static_assert(BUF < 65536, "offsets fit 16 bits");

    // Physical layout: storage index i lives at phys(i) (even indices first,
    // then odd ones) in both dimensions, so the entries a warp writes to
    // their sigma-permuted positions (even -> next even, odd -> previous odd)
    // are consecutive words.  Products and the rebuild work directly on the
    // physical arrays (the same permutation on every index).
    __host__ __device__ static constexpr int phys(int i) { return (i & 1) ? K + (i >> 1) : (i >> 1); }
    __host__ __device__ static constexpr int logical(int q) { return q < K ? 2 * q : 2 * (q - K) + 1; }
    __device__ __forceinline__ static int at(int r, int c) { return phys(r) * LDA + phys(c); }
    __device__ __forceinline__ static int lower(int r, int c) { return r >= c ? at(r, c) : at(c, r); }

    T* base; // four S x LDA buffers: A (two), V (two)
    T* X;    // A, current
    T* Y;    // A, next
    T* V;    // eigenvectors, current (column = storage index)
    T* Vn;   // next
    T* cs;   // [K] (tau, sin) pairs, tau = s / (1 + c)
    T* ta;   // [K] t * a_pq
    T* red;  // [32] reduction scratch
    T* lam;  // [S] max(lambda, 0), physical order

    // The pair-blocks a thread owns during the sweeps, three 16-bit pairs each:
    // (source, destination 0), (destination 1, destination 2), (destination 3,
    // meta) with meta = kind | I << 2 | J << 7 (kind 1: diagonal block of A,
    // 2: off-diagonal block of A, 3: block of V, 0: none).  The four source
    // entries of a block sit at source + {0, K, K LDA, K LDA + K}.
    struct Plan { unsigned w0[NPT], w1[NPT], w2[NPT]; };

    __device__ __forceinline__ void bind(unsigned char* smem_base) {
        base = reinterpret_cast<T*>(smem_base);
        X = base;
        Y = X + BUF;
        V = Y + BUF;
        Vn = V + BUF;
        cs = Vn + BUF;
        ta = cs + 2 * K;
        red = ta + K;
        lam = red + 32;
    }

    __device__ __forceinline__ static void plan(Plan& P) {
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int b = threadIdx.x + j * NT;
            int kind = 0, I = 0, J = 0;
            if (b < K) {
                kind = 1;
                I = J = b;
            } else if (b < NB) {
                int o = b - K;
                I = 1;
                while (o >= I) { o -= I; ++I; }
                J = o;
                kind = 2;
            } else if (b < NBLK) {
                const int v = b - NB;
                I = v / K;
                J = v - I * K;
                kind = 3;
            }
            const int r0 = 2 * I, r1 = r0 + 1, c0 = 2 * J, c1 = c0 + 1;
            const int sc0 = RR::sigma(c0), sc1 = RR::sigma(c1);
            int d0, d1, d2, d3;
            if (kind == 3) {  // rows of V stay, columns move with sigma
                d0 = at(r0, sc0);
                d1 = at(r1, sc0);
                d2 = at(r0, sc1);
                d3 = at(r1, sc1);
            } else {
                const int sr0 = RR::sigma(r0), sr1 = RR::sigma(r1);
                d0 = lower(sr0, sc0);
                d1 = lower(sr1, sc0);
                d2 = lower(sr0, sc1);
                d3 = lower(sr1, sc1);
            }
            const unsigned meta = unsigned(kind | (I << 2) | (J << 7));
            P.w0[j] = unsigned(I * LDA + J) | (unsigned(d0) << 16);  // = at(r0, c0)
            P.w1[j] = unsigned(d1) | (unsigned(d2) << 16);
            P.w2[j] = unsigned(d3) | (meta << 16);
        }
    }

    __device__ __forceinline__ void clear() {
        for (int i = threadIdx.x; i < BUF; i += blockDim.x) X[i] = T(0);
        __syncthreads();
    }
    __device__ __forceinline__ void put(int a, int b, T w) {
        X[at(a, b)] = w;
        X[at(b, a)] = w;
    }

    // block-wide max of |off-diagonal| of the lower triangle of A
    __device__ T off_max(const Plan& P) {
        T m = T(0);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int kind = (P.w2[j] >> 16) & 3, src = P.w0[j] & 0xffff;
            if (kind == 1) {
                m = fmax(m, fabs(X[src + K * LDA]));
            } else if (kind == 2) {
                m = fmax(fmax(m, fabs(X[src])), fabs(X[src + K]));
                m = fmax(fmax(m, fabs(X[src + K * LDA])), fabs(X[src + K * LDA + K]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) red[warp] = m;
        __syncthreads();
        T r = T(0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
        __syncthreads();
        return r;
    }

    // One round from buffer B into buffer 1 - B.  The buffers sit at fixed
    // offsets from the block's shared memory, so every access is a register
    // offset plus a constant.
    template <int B>
    __device__ __forceinline__ void round_b(T tol, const Plan& P) {
        const int tid = threadIdx.x;
        const T* Xc = base + B * BUF;
        T* Yn = base + (1 - B) * BUF;
        const T* Vc = base + (2 + B) * BUF;
        T* Vw = base + (3 - B) * BUF;
        if (tid < K) {  // rotation of pair tid (Rutishauser form)
            const T app = Xc[tid * LDA + tid], aqq = Xc[(K + tid) * LDA + K + tid];
            const T apq = Xc[(K + tid) * LDA + tid];
            T tau = T(0), sn = T(0), tq = T(0);
            if (fabs(apq) > tol) {
                const T zeta = T(0.5) * (aqq - app);
                const T r2 = zeta * zeta + apq * apq;
                const T r = r2 * rsqrt_t<T>(r2);
                const T tt = copysign(T(1), zeta) * div_t<T>(apq, fabs(zeta) + r);
                const T c = rsqrt_t<T>(T(1) + tt * tt);
                sn = tt * c;
                tau = div_t<T>(sn, T(1) + c);
                tq = tt * apq;
            }
            reinterpret_cast<T2*>(cs)[tid] = T2{tau, sn};
            ta[tid] = tq;
        }
        __syncthreads();
        const T2* rot = reinterpret_cast<const T2*>(cs);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const unsigned meta = P.w2[j] >> 16;
            const int kind = meta & 3;
            if (kind == 0) continue;
            const int I = (meta >> 2) & 31, J = meta >> 7, src = P.w0[j] & 0xffff;
            const int d0 = P.w0[j] >> 16, d1 = P.w1[j] & 0xffff, d2 = P.w1[j] >> 16, d3 = P.w2[j] & 0xffff;
            if (kind == 3) {
                const T v00 = Vc[src], v01 = Vc[src + K], v10 = Vc[src + K * LDA], v11 = Vc[src + K * LDA + K];
                const T2 r = rot[J];  // (tau, s)
                Vw[d0] = v00 - r.y * (v01 + r.x * v00);
                Vw[d2] = v01 + r.y * (v00 - r.x * v01);
                Vw[d1] = v10 - r.y * (v11 + r.x * v10);
                Vw[d3] = v11 + r.y * (v10 - r.x * v11);
            } else if (kind == 1) {
                const T t = ta[I];
                const bool rotated = t != T(0) || rot[I].y != T(0);
                const T b00 = Xc[src], b10 = Xc[src + K * LDA], b11 = Xc[src + K * LDA + K];
                Yn[d0] = b00 - t;
                Yn[d1] = rotated ? T(0) : b10;
                Yn[d3] = b11 + t;
            } else {
                const T b00 = Xc[src], b01 = Xc[src + K], b10 = Xc[src + K * LDA], b11 = Xc[src + K * LDA + K];
                const T2 ri = rot[I], rj = rot[J];  // (tau, s)
                const T q00 = b00 - ri.y * (b10 + ri.x * b00), q10 = b10 + ri.y * (b00 - ri.x * b10);
                const T q01 = b01 - ri.y * (b11 + ri.x * b01), q11 = b11 + ri.y * (b01 - ri.x * b11);
                Yn[d0] = q00 - rj.y * (q01 + rj.x * q00);
                Yn[d2] = q01 + rj.y * (q00 - rj.x * q01);
                Yn[d1] = q10 - rj.y * (q11 + rj.x * q10);
                Yn[d3] = q11 + rj.y * (q10 - rj.x * q11);
            }
        }
        __syncthreads();
    }
    // one sweep (R rounds, R odd) starting in buffer B; it ends in 1 - B
    template <int B>
    __device__ void sweep(T tol, const Plan& P) {
        for (int r = 0; r + 1 < R; r += 2) {
            round_b<B>(tol, P);
            round_b<1 - B>(tol, P);
        }
        round_b<B>(tol, P);
    }

    // V <- identity (cold) or keep the loaded basis (warm), then sweep; each
    // sweep returns the storage order to the identity.
    __device__ int run(T tol, int max_sweeps, bool v_preset) {
        if (!v_preset)
            for (int i = threadIdx.x; i < BUF; i += blockDim.x) V[i] = ((i / LDA) == (i % LDA)) ? T(1) : T(0);
        __syncthreads();
        // buffers 0/1 hold A and 2/3 V; X and V are buffers cur and 2 + cur
        Plan P;
        plan(P);
        const T noise = tol * T(2 * S);
        T prev = T(3.0e38);
        int sw = 0, cur = (X == base) ? 0 : 1;
        while (sw < max_sweeps) {
            X = base + cur * BUF;
            const T off = off_max(P);
            if (off <= tol) break;
            if (off <= noise && off > T(0.5) * prev) break;
            prev = off;
            ++sw;
            if (cur == 0) sweep<0>(tol, P); else sweep<1>(tol, P);
            cur ^= 1;
        }
        X = base + cur * BUF;
        Y = base + (1 - cur) * BUF;
        V = base + (2 + cur) * BUF;
        Vn = base + (3 - cur) * BUF;
        return sw;
    }

    // C = A^T B over 4x4 output tiles (physical S x S arrays, leading dimension LDA).
    __device__ void atb(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C) const {
        for (int tile = threadIdx.x; tile < S4 * S4; tile += blockDim.x) {
            const int tr = tile / S4, tc = tile - tr * S4;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
#pragma unroll 4
            for (int i = 0; i < S; ++i) {
                const T4 a = *reinterpret_cast<const T4*>(A + i * LDA + 4 * tr);
                const T4 b = *reinterpret_cast<const T4*>(B + i * LDA + 4 * tc);
                const T av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                *reinterpret_cast<T4*>(C + (4 * tr + u) * LDA + 4 * tc) = T4{acc[u][0], acc[u][1], acc[u][2], acc[u][3]};
        }
    }

    // A <- V^T W V (X holds the symmetric W in both triangles, V the basis).
    __device__ void rotate_into_basis() {
        atb(X, V, Y);  // Y = W V (W symmetric)
        __syncthreads();
        atb(V, Y, X);  // X = V^T Y
        __syncthreads();
    }

    __device__ void load_basis(const T* __restrict__ Vc, int s) {
        for (int i = threadIdx.x; i < BUF; i += blockDim.x) {
            const int qr = i / LDA, qc = i - qr * LDA;
            const int r = logical(qr), c = logical(qc);
            V[i] = (r < s && c < s && qc < S) ? Vc[r * s + c] : (r == c ? T(1) : T(0));
        }
        __syncthreads();
    }
    __device__ void store_basis(T* __restrict__ Vc, int s) const {
        for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
            const int r = i / s, c = i - r * s;
            Vc[i] = V[at(r, c)];
        }
    }

    // X <- V max(Lambda, 0) V^T over the lower physical 4x4 tiles, Lambda on
    // X's diagonal.
    __device__ void prepare_rebuild() {
        for (int i = threadIdx.x; i < S; i += blockDim.x) {
            const T l = X[i * LDA + i];
            lam[i] = l > T(0) ? l : T(0);
        }
        for (int idx = threadIdx.x; idx < S * S; idx += blockDim.x) {  // Y = V^T
            const int r = idx / S, c = idx - r * S;
            Y[c * LDA + r] = V[r * LDA + c];
        }
        __syncthreads();
        for (int tile = threadIdx.x; tile < S4 * (S4 + 1) / 2; tile += blockDim.x) {
            int tr = 0, o = tile;
            while (o > tr) { o -= tr + 1; ++tr; }
            const int tc = o;  // tr >= tc
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
#pragma unroll 4
            for (int c = 0; c < S; ++c) {
                const T l = lam[c];
                const T4 a = *reinterpret_cast<const T4*>(Y + c * LDA + 4 * tr);
                const T4 b = *reinterpret_cast<const T4*>(Y + c * LDA + 4 * tc);
                const T av[4] = {l * a.x, l * a.y, l * a.z, l * a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                *reinterpret_cast<T4*>(X + (4 * tr + u) * LDA + 4 * tc) = T4{acc[u][0], acc[u][1], acc[u][2], acc[u][3]};
        }
        __syncthreads();
    }
    // entry (a, b) of the rebuilt block (symmetric: read its lower physical half)
    __device__ __forceinline__ T rebuild(int a, int b, int) const {
        const int pa = phys(a), pb = phys(b);
        return pa >= pb ? X[pa * LDA + pb] : X[pb * LDA + pa];
    }
};

template <typename T, int S>
using CTASolver = typename std::conditional<(S <= 64), CTAJacobiMid<T, S>, CTAJacobi<T, S>>::type;

// Solver of k_project_cta: VARIANT 0 keeps V in shared memory (CTAJacobiMid,
// CTAJacobi); VARIANT 1 (float32, padded orders 36..64) keeps V in registers
// (CTAJacobiReg).
template <typename T, int S, int VARIANT>
struct CTAPick {
    using type = CTASolver<T, S>;
    static constexpr int threads = cta_threads<T, S>();
    static constexpr int min_blocks = cta_min_blocks<T, S>();
};
template <int S>
struct CTAPick<float, S, 1> {
    using type = CTAJacobiReg<S>;
    static constexpr int threads = CTAJacobiReg<S>::NT;
    // blocks per SM: as many as 64 registers a thread allow at orders 36..56
    // (6, 5 or 4 blocks); 3 at orders 60 and 64, which spill at 64 registers
    // and ran slower with 4 (measured on the 256-SDP batch)
    static constexpr int min_blocks = S >= 60 ? 3 : 65536 / (CTAJacobiReg<S>::NT * 64);
};

template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV], double* sh) {
    block_sum<NV>(v, sh);  // valid in thread 0
}

// One kernel for every form: FORM 0/1/2 = Algorithm 1/2/3 step (as the warp
// kernels of jacobi.cuh), FORM 3 = standalone projection; VARIANT selects the
// solver (CTAPick).
template <typename T, int S, int FORM, int VARIANT>
__global__ void __launch_bounds__(CTAPick<T, S, VARIANT>::threads, CTAPick<T, S, VARIANT>::min_blocks) k_project_cta(Dev d, const int* __restrict__ list, int nlist, ProjArgs pa,
                                                              FinishArgs fa, const int* __restrict__ off_arr,
                                                              const int* __restrict__ size_arr,
                                                              const T* __restrict__ Win, T* Xout) {
    using J = typename CTAPick<T, S, VARIANT>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double shr[32 * 6];
    if (FORM != 3 && stopped(d)) return;
    J jac;
    jac.bind(smem);
    const int tid = threadIdx.x;
    // clique state and eigenvector cache (taken from the parameters where used)
#define c0 (reinterpret_cast<T*>(d.ck0))
#define c1 (reinterpret_cast<T*>(d.ck1))
#define c2 (reinterpret_cast<T*>(d.ck2))
#define vc (reinterpret_cast<T*>(d.vcache))
    const bool warm = FORM != 3 && pa.warm_start && (d.ctl[CTL_ITER] % pa.restart) != 0;
    __shared__ double acc[6];  // block partial sums, kept by thread 0
    // the clique's scalars, read back after the eigensolve so that they hold
    // no registers during it: k, s, offset; rho, gamma, <c, x> (thread 0's sum)
    __shared__ int ck_i[3];
    __shared__ double ck_d[3];
    if (tid < 6) acc[tid] = 0.0;
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        const int k = FORM == 3 ? li : list[li];
        const int s = FORM == 3 ? size_arr[k] : d.csize[k];
        const int off = FORM == 3 ? off_arr[k] : d.pk_off[k];
        if (s > S || s < 1) continue;  // block-uniform
        if (FORM != 3 && frozen_clique(d, k)) continue;
        const double rho = (FORM == 0 || FORM == 1) ? rho_clique(d, k) : 1.0, irho = 1.0 / rho;
        const double gamma = FORM == 2 ? hs_gamma_c(d, comp_k(d, k)) : 0.0;
        const int npk = s * (s + 1) / 2;
        if (tid == 0) {
            ck_i[0] = k; ck_i[1] = s; ck_i[2] = off;
            ck_d[0] = rho; ck_d[1] = gamma;
        }
        jac.clear();
        double nrm = 0.0, cx = 0.0;
        if constexpr (VARIANT == 1) {
            if (FORM != 0 || pa.x_ready) {
                // the same gather with every load of this thread's entries issued
                // before their use: indices, then the values they address
                constexpr int NTH = CTAPick<T, S, VARIANT>::threads;
                constexpr int MAXF = (S * (S + 1) / 2 + NTH - 1) / NTH;
                int ent[MAXF];
                double v0[MAXF], v1[MAXF], v2[MAXF];
                bool own[MAXF];
#pragma unroll
                for (int u = 0; u < MAXF; ++u) {
                    const int f = tid + u * NTH;
                    const bool ok = f < npk;
                    ent[u] = (ok && (FORM == 0 || FORM == 2)) ? d.gmap[off + f] : 0;
                    own[u] = (ok && FORM == 0) ? d.owner[off + f] != 0 : false;
                    v1[u] = (ok && FORM != 3) ? double(c1[off + f]) : 0.0;
                    v2[u] = (ok && (FORM == 1 || FORM == 2)) ? double(c2[off + f]) : 0.0;
                    v0[u] = ok ? (FORM == 3 ? double(Win[off + f]) : (FORM == 2 ? double(c0[off + f]) : 0.0)) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < MAXF; ++u) {
                    const int f = tid + u * NTH;
                    if (f >= npk) continue;
                    const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
                    double w;
                    if (FORM == 0) {
                        const double xe = d.x[ent[u]];
                        if (own[u]) cx += d.wgt[ent[u]] * d.c[ent[u]] * xe;
                        w = xe - v1[u] * irho;
                        if (d.wstore) {
                            const int slot = d.ctl[CTL_ITER];
                            if (slot < d.wstore_count) reinterpret_cast<T*>(d.wstore)[(size_t)slot * d.nd + off + f] = T(w);
                        }
                    } else if (FORM == 1) {
                        w = v1[u] - v2[u] * irho;
                    } else if (FORM == 2) {
                        const double hs = d.s11[ent[u]];
                        const double s12 = 0.5 * (v0[u] + v1[u] - v2[u] + hs);
                        w = s12 - gamma * 0.5 * d.zhx[ent[u]] - v1[u];
                    } else {
                        w = v0[u];
                    }
                    jac.put(a, b, T(w));
                    nrm += (a == b ? 1.0 : 2.0) * w * w;
                }
            }
        }
        for (int f = tid; f < npk && (VARIANT != 1 || (FORM == 0 && !pa.x_ready)); f += blockDim.x) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            double w;
            if (FORM == 0) {
                const int ent = d.gmap[off + f];
                double xe;
                if (pa.x_ready) {
                    xe = d.x[ent];
                } else {
                    double aty = 0.0;
                    for (int q = d.at_ptr[ent]; q < d.at_ptr[ent + 1]; ++q) aty += d.at_val[q] * d.y[d.at_col[q]];
                    xe = d.t[ent] - d.dinv[ent] * aty;
                    if (d.owner[off + f]) d.x[ent] = xe;
                    d.q[ent] = xe;  // H_k x for the epilogue (scratch, same value from every clique)
                }
                if (d.owner[off + f]) cx += d.wgt[ent] * d.c[ent] * xe;
                w = xe - double(c1[off + f]) * irho;
                if (d.wstore) {
                    const int slot = d.ctl[CTL_ITER];
                    if (slot < d.wstore_count) reinterpret_cast<T*>(d.wstore)[(size_t)slot * d.nd + off + f] = T(w);
                }
            } else if (FORM == 1) {
                w = double(c1[off + f]) - double(c2[off + f]) * irho;
            } else if (FORM == 2) {
                const int ent = d.gmap[off + f];
                const double hs = d.s11[ent];
                const double s12 = 0.5 * (double(c0[off + f]) + double(c1[off + f]) - double(c2[off + f]) + hs);
                w = s12 - gamma * 0.5 * d.zhx[ent] - double(c1[off + f]);
            } else {
                w = double(Win[off + f]);
            }
            jac.put(a, b, T(w));
            nrm += (a == b ? 1.0 : 2.0) * w * w;
        }
        double tmp[2] = {nrm, cx};
        cta_sum<2>(tmp, shr);
        if (tid == 0) { shr[0] = tmp[0]; ck_d[2] = tmp[1]; }
        __syncthreads();
        nrm = shr[0];
        __syncthreads();
        if constexpr (VARIANT == 1) {  // V's registers assigned on both paths
            if (warm) {
                jac.load_basis(vc + d.vv_off[k], s);
                jac.rotate_into_basis();
            } else {
                jac.identity_basis();
            }
            jac.run(T(pa.tolrel) * T(sqrt(nrm)), pa.max_sweeps, true);
        } else {
            if (warm) {
                jac.load_basis(vc + d.vv_off[k], s);
                jac.rotate_into_basis();
            }
            jac.run(T(pa.tolrel) * T(sqrt(nrm)), pa.max_sweeps, warm);
        }
        {  // epilogue: the clique's scalars from shared memory
        const int k = ck_i[0], s = ck_i[1], off = ck_i[2];
        const double rho = ck_d[0], gamma = ck_d[1];
        const double cxk = tid == 0 ? ck_d[2] : 0.0;
        const int npk = s * (s + 1) / 2;
        if (FORM != 3 && pa.warm_start) jac.store_basis(vc + d.vv_off[k], s);
        jac.prepare_rebuild();
        double p[6] = {0, 0, 0, 0, 0, 0};
        T pf[5] = {0, 0, 0, 0, 0};  // float32 form of Algorithm 1: per-thread sums in float
        if constexpr (VARIANT == 1) {
            // the same epilogue with this thread's loads issued before their use
            constexpr int NTH = CTAPick<T, S, VARIANT>::threads;
            constexpr int MAXF = (S * (S + 1) / 2 + NTH - 1) / NTH;
            int ent[MAXF];
            T e0[MAXF], e1[MAXF], e2[MAXF];
#pragma unroll
            for (int u = 0; u < MAXF; ++u) {
                const int f = tid + u * NTH;
                const bool ok = f < npk && FORM != 3;
                ent[u] = (ok && (FORM == 0 || FORM == 2)) ? d.gmap[off + f] : 0;
                e0[u] = ok ? c0[off + f] : T(0);
                e1[u] = (ok && (FORM == 0 || FORM == 2)) ? c1[off + f] : T(0);
                e2[u] = (ok && FORM == 2) ? c2[off + f] : T(0);
            }
#pragma unroll
            for (int u = 0; u < MAXF; ++u) {
                const int f = tid + u * NTH;
                if (f >= npk) continue;
                const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
                const T xn = jac.rebuild(a, b, s);
                const T wt = (a == b) ? T(1) : T(2);
                if (FORM == 0) {  // float32 clique state and its sums
                    const T hxt = T(pa.x_ready ? d.x[ent[u]] : d.q[ent[u]]), lm = e1[u], xo = e0[u];
                    const T ln = lm + T(rho) * (xn - hxt);
                    c0[off + f] = xn;
                    c1[off + f] = ln;
                    const T dc = xn - hxt, dx = xn - xo;
                    pf[0] += wt * dc * dc; pf[1] += wt * xn * xn; pf[2] += wt * hxt * hxt;
                    pf[3] += wt * dx * dx; pf[4] += wt * ln * ln;
                } else if (FORM == 1) {
                    const T dz = xn - e0[u];
                    c0[off + f] = xn;
                    pf[0] += wt * dz * dz;
                } else if (FORM == 2) {
                    const double w = (a == b) ? 1.0 : 2.0;
                    const double hs = d.s11[ent[u]], zs = 0.5 * d.zhx[ent[u]];
                    const double u_s = e0[u], v_z = e1[u], u_t = e2[u];
                    const double s12 = 0.5 * (u_s + v_z - u_t + hs);
                    const double s22 = u_t - hs + s12;
                    const double uhs = s12 - gamma * zs, utn = s22 + gamma * zs;
                    const double hux = hs - gamma * d.zhx[ent[u]];
                    const double vn = v_z - uhs + double(xn);
                    c0[off + f] = xn;
                    c1[off + f] = T(vn);
                    c2[off + f] = T(utn);
                    const double d1 = double(xn) - hux, d2 = vn - utn;
                    p[0] += w * d1 * d1; p[1] += w * double(xn) * double(xn); p[2] += w * hux * hux;
                    p[3] += w * d2 * d2; p[4] += w * vn * vn; p[5] += w * utn * utn;
                } else {
                    Xout[off + f] = xn;
                }
            }
        }
        for (int f = tid; f < npk && VARIANT != 1; f += blockDim.x) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const T xn = jac.rebuild(a, b, s);
            const double w = (a == b) ? 1.0 : 2.0;
            if (FORM == 0) {
                const double hx = pa.x_ready ? d.x[d.gmap[off + f]] : d.q[d.gmap[off + f]];
                if constexpr (sizeof(T) == 4) {  // clique state in float32: its sums too
                    const T hxt = T(hx), lm = c1[off + f], xo = c0[off + f];
                    const T ln = lm + T(rho) * (xn - hxt);
                    c0[off + f] = xn;
                    c1[off + f] = ln;
                    const T wt = T(w), dc = xn - hxt, dx = xn - xo;
                    pf[0] += wt * dc * dc; pf[1] += wt * xn * xn; pf[2] += wt * hxt * hxt;
                    pf[3] += wt * dx * dx; pf[4] += wt * ln * ln;
                } else {
                    const double lm = c1[off + f];
                    const double xo = c0[off + f];
                    const double ln = lm + rho * (double(xn) - hx);
                    c0[off + f] = xn;
                    c1[off + f] = T(ln);
                    const double dc = double(xn) - hx, dx = double(xn) - xo;
                    p[0] += w * dc * dc; p[1] += w * double(xn) * double(xn); p[2] += w * hx * hx;
                    p[3] += w * dx * dx; p[4] += w * ln * ln;
                }
            } else if (FORM == 1) {
                const T dz = xn - c0[off + f];
                c0[off + f] = xn;
                if constexpr (sizeof(T) == 4) pf[0] += T(w) * dz * dz;
                else p[0] += w * double(dz) * double(dz);
            } else if (FORM == 2) {
                const int ent = d.gmap[off + f];
                const double hs = d.s11[ent], zs = 0.5 * d.zhx[ent];
                const double u_s = c0[off + f], v_z = c1[off + f], u_t = c2[off + f];
                const double s12 = 0.5 * (u_s + v_z - u_t + hs);
                const double s22 = u_t - hs + s12;
                const double uhs = s12 - gamma * zs, utn = s22 + gamma * zs;
                const double hux = hs - gamma * d.zhx[ent];
                const double vn = v_z - uhs + double(xn);
                c0[off + f] = xn;
                c1[off + f] = T(vn);
                c2[off + f] = T(utn);
                const double d1 = double(xn) - hux, d2 = vn - utn;
                p[0] += w * d1 * d1; p[1] += w * double(xn) * double(xn); p[2] += w * hux * hux;
                p[3] += w * d2 * d2; p[4] += w * vn * vn; p[5] += w * utn * utn;
            } else {
                Xout[off + f] = xn;
            }
        }
        if (FORM != 3) {
            if (FORM == 0 && sizeof(T) == 4)
                for (int c = 0; c < 5; ++c) p[c] = double(pf[c]);
            if (FORM == 1 && sizeof(T) == 4) p[0] = double(pf[0]);
            cta_sum<6>(p, shr);
            if (FORM != 2) p[5] = cxk;
            if (tid == 0 && d.comp_mode) {  // per-clique row, reduced per component
                double* pr = d.part + (size_t)k * PART_COLS;
                if (FORM == 0 || FORM == 2) { for (int c = 0; c < 6; ++c) pr[c] = p[c]; }
                else if (FORM == 1) { pr[5] = p[0]; }
            } else if (tid == 0) {
                for (int c = 0; c < 5; ++c) acc[c] += p[c];
                if (FORM != 1) acc[5] += p[5];
            }
        }
        __syncthreads();
        }
    }
    if (FORM == 3) return;
    if (d.comp_mode) return;
    if (tid == 0) {
        double* pr = d.part + (size_t)(pa.row_off + blockIdx.x) * PART_COLS;
        if (FORM == 0) { for (int c = 0; c < 6; ++c) pr[c] = acc[c]; }
        else if (FORM == 1) { pr[5] = acc[0]; }
        else { for (int c = 0; c < 6; ++c) pr[c] = acc[c]; }
    }
    if (FORM == 0 && fa.enabled && last_block_single_writer(d)) finish_primal_block(d, fa);
#undef c0
#undef c1
#undef c2
#undef vc
}

}  // namespace cdsdp_dev
