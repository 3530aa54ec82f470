// Batched PSD projection of float32 clique blocks of padded order 36..64 (in
// steps of 4), one thread block per clique, with the eigenvector matrix V held
// in registers.  Same method as jacobi.cuh and jacobi_cta.cuh: two-sided
// Jacobi in the Brent-Luk parallel ordering (storage re-indexed by the
// round-robin permutation sigma after every round), the 2x2 symmetric Schur
// step and rotations in Rutishauser's form (tau = s / (1 + c)), warm start from
// the clique's previous eigenvectors, stagnation stop at the rounding-noise
// floor.  The arithmetic of every rotation and of every updated entry of A is
// that of CTAJacobiMid; what changes is where the data live and how a round
// is synchronised.
//
//  * A (lower triangle, physical layout of CTAJacobiMid: even storage indices
//    first, then odd ones) is double-buffered in shared memory; each thread
//    owns fixed pair-blocks of A whose source and sigma-permuted destination
//    offsets are computed once per launch.
//  * V lives in registers: thread (row i, part g), g < 4, holds row i of V on
//    a contiguous range of storage pairs [k0_g, k0_g + n_g).  A round rotates
//    the pairs locally; sigma then moves every even column one pair up and
//    every odd column one pair down, so each thread passes one value to each
//    neighbouring part (two warp shuffles; the four parts of a row are
//    consecutive lanes).  V is written to shared memory only for the two
//    products of the warm start and for the rebuild.
//  * One barrier per round.  The rotation of pair k in round r + 1 acts on
//    entries that round r produces in a single pair-block (the block holding
//    (sigma^-1(2k+1), sigma^-1(2k))); the thread that updates that block also
//    forms the next rotation (its diagonal entries are the current diagonal
//    plus or minus t a_pq) and stores it into the other half of a
//    double-buffered rotation table.  Nothing else waits for a rotation.
//  * Shared memory: the two A buffers, a third buffer for the products of the
//    warm start and the rebuild (each writes its register tiles there without
//    a barrier in between) and the rotation tables: about 35 KB at order 52.
#pragma once

#include "jacobi.cuh"

namespace cdsdp_dev {

template <int S>
struct CTAJacobiReg {
    using T = float;
    static_assert(S % 4 == 0 && S >= 36 && S <= 64, "padded orders 36..64 in steps of 4");
    using RR = RoundRobin<S>;
    static constexpr int K = S / 2;
    static constexpr int R = S - 1;
    static constexpr int LDA = S + 4;  // rows stay 16-byte aligned
    static constexpr int BUF = S * LDA;
    static constexpr int NB = K * (K + 1) / 2;  // lower pair-blocks of A
    static constexpr int NVT = 4 * S;          // threads holding V (4 per row)
    static constexpr int NT = (NVT + 31) / 32 * 32;
    static constexpr int NPB = (NB + NT - 1) / NT;  // pair-blocks per thread
    static constexpr int PB = K / 4, PR = K % 4;    // pairs per part: PB + (g < PR)
    static constexpr int NPR = PB + (PR > 0 ? 1 : 0);
    static constexpr int S4 = S / 4;
    static_assert(PB >= 2, "part 0 holds pairs 0 and 1");
    static_assert(S4 * S4 <= NT, "one 4x4 product tile per thread");
    static_assert(BUF < 65536, "offsets fit 16 bits");
    // two A buffers, rotation tables [2][K] of (tau, sin) and [2][K] of t a_pq,
    // reduction scratch, max(lambda, 0)
    static constexpr size_t bytes = ((3 * (size_t)BUF + 4 * K + 2 * K + 32 + S) * sizeof(T) + 15) & ~size_t(15);

    __host__ __device__ static constexpr int phys(int i) { return (i & 1) ? K + (i >> 1) : (i >> 1); }
    __device__ __forceinline__ static int at(int r, int c) { return phys(r) * LDA + phys(c); }
    __device__ __forceinline__ static int lower(int r, int c) { return r >= c ? at(r, c) : at(c, r); }

    // shared memory: A buffers 0 and 1, then the rotation tables [2][K] of
    // (tau, sin) pairs and [2][K] of t a_pq, reduction scratch [32] and
    // max(lambda, 0) [S] in physical order
    T* base;
    int cur;  // A buffer holding the current matrix
    __device__ __forceinline__ T* cs() const { return base + 3 * BUF; }
    __device__ __forceinline__ T* ta() const { return base + 3 * BUF + 4 * K; }
    __device__ __forceinline__ T* red() const { return base + 3 * BUF + 6 * K; }
    __device__ __forceinline__ T* lam() const { return base + 3 * BUF + 6 * K + 32; }

    // V row `row` on pairs [k0, k0 + n) of storage order: ve[j] at column
    // 2 (k0 + j), vo[j] at 2 (k0 + j) + 1; thread = 4 row + part.
    T ve[NPR], vo[NPR];
    int k0, n;
    __device__ __forceinline__ static int row() { return threadIdx.x >> 2; }
    __device__ __forceinline__ static int part() { return threadIdx.x & 3; }

    // Pair-blocks of A owned by this thread: (destination 0 | destination 1 << 16),
    // (destination 2 | destination 3 << 16), meta = kind | I << 2 | J << 7 |
    // producer << 12 | entry << 13 | pair << 15 (kind 1: diagonal block, 2:
    // off-diagonal block, 0: none; a producer block forms the next round's
    // rotation of `pair` from its output `entry` = 2 r + c at offsets (r, c)).
    struct Plan { unsigned w0[NPB], w1[NPB], w2[NPB]; };

    __device__ __forceinline__ void bind(unsigned char* smem_base) {
        base = reinterpret_cast<T*>(smem_base);
        cur = 0;
        k0 = part() * PB + min(part(), PR);
        n = PB + (part() < PR ? 1 : 0);
    }
    __device__ __forceinline__ bool vthread() const { return threadIdx.x < NVT; }
    __device__ __forceinline__ T* X() const { return base + cur * BUF; }

    __device__ __forceinline__ static void plan(Plan& P) {
#pragma unroll
        for (int j = 0; j < NPB; ++j) {
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
            }
            const int r0 = 2 * I, r1 = r0 + 1, c0 = 2 * J, c1 = c0 + 1;
            const int sr0 = RR::sigma(r0), sr1 = RR::sigma(r1), sc0 = RR::sigma(c0), sc1 = RR::sigma(c1);
            const int d0 = lower(sr0, sc0), d1 = lower(sr1, sc0), d2 = lower(sr0, sc1), d3 = lower(sr1, sc1);
            // the block (I, J) = (pair of sigma^-1(2k+1), pair of sigma^-1(2k)) produces pair k's next rotation
            int prod = 0, ent = 0, pk = 0;
            if (kind == 2) {
                if (I == 1 && J == 0) { prod = 1; ent = 2; pk = 0; }                       // (3, 0)
                else if (I == 2 && J == 0) { prod = 1; ent = 3; pk = 1; }                  // (5, 1)
                else if (I == K - 1 && J == K - 2) { prod = 1; ent = 0; pk = K - 1; }      // (S-2, S-4)
                else if (J >= 1 && I == J + 2 && J + 1 <= K - 2) { prod = 1; ent = 2; pk = J + 1; }  // (2k+3, 2k-2)
            }
            P.w0[j] = unsigned(d0) | (unsigned(d1) << 16);
            P.w1[j] = unsigned(d2) | (unsigned(d3) << 16);
            P.w2[j] = unsigned(kind | (I << 2) | (J << 7) | (prod << 12) | (ent << 13) | (pk << 15));
        }
    }

    __device__ __forceinline__ void clear() {
        T* x = X();
        for (int i = threadIdx.x; i < BUF; i += blockDim.x) x[i] = T(0);
        __syncthreads();
    }
    __device__ __forceinline__ void put(int a, int b, T w) {
        T* x = X();
        x[at(a, b)] = w;
        x[at(b, a)] = w;
    }

    // 2x2 symmetric Schur step in Rutishauser's form: (tau, sin) and t a_pq,
    // all zero when |a_pq| <= tol.
    __device__ __forceinline__ static void schur(T app, T aqq, T apq, T tol, T& tau, T& sn, T& tq) {
        tau = T(0); sn = T(0); tq = T(0);
        if (fabsf(apq) > tol) {
            const T zeta = T(0.5) * (aqq - app);
            const T r2 = zeta * zeta + apq * apq;
            const T r = r2 * rsqrt_t<T>(r2);
            const T tt = copysignf(T(1), zeta) * div_t<T>(apq, fabsf(zeta) + r);
            const T c = rsqrt_t<T>(T(1) + tt * tt);
            sn = tt * c;
            tau = div_t<T>(sn, T(1) + c);
            tq = tt * apq;
        }
    }

    // block-wide max of |off-diagonal| of the lower triangle of A
    __device__ __forceinline__ T off_max(const Plan& P) {
        const T* x = X();
        T m = T(0);
#pragma unroll
        for (int j = 0; j < NPB; ++j) {
            const int kind = P.w2[j] & 3, I = (P.w2[j] >> 2) & 31, J = (P.w2[j] >> 7) & 31;
            const int src = I * LDA + J;
            if (kind == 1) {
                m = fmaxf(m, fabsf(x[src + K * LDA]));
            } else if (kind == 2) {
                m = fmaxf(fmaxf(m, fabsf(x[src])), fabsf(x[src + K]));
                m = fmaxf(fmaxf(m, fabsf(x[src + K * LDA])), fabsf(x[src + K * LDA + K]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) red()[warp] = m;
        __syncthreads();
        T r = T(0);
        for (int w = 0; w < NT / 32; ++w) r = fmaxf(r, red()[w]);
        __syncthreads();
        return r;
    }

    // One round from A buffer B into 1 - B, rotations from table B; producers
    // write table 1 - B.  Ends with the round's only barrier.
    template <int B>
    __device__ __forceinline__ void round_b(T tol, const Plan& P) {
        const T* Xc = base + B * BUF;
        T* Yn = base + (1 - B) * BUF;
        const float2* csr = reinterpret_cast<const float2*>(cs()) + K * B;
        const T* tar = ta() + K * B;
        float2* csw = reinterpret_cast<float2*>(cs()) + K * (1 - B);
        T* taw = ta() + K * (1 - B);
        // pair-blocks of A: J_I^T B J_J into the permuted positions of the other buffer
#pragma unroll
        for (int j = 0; j < NPB; ++j) {
            const unsigned w2 = P.w2[j];
            const int kind = w2 & 3;
            if (kind == 0) continue;
            const int I = (w2 >> 2) & 31, J = (w2 >> 7) & 31, src = I * LDA + J;
            const int d0 = P.w0[j] & 0xffff, d1 = P.w0[j] >> 16, d2 = P.w1[j] & 0xffff, d3 = P.w1[j] >> 16;
            if (kind == 1) {
                const T t = tar[I];
                const bool rotated = t != T(0) || csr[I].y != T(0);
                const T b00 = Xc[src], b10 = Xc[src + K * LDA], b11 = Xc[src + K * LDA + K];
                Yn[d0] = b00 - t;
                Yn[d1] = rotated ? T(0) : b10;
                Yn[d3] = b11 + t;
            } else {
                const T b00 = Xc[src], b01 = Xc[src + K], b10 = Xc[src + K * LDA], b11 = Xc[src + K * LDA + K];
                const float2 ri = csr[I], rj = csr[J];  // (tau, s)
                const T q00 = b00 - ri.y * (b10 + ri.x * b00), q10 = b10 + ri.y * (b00 - ri.x * b10);
                const T q01 = b01 - ri.y * (b11 + ri.x * b01), q11 = b11 + ri.y * (b01 - ri.x * b11);
                const T o00 = q00 - rj.y * (q01 + rj.x * q00);
                const T o01 = q01 + rj.y * (q00 - rj.x * q01);
                const T o10 = q10 - rj.y * (q11 + rj.x * q10);
                const T o11 = q11 + rj.y * (q10 - rj.x * q11);
                Yn[d0] = o00;
                Yn[d2] = o01;
                Yn[d1] = o10;
                Yn[d3] = o11;
                if ((w2 >> 12) & 1) {  // next round's rotation of pair pk
                    const int ent = (w2 >> 13) & 3, pk = (w2 >> 15) & 31;
                    const int ro = ent >> 1, co = ent & 1;
                    const T apq = ent == 0 ? o00 : (ent == 2 ? o10 : o11);
                    const T xa = Xc[(co ? K + J : J) * (LDA + 1)];
                    const T xb = Xc[(ro ? K + I : I) * (LDA + 1)];
                    const T app = co ? xa + tar[J] : xa - tar[J];
                    const T aqq = ro ? xb + tar[I] : xb - tar[I];
                    T tau, sn, tq;
                    schur(app, aqq, apq, tol, tau, sn, tq);
                    csw[pk] = make_float2(tau, sn);
                    taw[pk] = tq;
                }
            }
        }
        // V <- V J on this thread's pairs (after the pair-blocks, which keeps
        // the loads of both parts from being in flight at once)
        asm volatile("" ::: "memory");
        if (vthread()) {
#pragma unroll
            for (int j = 0; j < NPR; ++j) {
                if (j < n) {
                    const float2 r = csr[k0 + j];  // (tau, s)
                    const T vp = ve[j], vq = vo[j];
                    ve[j] = vp - r.y * (vq + r.x * vp);
                    vo[j] = vq + r.y * (vp - r.x * vq);
                }
            }
        }
        // V's columns re-indexed by sigma: even columns one pair up (position 0
        // fixed, position 1 to 2), odd columns one pair down (position S-2 to S-1)
        const T e_last = (n == NPR) ? ve[NPR - 1] : ve[NPR - 2];
        const T o_first = vo[0];
        const T up = __shfl_up_sync(0xffffffffu, e_last, 1);      // part g - 1: its last even column
        const T dn = __shfl_down_sync(0xffffffffu, o_first, 1);   // part g + 1: its first odd column
        {
            const T e0 = ve[0];
#pragma unroll
            for (int j = NPR - 1; j >= 1; --j) ve[j] = ve[j - 1];
            ve[0] = part() ? up : e0;
            if (part() == 0) ve[1] = o_first;
#pragma unroll
            for (int j = 0; j + 1 < NPR; ++j) vo[j] = vo[j + 1];
            const T in_o = part() < 3 ? dn : e_last;
            if (n == NPR) vo[NPR - 1] = in_o;
            else vo[NPR - 2] = in_o;
        }
        __syncthreads();
    }
    // one sweep (R rounds, R odd) starting in buffer B; it ends in 1 - B
    template <int B>
    __device__ __forceinline__ void sweep(T tol, const Plan& P) {
#pragma unroll 1
        for (int r = 0; r + 1 < R; r += 2) {
            round_b<B>(tol, P);
            round_b<1 - B>(tol, P);
        }
        round_b<B>(tol, P);
    }

    // V <- identity (cold) or keep the loaded basis (warm), then sweep; each
    // sweep returns the storage order to the identity.
    __device__ __forceinline__ void identity_basis() {
#pragma unroll
        for (int j = 0; j < NPR; ++j) {
            ve[j] = (row() == 2 * (k0 + j)) ? T(1) : T(0);
            vo[j] = (row() == 2 * (k0 + j) + 1) ? T(1) : T(0);
        }
    }
    __device__ __forceinline__ int run(T tol, int max_sweeps, bool v_preset) {
        if (!v_preset) identity_basis();
        Plan P;
        plan(P);
        const T noise = tol * T(2 * S);
        T prev = T(3.0e38);
        int sw = 0;
        bool have_rot = false;
        while (sw < max_sweeps) {
            const T off = off_max(P);
            if (off <= tol) break;
            if (off <= noise && off > T(0.5) * prev) break;
            prev = off;
            ++sw;
            if (!have_rot) {  // first round's rotations; later sweeps get theirs from the last round
                const T* x = X();
                const int k = threadIdx.x;
                if (k < K) {
                    T tau, sn, tq;
                    schur(x[k * (LDA + 1)], x[(K + k) * (LDA + 1)], x[(K + k) * LDA + k], tol, tau, sn, tq);
                    reinterpret_cast<float2*>(cs())[K * cur + k] = make_float2(tau, sn);
                    ta()[K * cur + k] = tq;
                }
                __syncthreads();
                have_rot = true;
            }
            if (cur == 0) sweep<0>(tol, P); else sweep<1>(tol, P);
            cur ^= 1;
        }
        return sw;
    }

    // 4x4 tile (tr, tc) of A^T B (physical S x S arrays, leading dimension LDA)
    __device__ __forceinline__ static void atb_tile(const T* __restrict__ A, const T* __restrict__ B, int tr, int tc,
                                                    T (&acc)[4][4]) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
#pragma unroll 2
        for (int i = 0; i < S; ++i) {
            const float4 a = *reinterpret_cast<const float4*>(A + i * LDA + 4 * tr);
            const float4 b = *reinterpret_cast<const float4*>(B + i * LDA + 4 * tc);
            const T av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
    }
    __device__ __forceinline__ static void store_tile(T* __restrict__ C, int tr, int tc, const T (&acc)[4][4]) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4*>(C + (4 * tr + u) * LDA + 4 * tc) =
                make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }

    // V <- the stored s x s eigenvector matrix (row-major at Vc), padded with
    // the identity, into the other A buffer; rotate_into_basis then takes the
    // registers' copy from there.
    __device__ __forceinline__ void load_basis(const T* __restrict__ Vc, int s) {
        T* vs = base + (1 - cur) * BUF;
        for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
            const int r = i / S, c = i - r * S;
            vs[at(r, c)] = (r < s && c < s) ? Vc[r * s + c] : (r == c ? T(1) : T(0));
        }
        __syncthreads();
    }
    __device__ __forceinline__ void store_basis(T* __restrict__ Vc, int s) const {
        const int row = this->row();
        if (vthread() && row < s) {
#pragma unroll
            for (int j = 0; j < NPR; ++j) {
                if (j < n) {
                    const int ce = 2 * (k0 + j), co = ce + 1;
                    if (ce < s) Vc[row * s + ce] = ve[j];
                    if (co < s) Vc[row * s + co] = vo[j];
                }
            }
        }
    }

    // A <- V^T W V (the current buffer holds the symmetric W in both
    // triangles, the other one V), through register tiles.
    __device__ __forceinline__ void rotate_into_basis() {
        T* x = base + cur * BUF;
        const T* vs = base + (1 - cur) * BUF;
        T* y = base + 2 * BUF;
        const int tile = threadIdx.x, tr = tile / S4, tc = tile - tr * S4;
        if (tile < S4 * S4) {  // Y = W V (W symmetric)
            T acc[4][4];
            atb_tile(x, vs, tr, tc, acc);
            store_tile(y, tr, tc, acc);
        }
        __syncthreads();
        if (tile < S4 * S4) {  // A = V^T Y
            T acc[4][4];
            atb_tile(vs, y, tr, tc, acc);
            store_tile(x, tr, tc, acc);
        }
        {  // V stays in the other buffer: the registers' copy (every register
           // assigned, clamped where a thread holds fewer pairs or no row)
            const int row = min(this->row(), S - 1);
#pragma unroll
            for (int j = 0; j < NPR; ++j) {
                const int ce = 2 * min(k0 + j, K - 1);
                ve[j] = vs[at(row, ce)];
                vo[j] = vs[at(row, ce + 1)];
            }
        }
        __syncthreads();
    }

    // Third buffer <- V max(Lambda, 0) V^T on its lower physical 4x4 tiles
    // (Lambda on the current buffer's diagonal), with V^T written from the
    // registers into the other buffer.
    __device__ __forceinline__ void prepare_rebuild() {
        const T* x = base + cur * BUF;
        T* vt = base + (1 - cur) * BUF;
        T* y = base + 2 * BUF;
        T* lam = this->lam();
        const int row = this->row();
        for (int i = threadIdx.x; i < S; i += blockDim.x) {
            const T l = x[i * LDA + i];
            lam[i] = l > T(0) ? l : T(0);
        }
        if (vthread()) {
#pragma unroll
            for (int j = 0; j < NPR; ++j) {
                if (j < n) {
                    const int ce = 2 * (k0 + j);
                    vt[at(ce, row)] = ve[j];
                    vt[at(ce + 1, row)] = vo[j];
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < S4 * (S4 + 1) / 2) {
            int tr = 0, o = threadIdx.x;
            while (o > tr) { o -= tr + 1; ++tr; }
            const int tc = o;  // tr >= tc
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
#pragma unroll 2
            for (int c = 0; c < S; ++c) {
                const T l = lam[c];
                const float4 a = *reinterpret_cast<const float4*>(vt + c * LDA + 4 * tr);
                const float4 b = *reinterpret_cast<const float4*>(vt + c * LDA + 4 * tc);
                const T av[4] = {l * a.x, l * a.y, l * a.z, l * a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
            }
            store_tile(y, tr, tc, acc);
        }
        __syncthreads();
    }
    // entry (a, b) of the rebuilt block (symmetric: its lower physical half)
    __device__ __forceinline__ T rebuild(int a, int b, int) const {
        const T* x = base + 2 * BUF;
        const int pa = phys(a), pb = phys(b);
        return pa >= pb ? x[pa * LDA + pb] : x[pb * LDA + pa];
    }
};

}  // namespace cdsdp_dev
