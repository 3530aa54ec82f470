// Batched PSD projection P(W) = V max(Lambda, 0) V^T of clique blocks
// (Section 4.1.2, Eq. XkUpdate; Eq. zkUpdate; Eq. HsdeStep2), one warp per
// block of order s <= 32.
//
// Eigensolver: two-sided cyclic Jacobi (Jacobi 1846; 2x2 symmetric Schur step
// of Golub and Van Loan, Matrix Computations, Section 8.5) in the parallel
// ordering of Brent and Luk (1985).  The block is padded with zero rows to an
// even order S (padding rows never rotate: their entries stay exactly zero and
// their eigenvalues are 0).  Storage positions are paired as (2k, 2k+1),
// k < S/2; after every round the matrix is re-indexed by the round-robin
// permutation sigma (position 0 fixed, the other S-1 positions rotate along the
// circle 2, 4, ..., S-2, S-1, S-3, ..., 1), so over one sweep of S-1 rounds
// every pair of indices meets exactly once and the storage order returns to
// the identity.  Each lane owns fixed 2x2 pair-blocks (I, J), I >= J, of the
// lower triangle: per round it loads them from one shared-memory buffer,
// applies J_I^T B J_J and writes them to their permuted positions in the other
// buffer (one warp barrier per round).  Row `lane` of V stays in registers
// and its columns are re-indexed by the same sigma (static register moves).
// Every rotation is applied in Rutishauser's form (Handbook for Automatic
// Computation II, contribution II/1, 1971): with tau = s / (1 + c),
//   x' = c x - s y = x - s (y + tau x),   y' = s x + c y = y + s (x - tau y).
// For the small angles of the late sweeps c rounds to 1 while s = t does not,
// so the plain (c, s) products grow every rotated row and column by a factor
// 1 + t^2 (a bias, not noise); in float32 this bias, summed over a few hundred
// rotations per eigenvector, dominated the error of the projection.  The tau
// form carries 1 - c = s tau implicitly and has no such bias.
// A rotation is skipped when |a_pq| <= tol = 2 u ||W||_F (u the unit
// roundoff), and a sweep starts only while some off-diagonal entry exceeds tol
// (or until max_sweeps).  Eigenvalues clustered within rounding noise of each
// other (typical near zero at ADMM convergence) can keep off-diagonal entries
// at about S u ||W||_F forever; a block whose largest off-diagonal entry is
// below 4 S u ||W||_F and did not halve over the last sweep has reached that
// floor and stops.
// Warm start (ADMM iterates move little between iterations): each clique keeps
// its eigenvectors V from the previous iteration; the new block W is first
// rotated into that basis (A = V^T W V, two warp-level products) and the
// sweeps continue from V, which typically needs one sweep instead of five or
// six.  Every `restart` iterations the eigensolve starts from the identity, so
// rounding in the accumulated V cannot drift.
#pragma once

#include "reduce.cuh"
#include "proj_launch.h"

namespace cdsdp_dev {

// ---- round-robin ordering on S storage positions ---------------------------
template <int S>
struct RoundRobin {
    static constexpr int K = S / 2;
    static constexpr int R = S - 1;
    __host__ __device__ static constexpr int circ_index(int p) {  // p > 0
        return (p % 2 == 0) ? (p / 2 - 1) : (K - 1 + (K - 1 - (p - 1) / 2));
    }
    __host__ __device__ static constexpr int circ_pos(int c) {
        return c < K - 1 ? 2 * (c + 1) : 2 * (K - 1 - (c - (K - 1))) + 1;
    }
    __host__ __device__ static constexpr int sigma(int p) { return p == 0 ? 0 : circ_pos((circ_index(p) + 1) % R); }
    __host__ __device__ static constexpr int sigma_inv(int p) {
        return p == 0 ? 0 : circ_pos((circ_index(p) + R - 1) % R);
    }
};

// (a, b) of packed element f of an s x s block, a >= b, column-major.
__device__ __forceinline__ int packed_ab(int f, int s) {
    const float t = float(2 * s + 1);
    int b = int((t - sqrtf(t * t - 8.0f * float(f))) * 0.5f);
    b = max(0, min(b, s - 1));
    while (b > 0 && b * (2 * s - b + 1) / 2 > f) --b;
    while (b + 1 < s && (b + 1) * (2 * s - b) / 2 <= f) ++b;
    const int a = b + f - b * (2 * s - b + 1) / 2;
    return (a << 8) | b;
}

template <typename T, int S, int LW = 32>
struct BLJacobi {
    static_assert(LW == 32 || LW == 16 || LW == 8, "lanes per clique");
    static_assert(LW == 32 || S <= LW, "row `lane` of V needs a lane per row");
    using RR = RoundRobin<S>;
    static constexpr int K = S / 2;
    static constexpr int R = S - 1;
    static constexpr int LDA = S + 1;
    static constexpr int BUF = S * LDA;
    static constexpr int NB = K * (K + 1) / 2;      // lower pair-blocks
    static constexpr int NS = (NB + LW - 1) / LW;   // blocks per lane
    static constexpr int NPK = S * (S + 1) / 2;
    static constexpr int MAXE = (NPK + LW - 1) / LW;  // packed elements per lane
    static constexpr size_t bytes = (2 * BUF * sizeof(T) + 15) & ~size_t(15);  // per clique

    T* X;  // current buffer
    T* Y;  // next buffer
    T v[S];  // row `lane` of V
    int src[NS][4], dst[NS][4];
    int bI[NS], bJ[NS];

    __device__ __forceinline__ void bind(unsigned char* base, int lane) {
        X = reinterpret_cast<T*>(base);
        Y = X + BUF;
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const int b = lane + LW * t;
            int I = 0, J = 0;
            if (b < K) {
                I = J = b;
            } else if (b < NB) {
                int o = b - K;
                I = 1;
                while (o >= I) { o -= I; ++I; }
                J = o;
            }
            const bool ok = b < NB;
            bI[t] = ok ? I : -1;
            bJ[t] = J;
            const int r0 = 2 * I, r1 = 2 * I + 1, c0 = 2 * J, c1 = 2 * J + 1;
            src[t][0] = r0 * LDA + c0;
            src[t][1] = r1 * LDA + c0;
            src[t][2] = (I == J) ? r1 * LDA + c0 : r0 * LDA + c1;
            src[t][3] = r1 * LDA + c1;
            const int rr[4] = {r0, r1, r0, r1}, cc[4] = {c0, c0, c1, c1};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int si = RR::sigma(rr[e]), sj = RR::sigma(cc[e]);
                dst[t][e] = max(si, sj) * LDA + min(si, sj);
            }
        }
    }

    // Zero the working buffer (padding rows must read as exact zeros).
    __device__ __forceinline__ void clear(int lane) {
        for (int i = lane; i < BUF; i += LW) X[i] = T(0);
        __syncwarp();
    }
    __device__ __forceinline__ void put(int a, int b, T w) {
        X[a * LDA + b] = w;
        X[b * LDA + a] = w;
    }

    // Largest |off-diagonal entry| of the lower triangle in X (same in all lanes).
    __device__ __forceinline__ T off_max(int lane) const {
        T m = T(0);
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            if (bI[t] < 0) continue;
            if (t == 0 && lane < K) {
                m = fmax(m, fabs(X[src[0][1]]));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) m = fmax(m, fabs(X[src[t][e]]));
            }
        }
#pragma unroll
        for (int o = LW / 2; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));  // within the group
        return m;
    }

    // Warm start: v holds the rows of an orthogonal V (lane r: row r), X the
    // symmetric block W (both triangles).  Replace X by V^T W V, so that the
    // sweeps continue from the basis V (the final eigenvectors are V J_1 J_2 ...).
    // Both products are spread element-wise over the 32 lanes; Y is scratch.
    __device__ void rotate_into_basis(int lane) {
        constexpr int NE1 = (S * S + LW - 1) / LW;
        if (lane < S) {
#pragma unroll
            for (int j = 0; j < S; ++j) Y[lane * LDA + j] = v[j];
        }
        __syncwarp();
        T acc[NE1];
#pragma unroll
        for (int e = 0; e < NE1; ++e) {  // (W V)_{rj}
            const int idx = lane + LW * e;
            T a = T(0);
            if (idx < S * S) {
                const int r = idx / S, j = idx - r * S;
                const T* xr = X + r * LDA;
#pragma unroll 4
                for (int i = 0; i < S; ++i) a += xr[i] * Y[i * LDA + j];
            }
            acc[e] = a;
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NE1; ++e) {
            const int idx = lane + LW * e;
            if (idx < S * S) {
                const int r = idx / S, j = idx - r * S;
                X[r * LDA + j] = acc[e];
            }
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NE1; ++e) {  // (V^T (W V))_{ij}
            const int idx = lane + LW * e;
            T a = T(0);
            if (idx < S * S) {
                const int i = idx / S, j = idx - i * S;
#pragma unroll 4
                for (int r = 0; r < S; ++r) a += Y[r * LDA + i] * X[r * LDA + j];
            }
            acc[e] = a;
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NE1; ++e) {
            const int idx = lane + LW * e;
            if (idx < S * S) {
                const int i = idx / S, j = idx - i * S;
                X[i * LDA + j] = acc[e];
            }
        }
        __syncwarp();
    }

    // X <- V X V^T (inverse of rotate_into_basis; X symmetric, both triangles).
    __device__ void rotate_out_of_basis(int lane) {
        constexpr int NE1 = (S * S + LW - 1) / LW;
        if (lane < S) {
#pragma unroll
            for (int j = 0; j < S; ++j) Y[lane * LDA + j] = v[j];
        }
        __syncwarp();
        T acc[NE1];
#pragma unroll
        for (int e = 0; e < NE1; ++e) {  // (X V^T)_{ib} = sum_j X_ij V_bj
            const int idx = lane + LW * e;
            T a = T(0);
            if (idx < S * S) {
                const int i = idx / S, b = idx - i * S;
#pragma unroll 4
                for (int j = 0; j < S; ++j) a += X[i * LDA + j] * Y[b * LDA + j];
            }
            acc[e] = a;
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NE1; ++e) {
            const int idx = lane + LW * e;
            if (idx < S * S) X[(idx / S) * LDA + idx % S] = acc[e];
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NE1; ++e) {  // (V (X V^T))_{ab} = sum_i V_ai (X V^T)_ib
            const int idx = lane + LW * e;
            T a = T(0);
            if (idx < S * S) {
                const int ar = idx / S, b = idx - ar * S;
#pragma unroll 4
                for (int i = 0; i < S; ++i) a += Y[ar * LDA + i] * X[i * LDA + b];
            }
            acc[e] = a;
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NE1; ++e) {
            const int idx = lane + LW * e;
            if (idx < S * S) X[(idx / S) * LDA + idx % S] = acc[e];
        }
        __syncwarp();
    }

    // v <- rows of the stored s x s eigenvector matrix (row-major at Vc), padded
    // with the identity on indices s..S-1.
    __device__ __forceinline__ void load_basis(const T* __restrict__ Vc, int s, int lane) {
#pragma unroll
        for (int j = 0; j < S; ++j) v[j] = (lane < s && j < s) ? Vc[lane * s + j] : (j == lane ? T(1) : T(0));
    }
    __device__ __forceinline__ void store_basis(T* __restrict__ Vc, int s, int lane) const {
        if (lane < s) {
#pragma unroll
            for (int j = 0; j < S; ++j)
                if (j < s) Vc[lane * s + j] = v[j];
        }
    }

    // One round: A (shared memory) from X into Y with the pair rotations, and
    // V's row from vin into vout (columns re-indexed by sigma).
    __device__ __forceinline__ void round(T tol, int lane, const T (&vin)[S], T (&vout)[S]) {
        T bv[NS][4];
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            if (bI[t] >= 0) {
#pragma unroll
                for (int e = 0; e < 4; ++e) bv[t][e] = X[src[t][e]];
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) bv[t][e] = T(0);
            }
        }
        // rotation of pair `lane` (lanes < K own the diagonal blocks in slot 0):
        // t = sign(zeta) a_pq / (|zeta| + sqrt(zeta^2 + a_pq^2)), zeta = (a_qq - a_pp)/2
        // (Rutishauser's form of the 2x2 Schur step), c = 1/sqrt(1+t^2), s = t c.
        T sn = T(0), tau = T(0), ta = T(0);
        bool my = false;
        if (lane < K) {
            const T apq = bv[0][1];
            if (fabs(apq) > tol) {
                const T zeta = T(0.5) * (bv[0][3] - bv[0][0]);
                const T r2 = zeta * zeta + apq * apq;
                const T r = r2 * rsqrt_t<T>(r2);
                const T tt = copysign(T(1), zeta) * div_t<T>(apq, fabs(zeta) + r);
                const T c = rsqrt_t<T>(T(1) + tt * tt);
                sn = tt * c;
                tau = div_t<T>(sn, T(1) + c);
                ta = tt * apq;
                my = true;
            }
        }
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const int I = bI[t] >= 0 ? bI[t] : 0, J = bJ[t];
            const T sI = __shfl_sync(0xffffffffu, sn, I, LW), uI = __shfl_sync(0xffffffffu, tau, I, LW);
            const T sJ = __shfl_sync(0xffffffffu, sn, J, LW), uJ = __shfl_sync(0xffffffffu, tau, J, LW);
            if (bI[t] < 0) continue;
            if (t == 0 && lane < K) {  // diagonal block: the 2x2 Schur result
                Y[dst[t][0]] = bv[t][0] - ta;
                Y[dst[t][1]] = my ? T(0) : bv[t][1];
                Y[dst[t][3]] = bv[t][3] + ta;
            } else {  // J_I^T B J_J, rows then columns, in the tau form
                const T r00 = bv[t][0] - sI * (bv[t][1] + uI * bv[t][0]);
                const T r10 = bv[t][1] + sI * (bv[t][0] - uI * bv[t][1]);
                const T r01 = bv[t][2] - sI * (bv[t][3] + uI * bv[t][2]);
                const T r11 = bv[t][3] + sI * (bv[t][2] - uI * bv[t][3]);
                Y[dst[t][0]] = r00 - sJ * (r01 + uJ * r00);
                Y[dst[t][2]] = r01 + sJ * (r00 - uJ * r01);
                Y[dst[t][1]] = r10 - sJ * (r11 + uJ * r10);
                Y[dst[t][3]] = r11 + sJ * (r10 - uJ * r11);
            }
        }
        // V <- V J on this lane's row, then re-index its columns by sigma like A
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T sk = __shfl_sync(0xffffffffu, sn, k, LW), uk = __shfl_sync(0xffffffffu, tau, k, LW);
            const T vp = vin[2 * k], vq = vin[2 * k + 1];
            vout[RR::sigma(2 * k)] = vp - sk * (vq + uk * vp);
            vout[RR::sigma(2 * k + 1)] = vq + sk * (vp - uk * vq);
        }
        __syncwarp();
        T* tmp = X; X = Y; Y = tmp;
    }

    // Diagonalise; returns the number of sweeps run.  Afterwards X holds
    // diag(lambda) (up to the threshold) and v the eigenvector row.  With
    // v_preset the sweeps start from the basis already in v (see
    // rotate_into_basis); otherwise from the identity.  A sweep runs only while
    // some off-diagonal entry exceeds tol.
    //
    // With LW < 32 the warp serves 32 / LW cliques, one per group of LW lanes;
    // the sweep loop runs while any group still sweeps, and a group that has
    // stopped (or is inactive) goes through the remaining rounds with every
    // rotation skipped (threshold +inf): its storage order returns to the
    // identity after each sweep and its matrix and V stay as they were, so each
    // clique's result is the one it gets alone.
    __device__ int run(T tol, int max_sweeps, int lane, bool v_preset = false, bool active = true) {
        const T noise = tol * T(2 * S);  // 4 S u ||W||_F when tol = 2 u ||W||_F
        if (!v_preset) {
#pragma unroll
            for (int j = 0; j < S; ++j) v[j] = (j == lane) ? T(1) : T(0);
        }
        __syncwarp();
        int sw = 0;
        T w[S];
        T prev = T(3.0e38);
        bool go = active;
        while (true) {
            const T off = off_max(lane);
            if (go && (sw >= max_sweeps || off <= tol || (off <= noise && off > T(0.5) * prev)))
                go = false;  // converged, or stagnated at the rounding-noise level
            if (!__any_sync(0xffffffffu, go)) break;
            prev = off;
            if (go) ++sw;
            const T t_eff = go ? tol : T(INFINITY);
            // rounds in pairs, V ping-ponging between v and w (R = S - 1 is odd)
#pragma unroll 1
            for (int r = 0; r + 1 < R; r += 2) {
                round(t_eff, lane, v, w);
                round(t_eff, lane, w, v);
            }
            round(t_eff, lane, v, w);
#pragma unroll
            for (int j = 0; j < S; ++j) v[j] = w[j];
        }
        return sw;
    }

    // Write V max(Lambda, 0) (into Y) and V (into X) row by row for rebuild().
    __device__ __forceinline__ void prepare_rebuild(int lane) {
        T lp[S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const T l = X[i * LDA + i];
            lp[i] = l > T(0) ? l : T(0);
        }
        __syncwarp();
        if (lane < S) {
#pragma unroll
            for (int i = 0; i < S; ++i) {
                Y[lane * LDA + i] = v[i] * lp[i];
                X[lane * LDA + i] = v[i];
            }
        }
        __syncwarp();
    }
    __device__ __forceinline__ void eigenvalues_to(T* lam_out, int s, int lane) const {
        // only valid before prepare_rebuild()
        if (lane < s) lam_out[lane] = X[lane * LDA + lane];
    }
    // (V max(Lambda,0) V^T)_{ab}, s active indices
    __device__ __forceinline__ T rebuild(int a, int b, int s) const {
        const T* ya = Y + a * LDA;
        const T* xb = X + b * LDA;
        T acc = T(0);
        for (int i = 0; i < s; ++i) acc += ya[i] * xb[i];
        return acc;
    }
};

// ---------------------------------------------------------------------------
// Algorithm 1, projection and multiplier step for every clique in `list`:
//   W = H_k x - lambda_k / rho,  x_k <- P(W),  lambda_k <- lambda_k + rho (x_k - H_k x)
// (Eqs. XkUpdate, LambdakUpdate).  x comes from k_xupd (pa.x_ready, the
// default) or is formed here on the clique's entries,
//   x_e = t_e - (A^T y)_e / D_e (Appendix A, Eq. KKTflops_s1),
// the first clique covering an entry storing it.  That clique also adds the
// entry's term of <c, x>.  Per-block sums of the stopping test (Eq.
// PrimalConsensusResidual and eps_lambda) go to the partial table:
//   |x_k - H_k x|^2, |x_k|^2, |H_k x|^2, |x_k - x_k_old|^2, |lambda_k|^2, <c, x>.
template <typename T, int S>
__global__ void __launch_bounds__(32 * proj_max_warps(S, sizeof(T) == 4)) k_project_primal(Dev d, const int* __restrict__ list, int nlist, ProjArgs pa,
                                                         FinishArgs fa) {
    constexpr int LW = proj_lanes(S), G = 32 / LW;  // lanes per clique, cliques per warp
    using J = BLJacobi<T, S, LW>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (stopped(d)) return;
    const int lane = (threadIdx.x & 31) % LW, grp = (threadIdx.x & 31) / LW;  // lane within its group
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + (warp * G + grp) * J::bytes, lane);
    T* xk = reinterpret_cast<T*>(d.ck0);
    T* lam = reinterpret_cast<T*>(d.ck1);
    T* vc = reinterpret_cast<T*>(d.vcache);
    const bool warm = pa.warm_start && (d.ctl[CTL_ITER] % pa.restart) != 0;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int li0 = (blockIdx.x * wpb + warp) * G; li0 < nlist; li0 += gridDim.x * wpb * G) {
        // group grp takes clique li0 + grp; a group past the list or on a
        // frozen clique is inactive: it touches no state and skips every rotation
        const int li = li0 + grp;
        const int k = list[li < nlist ? li : li0];
        const bool active = li < nlist && !frozen_clique(d, k);
        const double rho = rho_clique(d, k);
        const T rho_t = T(rho), irho = T(1.0 / rho);
        const int s = active ? d.csize[k] : 0, off = d.pk_off[k], npk = s * (s + 1) / 2;
        jac.clear(lane);
        T nrm = T(0);
        T hx[J::MAXE];
        double cx = 0.0;
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + LW * e;
            hx[e] = T(0);
            if (f < npk) {
                const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
                // read-only loads (__ldg): free to move past this kernel's stores
                const int ent = __ldg(d.gmap + off + f);
                const bool own = __ldg(d.owner + off + f) != 0;
                double xe;
                if (pa.x_ready) {
                    xe = d.x[ent];
                } else {
                    double aty = 0.0;
                    const int q0 = __ldg(d.at_ptr + ent), q1 = __ldg(d.at_ptr + ent + 1);
#pragma unroll 8
                    for (int q = q0; q < q1; ++q) aty += __ldg(d.at_val + q) * __ldg(d.y + __ldg(d.at_col + q));
                    xe = __ldg(d.t + ent) - __ldg(d.dinv + ent) * aty;
                    if (own) d.x[ent] = xe;
                }
                if (own) cx += __ldg(d.wgt + ent) * __ldg(d.c + ent) * xe;
                hx[e] = T(xe);
                const T w = hx[e] - lam[off + f] * irho;
                if (d.wstore) {
                    const int slot = d.ctl[CTL_ITER];
                    if (slot < d.wstore_count) reinterpret_cast<T*>(d.wstore)[(size_t)slot * d.nd + off + f] = w;
                }
                jac.put(a, b, w);
                nrm += (a == b ? T(1) : T(2)) * w * w;
            }
        }
        nrm = group_sum(nrm, LW);
        const double cxk = group_sum(cx, LW);
        __syncwarp();
        if (warm) {
            jac.load_basis(vc + d.vv_off[k], s, lane);
            jac.rotate_into_basis(lane);
        }
        jac.run(T(pa.tolrel) * sqrt(nrm), pa.max_sweeps, lane, warm, active);
        if (pa.warm_start) jac.store_basis(vc + d.vv_off[k], s, lane);
        jac.prepare_rebuild(lane);
        // per-clique sums of the stopping test in the clique state's precision
        // (float32 values; the sums over cliques are float64)
        T p0 = 0, p1 = 0, p2 = 0, p3 = 0, p4 = 0;
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + LW * e;
            if (f < npk) {
                const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
                const T lm = lam[off + f];
                const T xn = jac.rebuild(a, b, s);
                const T xo = xk[off + f];
                const T ln = lm + rho_t * (xn - hx[e]);
                xk[off + f] = xn;
                lam[off + f] = ln;
                const T w = (a == b) ? T(1) : T(2);
                const T dc = xn - hx[e], dx = xn - xo;
                p0 += w * dc * dc;
                p1 += w * xn * xn;
                p2 += w * hx[e] * hx[e];
                p3 += w * dx * dx;
                p4 += w * ln * ln;
            }
        }
        const double q[6] = {double(group_sum(p0, LW)), double(group_sum(p1, LW)), double(group_sum(p2, LW)),
                             double(group_sum(p3, LW)), double(group_sum(p4, LW)), cxk};
        if (d.comp_mode) {  // per-clique row, reduced per component
            if (lane == 0 && active)
#pragma unroll
                for (int c = 0; c < 6; ++c) d.part[(size_t)k * PART_COLS + c] = q[c];
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[c] += q[c];
        }
        __syncwarp();
    }
    if (d.comp_mode) return;
#pragma unroll
    for (int c = 0; c < 6; ++c)
        for (int o = LW; o < 32; o <<= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);  // over the groups
    const int cols[6] = {0, 1, 2, 3, 4, 5};
    block_partial_row<6>(acc, d.part, pa.row_off + blockIdx.x, cols);
    if (fa.enabled && last_block_single_writer(d)) finish_primal_block(d, fa);
}

// Algorithm 2, z-step (Eq. zkUpdate): z_k <- P(v_k - lambda_k / rho);
// part[k][5] = |z_k - z_k_old|^2 (for eps_lambda).
template <typename T, int S>
__global__ void __launch_bounds__(32 * proj_max_warps(S, sizeof(T) == 4)) k_project_dual(Dev d, const int* __restrict__ list, int nlist, ProjArgs pa) {
    constexpr int LW = proj_lanes(S), G = 32 / LW;  // lanes per clique, cliques per warp
    using J = BLJacobi<T, S, LW>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (stopped(d)) return;
    const int lane = (threadIdx.x & 31) % LW, grp = (threadIdx.x & 31) / LW;  // lane within its group
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + (warp * G + grp) * J::bytes, lane);
    T* z = reinterpret_cast<T*>(d.ck0);
    const T* v = reinterpret_cast<const T*>(d.ck1);
    const T* lam = reinterpret_cast<const T*>(d.ck2);
    T* vc = reinterpret_cast<T*>(d.vcache);
    const bool warm = pa.warm_start && (d.ctl[CTL_ITER] % pa.restart) != 0;
    double acc[1] = {0};
    for (int li0 = (blockIdx.x * wpb + warp) * G; li0 < nlist; li0 += gridDim.x * wpb * G) {
        // group grp takes clique li0 + grp; a group past the list or on a
        // frozen clique is inactive: it touches no state and skips every rotation
        const int li = li0 + grp;
        const int k = list[li < nlist ? li : li0];
        const bool active = li < nlist && !frozen_clique(d, k);
        const T irho = T(1.0 / rho_clique(d, k));
        const int s = active ? d.csize[k] : 0, off = d.pk_off[k], npk = s * (s + 1) / 2;
        jac.clear(lane);
        T nrm = T(0);
        for (int f = lane; f < npk; f += LW) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const T w = v[off + f] - lam[off + f] * irho;
            jac.put(a, b, w);
            nrm += (a == b ? T(1) : T(2)) * w * w;
        }
        nrm = group_sum(nrm, LW);
        __syncwarp();
        if (warm) {
            jac.load_basis(vc + d.vv_off[k], s, lane);
            jac.rotate_into_basis(lane);
        }
        jac.run(T(pa.tolrel) * sqrt(nrm), pa.max_sweeps, lane, warm, active);
        if (pa.warm_start) jac.store_basis(vc + d.vv_off[k], s, lane);
        jac.prepare_rebuild(lane);
        T p0 = 0;  // in the clique state's precision; float64 across cliques
        for (int f = lane; f < npk; f += LW) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const T zn = jac.rebuild(a, b, s);
            const T dz = zn - z[off + f];
            z[off + f] = zn;
            p0 += (a == b ? T(1) : T(2)) * dz * dz;
        }
        const double q0 = double(group_sum(p0, LW));
        if (d.comp_mode) {
            if (lane == 0 && active) d.part[(size_t)k * PART_COLS + 5] = q0;
        } else {
            acc[0] += q0;
        }
        __syncwarp();
    }
    if (d.comp_mode) return;
    for (int o = LW; o < 32; o <<= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);  // over the groups
    const int cols[1] = {5};
    block_partial_row<1>(acc, d.part, pa.row_off + blockIdx.x, cols);
}

// Algorithm 3, cone step on the s block (Eqs. HsdeStep2-3) with the pieces of
// the affine step that live on clique entries (Appendix B, Eqs.
// ThirBlkFlops_s2 and AppendixEqSigma2, then Eq. MatrixInverseResult with
// zeta_hat_s = H zeta_hat_x / 2, zeta_hat_t = -H zeta_hat_x / 2):
//   sigma_12 = (nu_12 - nu_22 + H sigma_11)/2,  sigma_22 = nu_22 - H sigma_11 + sigma_12
//   u_hat_s = sigma_12 - gamma zeta_hat_s,      u_hat_t = sigma_22 - gamma zeta_hat_t
//   u_s <- P(u_hat_s - v_z),  v_z <- v_z - u_hat_s + u_s,  u_t <- u_hat_t
// with nu_12 = u_s + v_z, nu_22 = u_t.  Partial sums for eps_c (Eq.
// HSDEconsensusResidual): |u_s - H u_x|^2, |u_s|^2, |H u_x|^2, |v_z - u_t|^2,
// |v_z|^2, |u_t|^2, where u_x = sigma_11 - gamma zeta_hat_x.
template <typename T, int S>
__global__ void __launch_bounds__(32 * proj_max_warps(S, sizeof(T) == 4)) k_project_hsde(Dev d, const int* __restrict__ list, int nlist, ProjArgs pa) {
    constexpr int LW = proj_lanes(S), G = 32 / LW;  // lanes per clique, cliques per warp
    using J = BLJacobi<T, S, LW>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (stopped(d)) return;
    const int lane = (threadIdx.x & 31) % LW, grp = (threadIdx.x & 31) / LW;  // lane within its group
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + (warp * G + grp) * J::bytes, lane);
    T* us = reinterpret_cast<T*>(d.ck0);
    T* vz = reinterpret_cast<T*>(d.ck1);
    T* ut = reinterpret_cast<T*>(d.ck2);
    T* vc = reinterpret_cast<T*>(d.vcache);
    const bool warm = pa.warm_start && (d.ctl[CTL_ITER] % pa.restart) != 0;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int li0 = (blockIdx.x * wpb + warp) * G; li0 < nlist; li0 += gridDim.x * wpb * G) {
        // group grp takes clique li0 + grp; a group past the list or on a
        // frozen clique is inactive: it touches no state and skips every rotation
        const int li = li0 + grp;
        const int k = list[li < nlist ? li : li0];
        const bool active = li < nlist && !frozen_clique(d, k);
        const double gamma = hs_gamma_c(d, comp_k(d, k));
        const int s = active ? d.csize[k] : 0, off = d.pk_off[k], npk = s * (s + 1) / 2;
        jac.clear(lane);
        T nrm = T(0);
        for (int f = lane; f < npk; f += LW) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const int ent = d.gmap[off + f];
            const double hs = d.s11[ent];
            const double zs = 0.5 * d.zhx[ent];
            const double u_s = us[off + f], v_z = vz[off + f], u_t = ut[off + f];
            const double s12 = 0.5 * (u_s + v_z - u_t + hs);
            const double uh_s = s12 - gamma * zs;
            const T w = T(uh_s - v_z);
            jac.put(a, b, w);
            nrm += (a == b ? T(1) : T(2)) * w * w;
        }
        nrm = group_sum(nrm, LW);
        __syncwarp();
        if (warm) {
            jac.load_basis(vc + d.vv_off[k], s, lane);
            jac.rotate_into_basis(lane);
        }
        jac.run(T(pa.tolrel) * sqrt(nrm), pa.max_sweeps, lane, warm, active);
        if (pa.warm_start) jac.store_basis(vc + d.vv_off[k], s, lane);
        jac.prepare_rebuild(lane);
        double p[6] = {0, 0, 0, 0, 0, 0};
        for (int f = lane; f < npk; f += LW) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const int ent = d.gmap[off + f];
            const double hs = d.s11[ent];
            const double zs = 0.5 * d.zhx[ent];
            const double u_s = us[off + f], v_z = vz[off + f], u_t = ut[off + f];
            const double s12 = 0.5 * (u_s + v_z - u_t + hs);
            const double s22 = u_t - hs + s12;
            const T uhs = T(s12 - gamma * zs);
            const T utn = T(s22 + gamma * zs);
            const T hux = T(hs - gamma * d.zhx[ent]);
            const T un = jac.rebuild(a, b, s);
            const T vn = T(v_z) - uhs + un;
            us[off + f] = un;
            vz[off + f] = vn;
            ut[off + f] = utn;
            const double w = (a == b) ? 1.0 : 2.0;
            const double d1 = double(un) - double(hux);
            const double d2 = double(vn) - double(utn);
            p[0] += w * d1 * d1;
            p[1] += w * double(un) * double(un);
            p[2] += w * double(hux) * double(hux);
            p[3] += w * d2 * d2;
            p[4] += w * double(vn) * double(vn);
            p[5] += w * double(utn) * double(utn);
        }
        double q[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] = group_sum(p[c], LW);
        if (d.comp_mode) {  // per-clique row, reduced per component
            if (lane == 0 && active)
#pragma unroll
                for (int c = 0; c < 6; ++c) d.part[(size_t)k * PART_COLS + c] = q[c];
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[c] += q[c];
        }
        __syncwarp();
    }
    if (d.comp_mode) return;
#pragma unroll
    for (int c = 0; c < 6; ++c)
        for (int o = LW; o < 32; o <<= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);  // over the groups
    const int cols[6] = {0, 1, 2, 3, 4, 5};
    block_partial_row<6>(acc, d.part, pa.row_off + blockIdx.x, cols);
}

// Standalone projection of packed blocks (the C ABI's cdsdp_psd_project).
template <typename T, int S>
__global__ void __launch_bounds__(128) k_project_standalone(int p, const int* __restrict__ off_arr,
                                                             const int* __restrict__ size_arr, const T* __restrict__ W,
                                                             T* X, T* eig, const int* __restrict__ voff, T* Vout,
                                                             const int* __restrict__ vvoff, double tolrel,
                                                             int max_sweeps) {
    using J = BLJacobi<T, S>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + warp * J::bytes, lane);
    for (int k = blockIdx.x * wpb + warp; k < p; k += gridDim.x * wpb) {
        const int s = size_arr[k];
        if (s > S || s < 1) continue;  // warp-uniform
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
        if (eig) jac.eigenvalues_to(eig + voff[k], s, lane);
        if (Vout && lane < s) {
#pragma unroll
            for (int col = 0; col < S; ++col)
                if (col < s) Vout[vvoff[k] + col * s + lane] = jac.v[col];
        }
        __syncwarp();
        jac.prepare_rebuild(lane);
        for (int f = lane; f < npk; f += 32) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            X[off + f] = jac.rebuild(a, b, s);
        }
        __syncwarp();
    }
}

}  // namespace cdsdp_dev
