// Batched PSD projection P(W) = V max(Lambda, 0) V^T of clique blocks
// (Section 4.1.2, Eq. XkUpdate; Eq. zkUpdate; Eq. HsdeStep2), one warp per
// block of order s <= 32, block held in shared memory.
//
// Eigensolver: two-sided parallel Jacobi (Jacobi 1846; parallel round-robin
// ordering of Brent and Luk 1985; 2x2 symmetric Schur step of Golub and Van
// Loan, Matrix Computations, Section 8.5).  In each round every index is
// paired with at most one partner (pairs {i, j} with i + j = 2r mod (S-1),
// index r with the extra index S-1, S = s rounded up to even), so the s/2
// rotations of a round commute and are applied together:
//   A <- J^T A J,  V <- V J,
// each new element of A mixing the four old elements of its two pairs.
// A rotation is skipped when |a_pq| <= tol = eps_rel * ||W||_F; the sweeps end
// when a whole sweep skips every rotation (or after max_sweeps).
#pragma once

#include "kernels.cuh"

namespace cdsdp_dev {

template <typename T, int MAXS>
struct WarpTile {
    static constexpr int LD = MAXS | 1;  // odd stride: conflict-free column walks
    static constexpr int NPK = MAXS * (MAXS + 1) / 2;
    static constexpr int MAXE = (NPK + 31) / 32;  // packed elements per lane
    static constexpr int NT = 2 * MAXS * LD + 3 * 32;
    static constexpr size_t bytes = ((NT * sizeof(T) + 32 * sizeof(int)) + 15) & ~size_t(15);
};

// (a, b) of packed element f of an s x s block, a >= b, column-major.
__device__ __forceinline__ int packed_ab(int f, int s) {
    int b = 0, rem = f;
    while (rem >= s - b) { rem -= s - b; ++b; }
    return ((b + rem) << 8) | b;
}

template <typename T, int MAXS>
struct WarpJacobi {
    using Tile = WarpTile<T, MAXS>;
    static constexpr int LD = Tile::LD;
    static constexpr int MAXE = Tile::MAXE;
    T* A;
    T* V;
    T* rc;   // per index: coefficient on itself (cosine)
    T* rsg;  // per index: coefficient on its partner (signed sine)
    T* rd;   // per index: change of its diagonal entry (Schur step)
    int* rp; // per index: partner (itself when not rotated)

    __device__ __forceinline__ void bind(unsigned char* base) {
        A = reinterpret_cast<T*>(base);
        V = A + MAXS * LD;
        rc = V + MAXS * LD;
        rsg = rc + 32;
        rd = rsg + 32;
        rp = reinterpret_cast<int*>(rd + 32);
    }

    // Diagonalise the symmetric block in A (s x s); V receives the
    // eigenvectors (columns).  `ab` holds this lane's packed elements.
    // Returns the number of sweeps run.
    __device__ int run(int s, int npk, T tol, int max_sweeps, int lane, const int (&ab)[MAXE]) {
        for (int idx = lane; idx < s * LD; idx += 32) {
            int i = idx / LD, j = idx - i * LD;
            V[idx] = (i == j) ? T(1) : T(0);
        }
        __syncwarp();
        if (s <= 1) return 0;
        const int S2 = (s + 1) & ~1, R = S2 - 1;
        int sweep = 0;
        for (; sweep < max_sweeps; ++sweep) {
            bool sweep_any = false;
            for (int r = 0; r < R; ++r) {
                bool my_rot = false;
                if (lane < s) {
                    const int i = lane;
                    const int j = (i == R) ? r : (i == r ? R : ((2 * r - i) % R + R) % R);
                    if (j >= s) {
                        rc[i] = T(1); rsg[i] = T(0); rd[i] = T(0); rp[i] = i;
                    } else if (i < j) {
                        const T aij = A[i * LD + j];
                        if (fabs(aij) > tol) {
                            const T aii = A[i * LD + i], ajj = A[j * LD + j];
                            const T theta = (ajj - aii) / (T(2) * aij);
                            const T tt = copysign(T(1), theta) / (fabs(theta) + sqrt(T(1) + theta * theta));
                            const T cc = rsqrt_t<T>(T(1) + tt * tt);
                            const T sn = tt * cc;
                            rc[i] = cc; rc[j] = cc;
                            rsg[i] = -sn; rsg[j] = sn;
                            rd[i] = -tt * aij; rd[j] = tt * aij;
                            rp[i] = j; rp[j] = i;
                            my_rot = true;
                        } else {
                            rc[i] = T(1); rc[j] = T(1); rsg[i] = T(0); rsg[j] = T(0);
                            rd[i] = T(0); rd[j] = T(0); rp[i] = i; rp[j] = j;
                        }
                    }
                }
                const bool any = __any_sync(0xffffffffu, my_rot);
                __syncwarp();
                if (!any) continue;
                sweep_any = true;
                T nv[MAXE];
#pragma unroll
                for (int e = 0; e < MAXE; ++e) {
                    const int f = lane + 32 * e;
                    nv[e] = T(0);
                    if (f < npk) {
                        const int a = ab[e] >> 8, b = ab[e] & 255;
                        if (a == b) {
                            nv[e] = A[a * LD + a] + rd[a];
                        } else {
                            const int pa = rp[a], pb = rp[b];
                            if (pa == b) {
                                nv[e] = T(0);  // the rotated pair's off-diagonal entry
                            } else {
                                const T ca = rc[a], sa = rsg[a], cb = rc[b], sb = rsg[b];
                                nv[e] = ca * (cb * A[a * LD + b] + sb * A[a * LD + pb]) +
                                        sa * (cb * A[pa * LD + b] + sb * A[pa * LD + pb]);
                            }
                        }
                    }
                }
                if (lane < s) {  // V <- V J, lane owns row `lane`
                    T* vr = V + lane * LD;
                    for (int i = 0; i < s; ++i) {
                        const int j = rp[i];
                        if (j > i) {
                            const T vi = vr[i], vj = vr[j];
                            vr[i] = rc[i] * vi + rsg[i] * vj;
                            vr[j] = rc[j] * vj + rsg[j] * vi;
                        }
                    }
                }
                __syncwarp();
#pragma unroll
                for (int e = 0; e < MAXE; ++e) {
                    const int f = lane + 32 * e;
                    if (f < npk) {
                        const int a = ab[e] >> 8, b = ab[e] & 255;
                        A[a * LD + b] = nv[e];
                        A[b * LD + a] = nv[e];
                    }
                }
                __syncwarp();
            }
            if (!sweep_any) break;
        }
        return sweep;
    }

    // After run(): rc[i] <- max(lambda_i, 0) for the rebuild.
    __device__ __forceinline__ void prepare_rebuild(int s, int lane) {
        if (lane < s) rc[lane] = A[lane * LD + lane] > T(0) ? A[lane * LD + lane] : T(0);
        __syncwarp();
    }
    // (V max(Lambda,0) V^T)_{ab}
    __device__ __forceinline__ T rebuild(int a, int b, int s) const {
        const T* va = V + a * LD;
        const T* vb = V + b * LD;
        T acc = T(0);
        for (int i = 0; i < s; ++i) acc += va[i] * rc[i] * vb[i];
        return acc;
    }
};

// ---------------------------------------------------------------------------
// Algorithm 1, projection and multiplier step for every clique in `list`:
//   W = H_k x - lambda_k / rho,  x_k <- P(W),  lambda_k <- lambda_k + rho (x_k - H_k x)
// (Eqs. XkUpdate, LambdakUpdate), with the per-clique sums of the stopping
// test (Eq. PrimalConsensusResidual and eps_lambda):
//   part[k] = (|x_k - H_k x|^2, |x_k|^2, |H_k x|^2, |x_k - x_k_old|^2, |lambda_k|^2)
template <typename T, int MAXS>
__global__ void __launch_bounds__(128) k_project_primal(Dev d, const int* __restrict__ list, int nlist, double rho,
                                                         double tolrel, int max_sweeps) {
    using J = WarpJacobi<T, MAXS>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (stopped(d)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + warp * WarpTile<T, MAXS>::bytes);
    T* xk = reinterpret_cast<T*>(d.ck0);
    T* lam = reinterpret_cast<T*>(d.ck1);
    const T rho_t = T(rho), irho = T(1.0 / rho);
    for (int li = blockIdx.x * wpb + warp; li < nlist; li += gridDim.x * wpb) {
        const int k = list[li];
        const int s = d.csize[k], off = d.pk_off[k], npk = s * (s + 1) / 2;
        int ab[J::MAXE];
        T hx[J::MAXE], lm[J::MAXE];
        T nrm = T(0);
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            ab[e] = 0; hx[e] = T(0); lm[e] = T(0);
            if (f < npk) {
                ab[e] = packed_ab(f, s);
                const int a = ab[e] >> 8, b = ab[e] & 255;
                hx[e] = T(d.x[d.gmap[off + f]]);
                lm[e] = lam[off + f];
                const T w = hx[e] - lm[e] * irho;
                jac.A[a * J::LD + b] = w;
                jac.A[b * J::LD + a] = w;
                nrm += (a == b ? T(1) : T(2)) * w * w;
            }
        }
        nrm = warp_sum(nrm);
        __syncwarp();
        jac.run(s, npk, T(tolrel) * sqrt(nrm), max_sweeps, lane, ab);
        jac.prepare_rebuild(s, lane);
        double p0 = 0, p1 = 0, p2 = 0, p3 = 0, p4 = 0;
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            if (f < npk) {
                const int a = ab[e] >> 8, b = ab[e] & 255;
                const T xn = jac.rebuild(a, b, s);
                const T xo = xk[off + f];
                const T ln = lm[e] + rho_t * (xn - hx[e]);
                xk[off + f] = xn;
                lam[off + f] = ln;
                const double w = (a == b) ? 1.0 : 2.0;
                const double dc = double(xn) - double(hx[e]), dx = double(xn) - double(xo);
                p0 += w * dc * dc;
                p1 += w * double(xn) * double(xn);
                p2 += w * double(hx[e]) * double(hx[e]);
                p3 += w * dx * dx;
                p4 += w * double(ln) * double(ln);
            }
        }
        p0 = warp_sum(p0); p1 = warp_sum(p1); p2 = warp_sum(p2); p3 = warp_sum(p3); p4 = warp_sum(p4);
        if (lane == 0) {
            double* pk = d.part + (size_t)k * PART_COLS;
            pk[0] = p0; pk[1] = p1; pk[2] = p2; pk[3] = p3; pk[4] = p4;
        }
        __syncwarp();
    }
}

// Algorithm 2, z-step (Eq. zkUpdate): z_k <- P(v_k - lambda_k / rho);
// part[k][0] = |z_k - z_k_old|^2 (for eps_lambda).
template <typename T, int MAXS>
__global__ void __launch_bounds__(128) k_project_dual(Dev d, const int* __restrict__ list, int nlist, double rho,
                                                       double tolrel, int max_sweeps) {
    using J = WarpJacobi<T, MAXS>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (stopped(d)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + warp * WarpTile<T, MAXS>::bytes);
    T* z = reinterpret_cast<T*>(d.ck0);
    const T* v = reinterpret_cast<const T*>(d.ck1);
    const T* lam = reinterpret_cast<const T*>(d.ck2);
    const T irho = T(1.0 / rho);
    for (int li = blockIdx.x * wpb + warp; li < nlist; li += gridDim.x * wpb) {
        const int k = list[li];
        const int s = d.csize[k], off = d.pk_off[k], npk = s * (s + 1) / 2;
        int ab[J::MAXE];
        T nrm = T(0);
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            ab[e] = 0;
            if (f < npk) {
                ab[e] = packed_ab(f, s);
                const int a = ab[e] >> 8, b = ab[e] & 255;
                const T w = v[off + f] - lam[off + f] * irho;
                jac.A[a * J::LD + b] = w;
                jac.A[b * J::LD + a] = w;
                nrm += (a == b ? T(1) : T(2)) * w * w;
            }
        }
        nrm = warp_sum(nrm);
        __syncwarp();
        jac.run(s, npk, T(tolrel) * sqrt(nrm), max_sweeps, lane, ab);
        jac.prepare_rebuild(s, lane);
        double p0 = 0;
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            if (f < npk) {
                const int a = ab[e] >> 8, b = ab[e] & 255;
                const T zn = jac.rebuild(a, b, s);
                const double dz = double(zn) - double(z[off + f]);
                z[off + f] = zn;
                p0 += (a == b ? 1.0 : 2.0) * dz * dz;
            }
        }
        p0 = warp_sum(p0);
        if (lane == 0) d.part[(size_t)k * PART_COLS + 5] = p0;
        __syncwarp();
    }
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
template <typename T, int MAXS>
__global__ void __launch_bounds__(128) k_project_hsde(Dev d, const int* __restrict__ list, int nlist,
                                                       double tolrel, int max_sweeps) {
    using J = WarpJacobi<T, MAXS>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (stopped(d)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + warp * WarpTile<T, MAXS>::bytes);
    T* us = reinterpret_cast<T*>(d.ck0);
    T* vz = reinterpret_cast<T*>(d.ck1);
    T* ut = reinterpret_cast<T*>(d.ck2);
    const double gamma = d.scal[SC_GAMMA];
    for (int li = blockIdx.x * wpb + warp; li < nlist; li += gridDim.x * wpb) {
        const int k = list[li];
        const int s = d.csize[k], off = d.pk_off[k], npk = s * (s + 1) / 2;
        int ab[J::MAXE];
        T uhs[J::MAXE], vzo[J::MAXE], hux[J::MAXE], utn[J::MAXE];
        T nrm = T(0);
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            ab[e] = 0; uhs[e] = T(0); vzo[e] = T(0); hux[e] = T(0); utn[e] = T(0);
            if (f < npk) {
                ab[e] = packed_ab(f, s);
                const int a = ab[e] >> 8, b = ab[e] & 255;
                const int ent = d.gmap[off + f];
                const double hs = d.s11[ent];
                const double zs = 0.5 * d.zhx[ent];
                const double u_s = us[off + f], v_z = vz[off + f], u_t = ut[off + f];
                const double nu12 = u_s + v_z, nu22 = u_t;
                const double s12 = 0.5 * (nu12 - nu22 + hs);
                const double s22 = nu22 - hs + s12;
                const double uh_s = s12 - gamma * zs;
                const double uh_t = s22 + gamma * zs;
                uhs[e] = T(uh_s);
                vzo[e] = T(v_z);
                utn[e] = T(uh_t);
                hux[e] = T(hs - gamma * d.zhx[ent]);
                const T w = T(uh_s - v_z);
                jac.A[a * J::LD + b] = w;
                jac.A[b * J::LD + a] = w;
                nrm += (a == b ? T(1) : T(2)) * w * w;
            }
        }
        nrm = warp_sum(nrm);
        __syncwarp();
        jac.run(s, npk, T(tolrel) * sqrt(nrm), max_sweeps, lane, ab);
        jac.prepare_rebuild(s, lane);
        double p[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            if (f < npk) {
                const int a = ab[e] >> 8, b = ab[e] & 255;
                const T un = jac.rebuild(a, b, s);
                const T vn = vzo[e] - uhs[e] + un;
                us[off + f] = un;
                vz[off + f] = vn;
                ut[off + f] = utn[e];
                const double w = (a == b) ? 1.0 : 2.0;
                const double d1 = double(un) - double(hux[e]);
                const double d2 = double(vn) - double(utn[e]);
                p[0] += w * d1 * d1;
                p[1] += w * double(un) * double(un);
                p[2] += w * double(hux[e]) * double(hux[e]);
                p[3] += w * d2 * d2;
                p[4] += w * double(vn) * double(vn);
                p[5] += w * double(utn[e]) * double(utn[e]);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) p[c] = warp_sum(p[c]);
        if (lane == 0) {
            double* pk = d.part + (size_t)k * PART_COLS;
#pragma unroll
            for (int c = 0; c < 6; ++c) pk[c] = p[c];
        }
        __syncwarp();
    }
}

// Standalone projection of packed blocks (the C ABI's cdsdp_psd_project).
template <typename T, int MAXS>
__global__ void __launch_bounds__(128) k_project_standalone(int p, const int* __restrict__ off_arr,
                                                             const int* __restrict__ size_arr, const T* __restrict__ W,
                                                             T* X, T* eig, const int* __restrict__ voff, T* Vout,
                                                             const int* __restrict__ vvoff, double tolrel,
                                                             int max_sweeps) {
    using J = WarpJacobi<T, MAXS>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + warp * WarpTile<T, MAXS>::bytes);
    for (int k = blockIdx.x * wpb + warp; k < p; k += gridDim.x * wpb) {
        const int s = size_arr[k];
        if (s > MAXS || s < 1) continue;
        const int off = off_arr[k], npk = s * (s + 1) / 2;
        int ab[J::MAXE];
        T nrm = T(0);
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            ab[e] = 0;
            if (f < npk) {
                ab[e] = packed_ab(f, s);
                const int a = ab[e] >> 8, b = ab[e] & 255;
                const T w = W[off + f];
                jac.A[a * J::LD + b] = w;
                jac.A[b * J::LD + a] = w;
                nrm += (a == b ? T(1) : T(2)) * w * w;
            }
        }
        nrm = warp_sum(nrm);
        __syncwarp();
        jac.run(s, npk, T(tolrel) * sqrt(nrm), max_sweeps, lane, ab);
        if (eig && lane < s) eig[voff[k] + lane] = jac.A[lane * J::LD + lane];
        if (Vout)
            for (int idx = lane; idx < s * s; idx += 32) {
                const int col = idx / s, row = idx - col * s;
                Vout[vvoff[k] + idx] = jac.V[row * J::LD + col];
            }
        jac.prepare_rebuild(s, lane);
#pragma unroll
        for (int e = 0; e < J::MAXE; ++e) {
            const int f = lane + 32 * e;
            if (f < npk) {
                const int a = ab[e] >> 8, b = ab[e] & 255;
                X[off + f] = jac.rebuild(a, b, s);
            }
        }
        __syncwarp();
    }
}

}  // namespace cdsdp_dev
