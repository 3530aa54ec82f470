// The projection step of Algorithms 1-3 for cliques of order > 128 (FP32
// clique state): the per-entry work of the thread-block projection kernels
// (jacobi_cta.cuh), with the eigensolve replaced by the tensor-core sign
// iteration of large.cu on dense copies of the blocks.
//   gather   W_k of the form (Eq. XkUpdate / zkUpdate / HsdeStep2 inputs) into
//            the dense (hi, lo) buffer, both triangles;
//   ns_scale_and_iterate   P_k = (W_k + W_k sign(W_k)) / 2;
//   update   the clique state of the form from P_k and per-chunk partial sums
//            of the stopping tests;
//   reduce   per clique, the chunk sums in a fixed order into its row of the
//            partial table; for Algorithm 1 the last block runs the test.
#include <cuda_runtime.h>

#include "large_launch.h"
#include "reduce.cuh"

namespace cdsdp_large {
namespace {

using cdsdp_dev::Dev;
using cdsdp_dev::FinishArgs;

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// (a, b), a >= b, of packed (lower, column-major) element f of an s x s block.
__device__ __forceinline__ void packed_ab64(long long f, int s, int& a, int& b) {
    const double t = 2.0 * s + 1.0;
    int bb = (int)((t - sqrt(t * t - 8.0 * (double)f)) * 0.5);
    bb = max(0, min(bb, s - 1));
    while (bb > 0 && (long long)bb * (2 * s - bb + 1) / 2 > f) --bb;
    while (bb + 1 < s && (long long)(bb + 1) * (2 * s - bb) / 2 <= f) ++bb;
    b = bb;
    a = bb + (int)(f - (long long)bb * (2 * s - bb + 1) / 2);
}

struct Step {
    const Block* blocks;
    const int* list;     // clique of each block
    const int* upd;      // chunk offsets per block
    double* part;        // [chunks * 8] chunk partial sums
    float* Wh;
    float* Wl;
    const float* P;      // dense P (BUF_X2 hi)
};

template <int FORM>
__global__ void __launch_bounds__(256) k_large_gather(Dev d, Step t) {
    const int i = blockIdx.y;
    const int k = t.list[i];
    if (cdsdp_dev::stopped(d) || cdsdp_dev::frozen_clique(d, k)) return;
    if ((int)blockIdx.x >= t.upd[i + 1] - t.upd[i]) return;
    const Block B = t.blocks[i];
    const long long npk = (long long)B.s * (B.s + 1) / 2;
    const long long f0 = (long long)blockIdx.x * kUpdChunk, f1 = min(npk, f0 + kUpdChunk);
    const int off = d.pk_off[k];
    const float* c0 = reinterpret_cast<const float*>(d.ck0);
    const float* c1 = reinterpret_cast<const float*>(d.ck1);
    const float* c2 = reinterpret_cast<const float*>(d.ck2);
    const double irho = (FORM == 2) ? 1.0 : 1.0 / cdsdp_dev::rho_clique(d, k);
    const double gamma = FORM == 2 ? cdsdp_dev::hs_gamma_c(d, cdsdp_dev::comp_k(d, k)) : 0.0;
    for (long long f = f0 + threadIdx.x; f < f1; f += blockDim.x) {
        int a, b;
        packed_ab64(f, B.s, a, b);
        double w;
        if (FORM == 0) {         // H_k x - lambda_k / rho (x from its own kernel)
            w = d.x[d.gmap[off + f]] - double(c1[off + f]) * irho;
        } else if (FORM == 1) {  // v_k - lambda_k / rho
            w = double(c1[off + f]) - double(c2[off + f]) * irho;
        } else {                 // u_hat_s - v_z with sigma_12 of Appendix B
            const int ent = d.gmap[off + f];
            const double s12 = 0.5 * (double(c0[off + f]) + double(c1[off + f]) - double(c2[off + f]) + d.s11[ent]);
            w = s12 - gamma * 0.5 * d.zhx[ent] - double(c1[off + f]);
        }
        const float wf = float(w);
        const float h = tf32_rn(wf), l = wf - h;
        t.Wh[B.off + (long long)a * B.S + b] = h;
        t.Wl[B.off + (long long)a * B.S + b] = l;
        t.Wh[B.off + (long long)b * B.S + a] = h;
        t.Wl[B.off + (long long)b * B.S + a] = l;
    }
}

template <int FORM>
__global__ void __launch_bounds__(256) k_large_update(Dev d, Step t) {
    const int i = blockIdx.y;
    const int k = t.list[i];
    if (cdsdp_dev::stopped(d) || cdsdp_dev::frozen_clique(d, k)) return;
    if ((int)blockIdx.x >= t.upd[i + 1] - t.upd[i]) return;
    const Block B = t.blocks[i];
    const long long npk = (long long)B.s * (B.s + 1) / 2;
    const long long f0 = (long long)blockIdx.x * kUpdChunk, f1 = min(npk, f0 + kUpdChunk);
    const int off = d.pk_off[k];
    float* c0 = reinterpret_cast<float*>(d.ck0);
    float* c1 = reinterpret_cast<float*>(d.ck1);
    float* c2 = reinterpret_cast<float*>(d.ck2);
    const double rho = (FORM == 0 || FORM == 1) ? cdsdp_dev::rho_clique(d, k) : 1.0;
    const double gamma = FORM == 2 ? cdsdp_dev::hs_gamma_c(d, cdsdp_dev::comp_k(d, k)) : 0.0;
    double p[6] = {0, 0, 0, 0, 0, 0};
    for (long long f = f0 + threadIdx.x; f < f1; f += blockDim.x) {
        int a, b;
        packed_ab64(f, B.s, a, b);
        const float xn = t.P[B.off + (long long)a * B.S + b];
        const double w = (a == b) ? 1.0 : 2.0;
        if (FORM == 0) {  // x_k <- P(W), lambda_k <- lambda_k + rho (x_k - H_k x)
            const int ent = d.gmap[off + f];
            const double hx = d.x[ent];
            const float hxt = float(hx), lm = c1[off + f], xo = c0[off + f];
            const float ln = lm + float(rho) * (xn - hxt);
            c0[off + f] = xn;
            c1[off + f] = ln;
            const double dc = double(xn) - double(hxt), dx = double(xn) - double(xo);
            p[0] += w * dc * dc; p[1] += w * double(xn) * double(xn); p[2] += w * double(hxt) * double(hxt);
            p[3] += w * dx * dx; p[4] += w * double(ln) * double(ln);
            if (d.owner[off + f]) p[5] += d.wgt[ent] * d.c[ent] * hx;
        } else if (FORM == 1) {  // z_k <- P(W); |z_k - z_k_old|^2
            const double dz = double(xn) - double(c0[off + f]);
            c0[off + f] = xn;
            p[0] += w * dz * dz;
        } else {  // u_s <- P(u_hat_s - v_z), v_z <- v_z - u_hat_s + u_s, u_t <- u_hat_t
            const int ent = d.gmap[off + f];
            const double hs = d.s11[ent], zs = 0.5 * d.zhx[ent];
            const double u_s = c0[off + f], v_z = c1[off + f], u_t = c2[off + f];
            const double s12 = 0.5 * (u_s + v_z - u_t + hs);
            const double s22 = u_t - hs + s12;
            const double uhs = s12 - gamma * zs, utn = s22 + gamma * zs;
            const double hux = hs - gamma * d.zhx[ent];
            const double vn = v_z - uhs + double(xn);
            c0[off + f] = xn;
            c1[off + f] = float(vn);
            c2[off + f] = float(utn);
            const double d1 = double(xn) - hux, d2 = vn - utn;
            p[0] += w * d1 * d1; p[1] += w * double(xn) * double(xn); p[2] += w * hux * hux;
            p[3] += w * d2 * d2; p[4] += w * vn * vn; p[5] += w * utn * utn;
        }
    }
    __shared__ double sh[32 * 6];
    cdsdp_dev::block_sum<6>(p, sh);
    if (threadIdx.x == 0) {
        double* q = t.part + (size_t)(t.upd[i] + blockIdx.x) * 8;
        for (int c = 0; c < 6; ++c) q[c] = p[c];
    }
}

template <int FORM>
__global__ void __launch_bounds__(128) k_large_reduce(Dev d, Step t, int row_off, FinishArgs fa) {
    if (cdsdp_dev::stopped(d)) return;
    const int i = blockIdx.x;
    const int k = t.list[i];
    const bool frozen = cdsdp_dev::frozen_clique(d, k);
    if (threadIdx.x == 0 && !frozen) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int c = t.upd[i]; c < t.upd[i + 1]; ++c)
            for (int j = 0; j < 6; ++j) s[j] += t.part[(size_t)c * 8 + j];
        double* pr = d.part + (size_t)(d.comp_mode ? k : row_off + i) * cdsdp_dev::PART_COLS;
        if (FORM == 1) {
            pr[5] = s[0];
        } else {
            for (int j = 0; j < 6; ++j) pr[j] = s[j];
        }
    }
    if (FORM == 0 && fa.enabled) {
        __syncthreads();
        if (cdsdp_dev::last_block_single_writer(d)) cdsdp_dev::finish_primal_block(d, fa);
    }
}

template <int FORM>
cudaError_t run(const Dev& d, const NsLayout& L, unsigned char* base, int row_off, const FinishArgs& fa,
                cudaStream_t st) {
    Step t;
    t.blocks = reinterpret_cast<const Block*>(base + L.o_blocks);
    t.list = reinterpret_cast<const int*>(base + L.o_list);
    t.upd = reinterpret_cast<const int*>(base + L.o_upd);
    t.part = reinterpret_cast<double*>(base + L.o_updpart);
    t.Wh = reinterpret_cast<float*>(base + L.o_buf[2 * BUF_W]);
    t.Wl = reinterpret_cast<float*>(base + L.o_buf[2 * BUF_W + 1]);
    t.P = reinterpret_cast<const float*>(base + L.o_buf[2 * BUF_X2]);
    const dim3 grid(std::max(1, L.max_upd), L.nb);
    k_large_gather<FORM><<<grid, 256, 0, st>>>(d, t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = ns_scale_and_iterate(L, base, st);
    if (e != cudaSuccess) return e;
    k_large_update<FORM><<<grid, 256, 0, st>>>(d, t);
    k_large_reduce<FORM><<<L.nb, 128, 0, st>>>(d, t, row_off, fa);
    return cudaGetLastError();
}

}  // namespace

cudaError_t large_step(int form, const Dev& d, const NsLayout& L, unsigned char* base, int row_off,
                       const FinishArgs& fa, cudaStream_t st) {
    if (L.nb == 0) return cudaSuccess;
    switch (form) {
        case 0: return run<0>(d, L, base, row_off, fa, st);
        case 1: return run<1>(d, L, base, row_off, fa, st);
        default: return run<2>(d, L, base, row_off, fa, st);
    }
}

}  // namespace cdsdp_large
