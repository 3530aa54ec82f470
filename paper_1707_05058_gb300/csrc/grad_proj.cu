// Adjoint of the batched PSD projection (Daleckii-Krein form), one warp per
// clique of order <= 32.  Not in the paper: the derivative of
// P(W) = V max(Lambda, 0) V^T at W = V Lambda V^T in direction E is
//   V (Gamma o (V^T E V)) V^T,  Gamma_ij = (f(l_i) - f(l_j)) / (l_i - l_j),
//   f = max(., 0), Gamma_ij = f'(l_i) (1, 0, or 1/2 at 0) when l_i == l_j
// (Daleckii and Krein 1965; Bhatia, Matrix Analysis, Thm V.3.3).  It is
// self-adjoint in the Frobenius inner product, so the vector-Jacobian product
// of a symmetric cotangent G is the same expression with E = G.
//
// In the lower-packed coordinates of the solver (off-diagonal entries stand
// for two matrix entries) the packed cotangent g maps to G = unpack(g / w) and
// the packed adjoint of W is w o pack(DK(G)), w = 1 on the diagonal, 2 off it.
#include "grad_launch.h"
#include "jacobi.cuh"

namespace cdsdp_dev {
namespace {

// For every clique of `list` at reverse iteration `slot`:
//   g   = xkbar + rho lambar                       (adjoint of x_k' in total)
//   Wbar = w o pack(DK_W(unpack(g / w)))           (W from the recorded forward)
//   hxbar  <- Wbar - rho lambar
//   lamprev <- lambar - Wbar / rho
template <typename T, int S>
__global__ void __launch_bounds__(128) k_bwd_proj(Dev d, const int* __restrict__ list, int nlist, GradArgs ga) {
    using J = BLJacobi<T, S>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    J jac;
    jac.bind(smem + warp * J::bytes, lane);
    const T* Wrec = reinterpret_cast<const T*>(d.wstore) + (size_t)ga.slot * d.nd;
    const double rho = ga.rho;
    for (int li = blockIdx.x * wpb + warp; li < nlist; li += gridDim.x * wpb) {
        const int k = list[li];
        const int s = d.csize[k], off = d.pk_off[k], npk = s * (s + 1) / 2;
        jac.clear(lane);
        T nrm = T(0);
        for (int f = lane; f < npk; f += 32) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const T w = Wrec[off + f];
            jac.put(a, b, w);
            nrm += (a == b ? T(1) : T(2)) * w * w;
        }
        nrm = warp_sum(nrm);
        __syncwarp();
        jac.run(T(ga.tolrel) * sqrt(nrm), ga.max_sweeps, lane, false);
        const T lam_lane = lane < S ? jac.X[lane * J::LDA + lane] : T(0);
        jac.clear(lane);
        if (lane < S) jac.Y[lane * J::LDA + S] = lam_lane;  // padding column: survives the congruences
        for (int f = lane; f < npk; f += 32) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const double g = ga.xkbar[off + f] + rho * ga.lambar[off + f];
            jac.put(a, b, T(a == b ? g : 0.5 * g));
        }
        __syncwarp();
        jac.rotate_into_basis(lane);  // X = V^T G V
        for (int idx = lane; idx < S * S; idx += 32) {
            const int i = idx / S, j = idx - i * S;
            const T li = jac.Y[i * J::LDA + S], lj = jac.Y[j * J::LDA + S];
            const T fi = li > T(0) ? li : T(0), fj = lj > T(0) ? lj : T(0);
            T gam;
            if (li == lj) gam = li > T(0) ? T(1) : (li < T(0) ? T(0) : T(0.5));
            else gam = (fi - fj) / (li - lj);
            jac.X[i * J::LDA + j] *= gam;
        }
        __syncwarp();
        jac.rotate_out_of_basis(lane);  // X = V (Gamma o V^T G V) V^T
        for (int f = lane; f < npk; f += 32) {
            const int ab = packed_ab(f, s), a = ab >> 8, b = ab & 255;
            const double wbar = (a == b ? 1.0 : 2.0) * double(jac.X[a * J::LDA + b]);
            const double lb = ga.lambar[off + f];
            ga.hxbar[off + f] = wbar - rho * lb;
            ga.lamprev[off + f] = lb - wbar / rho;
        }
        __syncwarp();
    }
}

template <typename T, int S>
cudaError_t launch_bwd(const Dev& d, const int* list, int nlist, const GradArgs& ga, cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    const size_t smem = 4 * BLJacobi<T, S>::bytes;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_bwd_proj<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    GradArgs g = ga;
    g.tolrel = jacobi_tolrel(S, sizeof(T) == 4);
    const int grid = nlist < 4 * 152 * 32 ? (nlist + 3) / 4 : 152 * 32;
    k_bwd_proj<T, S><<<grid, 128, smem, st>>>(d, list, nlist, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_bwd(int cls, const Dev& d, const int* list, int nlist, const GradArgs& ga, cudaStream_t st) {
    switch (kProjClasses[cls]) {
        case 2: return launch_bwd<T, 2>(d, list, nlist, ga, st);
        case 4: return launch_bwd<T, 4>(d, list, nlist, ga, st);
        case 6: return launch_bwd<T, 6>(d, list, nlist, ga, st);
        case 8: return launch_bwd<T, 8>(d, list, nlist, ga, st);
        case 10: return launch_bwd<T, 10>(d, list, nlist, ga, st);
        case 12: return launch_bwd<T, 12>(d, list, nlist, ga, st);
        case 14: return launch_bwd<T, 14>(d, list, nlist, ga, st);
        case 16: return launch_bwd<T, 16>(d, list, nlist, ga, st);
        case 20: return launch_bwd<T, 20>(d, list, nlist, ga, st);
        case 24: return launch_bwd<T, 24>(d, list, nlist, ga, st);
        case 28: return launch_bwd<T, 28>(d, list, nlist, ga, st);
        case 32: return launch_bwd<T, 32>(d, list, nlist, ga, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_bwd_proj(bool fp32, int cls, const Dev& d, const int* list, int nlist, const GradArgs& ga,
                            cudaStream_t st) {
    return fp32 ? dispatch_bwd<float>(cls, d, list, nlist, ga, st) : dispatch_bwd<double>(cls, d, list, nlist, ga, st);
}

}  // namespace cdsdp_dev
