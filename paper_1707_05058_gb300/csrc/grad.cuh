// Kernels of the reverse pass through unrolled Algorithm 1 that transpose its
// linear steps (plain transposes in the lower-packed coordinates):
//   forward                                   reverse
//   t = D^-1 (H^T(x_k + lambda/rho) - c/rho)  x_k_bar = H s_bar, lambda_bar += H s_bar / rho, c_bar -= s_bar / rho
//   r = A W t - b,  y = Minv r                 t_bar += W A^T r_bar, b_bar -= r_bar, r_bar = Minv y_bar
//   x = t - D^-1 A^T y                         y_bar = -A (D^-1 x_bar), t_bar = x_bar
//   Hx = H x                                   x_bar = x_out_bar + H^T Hx_bar
// with s_bar = D^-1 t_bar.  All in float64.
#pragma once

#include "reduce.cuh"

namespace cdsdp_dev {

// x_bar_e = xout_e + sum_{j in H^T(e)} hxbar_j ;  u_e = x_bar_e / D_e
__global__ void __launch_bounds__(ETHREADS) k_bwd_scatter(Dev d, const double* __restrict__ hxbar,
                                                          const double* __restrict__ xout, double* __restrict__ xbar,
                                                          double* __restrict__ u) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.NE; e += gridDim.x * blockDim.x) {
        double acc = xout ? xout[e] : 0.0;
        for (int j = d.sc_ptr[e]; j < d.sc_ptr[e + 1]; ++j) acc += hxbar[d.sc_idx[j]];
        xbar[e] = acc;
        u[e] = acc * d.dinv[e];
    }
}

// y_bar_i = -(A u)_i  (A unweighted)
__global__ void __launch_bounds__(RTHREADS) k_bwd_ybar(Dev d, const double* __restrict__ u, double* __restrict__ ybar) {
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = w0; i < d.m; i += nw) {
        double s = 0.0;
        for (int q = d.a_ptr[i] + lane; q < d.a_ptr[i + 1]; q += 32) s += d.a_valu[q] * u[d.a_col[q]];
        s = warp_sum(s);
        if (lane == 0) ybar[i] = -s;
    }
}

// r_bar = Minv y_bar ;  b_bar -= r_bar
__global__ void __launch_bounds__(RTHREADS) k_bwd_rbar(Dev d, const double* __restrict__ ybar, double* __restrict__ rbar,
                                                       double* __restrict__ bbar) {
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = w0; i < d.m; i += nw) {
        double s;
        if (d.diag_factor) {
            s = d.minv[i] * ybar[i];
        } else {
            s = warp_sum(factor_row_dot(d, d.minv, i, ybar, lane, 32));
        }
        if (lane == 0) {
            rbar[i] = s;
            bbar[i] -= s;
        }
    }
}

// t_bar_e = x_bar_e + w_e (A^T r_bar)_e ;  s_bar_e = t_bar_e / D_e ;  c_bar_e -= s_bar_e / rho
__global__ void __launch_bounds__(ETHREADS) k_bwd_tbar(Dev d, const double* __restrict__ xbar,
                                                       const double* __restrict__ rbar, double* __restrict__ sbar,
                                                       double* __restrict__ cbar, double rho) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.NE; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = d.at_ptr[e]; q < d.at_ptr[e + 1]; ++q) s += d.at_val[q] * rbar[d.at_col[q]];
        const double sb = (xbar[e] + d.wgt[e] * s) * d.dinv[e];
        sbar[e] = sb;
        cbar[e] -= sb / rho;
    }
}

// x_k_bar_j = s_bar(gmap_j) ;  lambda_bar_j = lamprev_j + s_bar(gmap_j) / rho
__global__ void __launch_bounds__(ETHREADS) k_bwd_state(Dev d, const double* __restrict__ sbar,
                                                        const double* __restrict__ lamprev, double* __restrict__ xkbar,
                                                        double* __restrict__ lambar, double rho) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.nd; j += gridDim.x * blockDim.x) {
        const double sb = sbar[d.gmap[j]];
        xkbar[j] = sb;
        lambar[j] = lamprev[j] + sb / rho;
    }
}

// Reset the per-segment iteration counters (the replay counts from 0).
__global__ void k_reset_ctl(Dev d, double rho) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        d.rho[0] = rho;
        d.ctl[CTL_DONE] = 0;
        d.ctl[CTL_ITER] = 0;
        d.ctl[CTL_STATUS] = 1;
        d.ctl[CTL_COUNTER] = 0;
    }
}

}  // namespace cdsdp_dev
