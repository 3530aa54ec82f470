// Reverse pass through unrolled Algorithm 1: shared declarations.
#pragma once

#include <cuda_runtime.h>

#include "proj_launch.h"

namespace cdsdp_dev {

// Buffers and scalars of one reverse iteration (all adjoints in float64).
struct GradArgs {
    const double* xkbar;  // [nd] adjoint of the clique vectors after the iteration
    const double* lambar; // [nd] adjoint of the multipliers after the iteration
    double* hxbar;        // [nd] out: adjoint of H x
    double* lamprev;      // [nd] out: multiplier adjoint before the affine-step terms
    double rho, tolrel;
    int max_sweeps;
    int slot;             // recorded iteration within the replayed segment
};

// Daleckii-Krein kernel over the cliques of one size class (orders <= 32).
cudaError_t launch_bwd_proj(bool fp32, int cls, const Dev& d, const int* list, int nlist, const GradArgs& ga,
                            cudaStream_t st);

}  // namespace cdsdp_dev
