// float instantiations of the batched projection kernels, padded orders 2..16.
#define PROJ_T float
#define PROJ_PART 0
#define PROJ_SUFFIX(name) name##_f32_small
#include "proj_impl.cuh"
