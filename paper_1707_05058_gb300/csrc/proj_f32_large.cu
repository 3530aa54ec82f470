// float instantiations of the batched projection kernels, padded orders 20..32.
#define PROJ_T float
#define PROJ_PART 1
#define PROJ_SUFFIX(name) name##_f32_large
#include "proj_impl.cuh"
