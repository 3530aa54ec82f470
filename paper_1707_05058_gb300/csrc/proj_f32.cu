// float32 instantiations of the batched projection kernels.
#define PROJ_T float
#define PROJ_SUFFIX(name) name##_f32
#include "proj_impl.cuh"
