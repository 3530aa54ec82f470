// float64 instantiations of the batched projection kernels.
#define PROJ_T double
#define PROJ_SUFFIX(name) name##_f64
#include "proj_impl.cuh"
