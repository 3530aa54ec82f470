// double instantiations of the batched projection kernels, padded orders 2..16.
#define PROJ_T double
#define PROJ_PART 0
#define PROJ_SUFFIX(name) name##_f64_small
#include "proj_impl.cuh"
