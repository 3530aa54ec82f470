// float thread-block-per-clique projection kernels, padded orders 96, 128.
#define CTA_T float
#define CTA_SUFFIX(name) name##_f32c
#define CTA_SIZES(X) X(96) X(128)
#include "proj_cta_impl.cuh"
