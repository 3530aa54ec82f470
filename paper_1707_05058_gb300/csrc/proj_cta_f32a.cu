// float thread-block-per-clique projection kernels, padded orders 36, 40, 44, 48.
#define CTA_T float
#define CTA_SUFFIX(name) name##_f32a
#define CTA_SIZES(X) X(36) X(40) X(44) X(48)
#include "proj_cta_impl.cuh"
