// double thread-block-per-clique projection kernels, padded orders 52, 56, 60, 64.
#define CTA_T double
#define CTA_SUFFIX(name) name##_f64b
#define CTA_SIZES(X) X(52) X(56) X(60) X(64)
#include "proj_cta_impl.cuh"
