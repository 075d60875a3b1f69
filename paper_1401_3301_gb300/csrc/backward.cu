// Stiffness backward (placeholder until the kernels land).
#include "fe_internal.cuh"
int fe_launch_backward(fe_pattern_s*, const double*, const void*, int, const void*, const void*,
                       void*, void*, void*, int, cudaStream_t) {
  return FE_ERR_ARG;
}
