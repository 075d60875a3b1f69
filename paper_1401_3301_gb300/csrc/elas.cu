// Linear elasticity (placeholder until the vector kernels land).
#include "fe_internal.cuh"
int fe_launch_elas(fe_pattern_s*, const double*, const void*, int, const void*, int, int, void*,
                   cudaStream_t) {
  return FE_ERR_ARG;
}
