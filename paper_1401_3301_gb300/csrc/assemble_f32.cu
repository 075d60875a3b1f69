// Scalar operators, FP32 form (double-float det B, compensated sums).
#define FE_T float
#define FE_LAUNCH_SCALAR fe_launch_scalar_f32
#include "assemble_scalar.inc"
#define FE_LAUNCH_PAIR fe_launch_pair_f32
#include "assemble_pair.inc"
