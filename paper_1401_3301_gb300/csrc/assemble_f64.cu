// Scalar operators, FP64 form.
#define FE_T double
#define FE_LAUNCH_SCALAR fe_launch_scalar_f64
#include "assemble_scalar.inc"
#define FE_LAUNCH_PAIR fe_launch_pair_f64
#include "assemble_pair.inc"
