// Tangent-action kernels, double, dim 3, degrees 1-4, all five variants.
#define INST_DIM 3
#define INST_T double
#define INST_NAME apply_fn_f64_3d
#include "inst_apply.inc"
