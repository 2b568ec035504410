// Tangent-action kernels, double, dim 2, degrees 1-4, all five variants.
#define INST_DIM 2
#define INST_T double
#define INST_NAME apply_fn_f64_2d
#include "inst_apply.inc"
