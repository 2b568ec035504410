// Tangent-action kernels, float, dim 2, degrees 1-4, all five variants.
#define INST_DIM 2
#define INST_T float
#define INST_NAME apply_fn_f32_2d
#include "inst_apply.inc"
