// Tangent-action kernels, float, dim 3, degrees 1-4, all five variants.
#define INST_DIM 3
#define INST_T float
#define INST_NAME apply_fn_f32_3d
#include "inst_apply.inc"
