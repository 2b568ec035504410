// Tangent-action kernels, double-float (FP64 vectors, FP32-pipe arithmetic), dim 2, degrees 3-4, variant
// T4, one problem or a work list (one translation unit per variant and degree pair).
#define INST_DIM 2
#define INST_T ff
#define INST_VAR VAR_T4
#define INST_N0 4
#define INST_NAME apply_fn_ff_2d_v0_hi
#define INST_LIST_NAME apply_list_fn_ff_2d_v0_hi
#include "inst_apply.inc"
