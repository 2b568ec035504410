// Tangent-action kernels, double-float (FP64 vectors, FP32-pipe arithmetic), dim 3, degrees 3-4, variant
// SC, one problem or a work list (one translation unit per variant and degree pair).
#define INST_DIM 3
#define INST_T ff
#define INST_VAR VAR_SC
#define INST_N0 4
#define INST_NAME apply_fn_ff_3d_v3_hi
#define INST_LIST_NAME apply_list_fn_ff_3d_v3_hi
#include "inst_apply.inc"
