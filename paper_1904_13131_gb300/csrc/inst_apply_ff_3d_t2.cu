// Tangent-action kernels, double-float (FP64 vectors, FP32-pipe arithmetic), dim 3, degrees 1-2, variant
// T2, one problem or a work list (one translation unit per variant: double-float kernels are long).
#define INST_DIM 3
#define INST_T ff
#define INST_VAR VAR_T2
#define INST_NAME apply_fn_ff_3d_v1_lo
#define INST_LIST_NAME apply_list_fn_ff_3d_v1_lo
#include "inst_apply.inc"
