// Tangent-action kernels, double, dim 2, degrees 3-4, all five variants, one problem or a work list.
#define INST_DIM 2
#define INST_T double
#define INST_NLO 4
#define INST_NAME apply_fn_f64_2d_hi
#define INST_LIST_NAME apply_list_fn_f64_2d_hi
#include "inst_apply.inc"
