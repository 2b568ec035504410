// Tangent-action kernels, double, dim 2, degrees 3-4: the general builds of FC, SC and NC (the reference
// map per Gauss point from the cache, the volumetric function chosen at run time), one problem or a
// work list.
#define INST_DIM 2
#define INST_T double
#define INST_GEN 1
#define INST_NLO 4
#define INST_NAME apply_fn_f64_2d_gen_hi
#define INST_LIST_NAME apply_list_fn_f64_2d_gen_hi
#include "inst_apply.inc"
