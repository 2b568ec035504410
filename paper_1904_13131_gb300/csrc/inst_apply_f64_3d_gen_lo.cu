// Tangent-action kernels, double, dim 3, degrees 1-2: the general builds of FC, SC and NC (the reference
// map per Gauss point from the cache, the volumetric function chosen at run time), one problem or a
// work list.
#define INST_DIM 3
#define INST_T double
#define INST_GEN 1
#define INST_NLO 2
#define INST_NAME apply_fn_f64_3d_gen_lo
#define INST_LIST_NAME apply_list_fn_f64_3d_gen_lo
#include "inst_apply.inc"
