// Internal interface between the solve server (server.cu) and the library core (capi.cu). Not part of
// the C ABI: nothing here is declared in include/hyperelastic.h.
#pragma once
#include "../../include/hyperelastic.h"

// A replacement for the outer preconditioned CG of hy_newton_solve: solve the finest-level Newton system
// A(u) x = rhs of ctx (its current linearisation) to ||r|| <= rtol ||rhs|| from x = 0, set *iterations and
// return the status pcg would return (the same messages in hy_last_error(ctx)). It is called from the
// thread running hy_newton_solve; ctx must not be used by anyone else until it returns.
typedef hy_status (*hy_linear_solve_hook)(void* user, hy_ctx* ctx, const double* rhs, double* x, double rtol,
                                          int max_iter, int* iterations);
// NULL hook: the context's own PCG.
void hy_ctx_set_solve_hook(hy_ctx* ctx, hy_linear_solve_hook hook, void* user);

// Grouping key of contexts whose outer CG can share one work-list batch: equal for equal dimension,
// degree, cache variants of the finest level and finest-level action precision.
long long hy_ctx_batch_key(const hy_ctx* ctx);

// A work-list batch with room for `capacity` problems and no members yet; hy_batch_bind sets the members
// (1..capacity contexts of one device, dimension and degree) before each hy_batch_pcg / hy_batch_apply.
hy_status hy_batch_create_empty(hy_batch** out, int device, int capacity);
hy_status hy_batch_bind(hy_batch* b, hy_ctx* const* ctxs, int count);

// hy_footprint with `general` set: the bytes when FC, SC and NC run their general builds (curved cells or
// a volumetric function other than the paper's), whose caches add dim^2 + 1 values per Gauss point.
hy_status hy_footprint_general(int dim, int degree, int m, int n_levels, hy_variant variant, hy_dtype level_dtype,
                               const hy_solver_params* sp, const uint32_t* face_masks, bool general,
                               int64_t* bytes);
