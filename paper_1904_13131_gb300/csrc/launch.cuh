// Host-side launchers of the device kernels (declarations; definitions live in the .cu files that
// instantiate the templates, so that those translation units compile in parallel).
#pragma once
#include <cuda_runtime.h>
#include "hy_internal.cuh"

namespace hy {

template <typename T> struct CellArgs;

template <typename T>
using CellFn = void (*)(const CellArgs<T>&, cudaStream_t);
// tangent action: form FORM_POINT (thread per Gauss point) or FORM_LINE (thread per x-line)
template <typename T>
using ApplyFn = void (*)(const CellArgs<T>&, int form, cudaStream_t);
template <typename TOUT>
using StateFn = void (*)(const CellArgs<double>&, TOUT*, cudaStream_t);

// tangent action over a work list of problems in one launch: list[count] arguments in device memory,
// start[count + 1] first thread block of each problem, blocks = start[count]
template <typename T>
using ApplyListFn = void (*)(const CellArgs<T>* list, const int* start, int count, int blocks, int form,
                             cudaStream_t);
// cells per thread block of the tangent action (both forms) for element type T: the work-list block counts
template <typename T>
inline int apply_cells_per_block(int dim, int n) { return layout_cells<T>(dim, n); }

// n = degree + 1 in 2..5; var in Variant; returns nullptr for unsupported combinations. The kernels of
// degrees 1-2 (n <= 3) and 3-4 live in separate translation units (_lo, _hi) that compile in parallel, and
// so do the general builds of FC, SC, NC (_gen).
#define HY_APPLY_TABLES(P, TAG, D)                                                                      \
  ApplyFn<P> apply_fn_##TAG##_##D##_lo(int n, int var);                                              \
  ApplyFn<P> apply_fn_##TAG##_##D##_hi(int n, int var);                                              \
  ApplyFn<P> apply_fn_##TAG##_##D##_gen_lo(int n, int var);                                          \
  ApplyFn<P> apply_fn_##TAG##_##D##_gen_hi(int n, int var);                                          \
  ApplyListFn<P> apply_list_fn_##TAG##_##D##_lo(int n, int var);                                     \
  ApplyListFn<P> apply_list_fn_##TAG##_##D##_hi(int n, int var);                                     \
  ApplyListFn<P> apply_list_fn_##TAG##_##D##_gen_lo(int n, int var);                                 \
  ApplyListFn<P> apply_list_fn_##TAG##_##D##_gen_hi(int n, int var);                                 \
  inline ApplyFn<P> apply_fn_##TAG##_##D(int n, int var) {                                           \
    if (is_general(var))                                                                           \
      return n <= 3 ? apply_fn_##TAG##_##D##_gen_lo(n, var) : apply_fn_##TAG##_##D##_gen_hi(n, var);    \
    return n <= 3 ? apply_fn_##TAG##_##D##_lo(n, var) : apply_fn_##TAG##_##D##_hi(n, var);             \
  }                                                                                                \
  inline ApplyListFn<P> apply_list_fn_##TAG##_##D(int n, int var) {                                  \
    if (is_general(var))                                                                           \
      return n <= 3 ? apply_list_fn_##TAG##_##D##_gen_lo(n, var) : apply_list_fn_##TAG##_##D##_gen_hi(n, var); \
    return n <= 3 ? apply_list_fn_##TAG##_##D##_lo(n, var) : apply_list_fn_##TAG##_##D##_hi(n, var);   \
  }
HY_APPLY_TABLES(double, f64, 2d)
HY_APPLY_TABLES(double, f64, 3d)
HY_APPLY_TABLES(float, f32, 2d)
HY_APPLY_TABLES(float, f32, 3d)
// double-float: one translation unit per (dim, variant) for degrees 1-2 (_lo) and per (dim, variant) for
// degrees 3-4 (_hi)
#define HY_FF_VAR(D, V)                                                                            \
  ApplyFn<ff> apply_fn_ff_##D##_v##V##_lo(int n);                                                  \
  ApplyFn<ff> apply_fn_ff_##D##_v##V##_hi(int n);                                                  \
  ApplyListFn<ff> apply_list_fn_ff_##D##_v##V##_lo(int n);                                         \
  ApplyListFn<ff> apply_list_fn_ff_##D##_v##V##_hi(int n);                                         \
  inline ApplyFn<ff> apply_fn_ff_##D##_v##V(int n) {                                               \
    return n <= 3 ? apply_fn_ff_##D##_v##V##_lo(n) : apply_fn_ff_##D##_v##V##_hi(n);                \
  }                                                                                                \
  inline ApplyListFn<ff> apply_list_fn_ff_##D##_v##V(int n) {                                      \
    return n <= 3 ? apply_list_fn_ff_##D##_v##V##_lo(n) : apply_list_fn_ff_##D##_v##V##_hi(n);      \
  }
#define HY_FF_TABLES(D)                                                                            \
  HY_FF_VAR(D, 0)                                                                                  \
  HY_FF_VAR(D, 1)                                                                                  \
  HY_FF_VAR(D, 2)                                                                                  \
  HY_FF_VAR(D, 3)                                                                                  \
  HY_FF_VAR(D, 4)                                                                                  \
  inline ApplyFn<ff> apply_fn_ff_##D(int n, int var) {                                             \
    switch (var) {                                                                                 \
      case 0: return apply_fn_ff_##D##_v0(n);                                                      \
      case 1: return apply_fn_ff_##D##_v1(n);                                                      \
      case 2: return apply_fn_ff_##D##_v2(n);                                                      \
      case 3: return apply_fn_ff_##D##_v3(n);                                                      \
      case 4: return apply_fn_ff_##D##_v4(n);                                                      \
    }                                                                                              \
    return nullptr;                                                                                \
  }                                                                                                \
  inline ApplyListFn<ff> apply_list_fn_ff_##D(int n, int var) {                                    \
    switch (var) {                                                                                 \
      case 0: return apply_list_fn_ff_##D##_v0(n);                                                 \
      case 1: return apply_list_fn_ff_##D##_v1(n);                                                 \
      case 2: return apply_list_fn_ff_##D##_v2(n);                                                 \
      case 3: return apply_list_fn_ff_##D##_v3(n);                                                 \
      case 4: return apply_list_fn_ff_##D##_v4(n);                                                 \
    }                                                                                              \
    return nullptr;                                                                                \
  }
HY_FF_TABLES(2d)
HY_FF_TABLES(3d)
#undef HY_FF_TABLES
#undef HY_FF_VAR
#undef HY_APPLY_TABLES
StateFn<double> state_fn_f64(int dim, int n, int var);   // var VAR_NONE: J check only
StateFn<float> state_fn_f32(int dim, int n, int var);
StateFn<ff> state_fn_ff(int dim, int n, int var);
// FP32 cache (nvd values per Gauss point) of a level derived from its FP64 (src_ff false) or double-float
// cache (nvs values) of the same state: the same variant, or T2 from T4 (t4_to_t2).
void launch_derive_f32(int dim, int n, bool src_ff, const void* src, int nvs, float* dst, int nvd, bool t4_to_t2,
                       int ncells, cudaStream_t st);
CellFn<double> residual_fn(int dim, int n);
// diagonal: the sum over (node, Gauss point) pairs in FP64, or in double-float (ff_arith)
CellFn<double> diag_fn(int dim, int n, bool ff_arith);
// The diagonal with the Gauss-point state read from the level's T4 or T2 cache (a.cache) in the diagonal's
// element type (double-float when ff_arith) instead of evaluated from the displacement.
CellFn<double> diag_cached_fn(int dim, int n, bool ff_arith, int var);

constexpr int VAR_NONE = 5;

// ---- vector kernels (vec_kernels.cu) ----------------------------------------------------------
template <typename T> void launch_prep_out(const T* x, T* y, long long n_nodes, int dim, const Geom& g, cudaStream_t st);
// prep_out of each problem of a work list (list in device memory, count problems, the largest with
// max_nodes lattice nodes), one launch
template <typename T> void launch_prep_out_list(const CellArgs<T>* list, int count, int dim, long long max_nodes,
                                                cudaStream_t st);
template <typename T> void launch_zero_constrained(T* y, long long n_nodes, int dim, const Geom& g, cudaStream_t st);
template <typename T> void launch_set_constrained_one(T* y, long long n_nodes, int dim, const Geom& g, cudaStream_t st);
template <typename T> void launch_invert(const double* d, T* dinv, long long n, cudaStream_t st);
template <typename TA, typename TB> void launch_convert(const TA* a, TB* b, long long n, cudaStream_t st);
// y = a*x + b*y
template <typename T> void launch_axpby(T a, const T* x, T b, T* y, long long n, cudaStream_t st);
// z = x + a*y
template <typename T> void launch_xpay(const T* x, T a, const T* y, T* z, long long n, cudaStream_t st);
// Chebyshev: first step. r = b (x0 zero) or r = b - t; d = dinv*r*inv_theta; x = d (x0 zero) or x += d.
// prep (the level geometry, or null): also t = (constrained ? d : 0), the next application's output
// prepared as launch_prep_out would -- or, with prep_x, prepared for an application of the new x.
template <typename T> void launch_cheb_init(const T* b, T* t, const T* dinv, T* r, T* d, T* x, T inv_theta,
                                            bool x0_zero, long long n, const Geom* prep, int dim, cudaStream_t st,
                                            bool prep_x = false);
// Chebyshev: later step. r -= t; d = cd*d + cr*dinv*r; x += d; prep as above
template <typename T> void launch_cheb_step(T* t, const T* dinv, T* r, T* d, T* x, T cd, T cr, long long n,
                                            const Geom* prep, int dim, cudaStream_t st, bool prep_x = false);
// z = a * b (elementwise)
template <typename T> void launch_mul(const T* a, const T* b, T* z, long long n, cudaStream_t st);
// out[i] = SplitMix64 uniform on [-1, 1) at counter i (seeded)
template <typename T> void launch_splitmix(T* out, long long n, unsigned long long seed, cudaStream_t st);
// y += sign * (*alpha_dev) x ; z = x + (*beta_dev) y
template <typename T> void launch_axpy_dev(const double* alpha, double sign, const T* x, T* y, long long n, cudaStream_t st);
template <typename T> void launch_xpay_dev(const T* x, const double* beta, const T* y, T* z, long long n, cudaStream_t st);
// device-side scalars of one CG step of the eigenvalue estimate (s: 8 doubles; hist: 2 * iters)
void launch_eig_alpha(double* s, double* hist, int it, cudaStream_t st);
void launch_eig_beta(double* s, double* hist, int it, int iters, cudaStream_t st);
// device-side scalars of one preconditioned CG step (s: 9 doubles {rz, pq, alpha, rr, rzn, beta, tol,
// converged, not_spd}); op 0 alpha, 1 convergence test, 2 beta
constexpr int PCG_SCALARS = 16;  // stride of one problem's scalars
void launch_pcg_scalar(double* s, int op, cudaStream_t st);
// one thread block whose bounded mbarrier wait can never complete: sets ERRBIT_TIMEOUT in *err after limit_ns
void launch_bounded_wait_check(unsigned* err, unsigned long long limit_ns, cudaStream_t st);
// r = b - t
template <typename T> void launch_sub(const T* b, const T* t, T* r, long long n, cudaStream_t st);
// f += t * int_face N_a dA on face `face` (0..2 dim-1: -x, +x, -y, +y, -z, +z); FaceLoad carries the traction t
// and w1[i], the integral of 1D GLL-basis function i over the unit interval (i = 0..k)
struct FaceLoad {
  double t[3];
  double w1[MAXN];
  int k;
};
void launch_face_load(double* f, int dim, const Geom& g, int face, const FaceLoad& fl, cudaStream_t st);
// du0 = constrained ? target - u : 0, target from per-face values scaled by factor
void launch_lift(const double* u, double* du0, double factor, const double* face_vals /*device [6][3]*/,
                 long long n_nodes, int dim, const Geom& g, cudaStream_t st);
// deterministic dot: partial sums in fixed blocks, then one block; result in out[0]
constexpr int DOT_BLOCKS = 304;
template <typename T> void launch_dot(const T* a, const T* b, long long n, double* partials, double* out,
                                      cudaStream_t st);
// separable 1D transfer sweep along `axis`: out(i with i_axis = o) = sum_e w[o*E+e] in(i with i_axis = start[o]+e).
// in_minus (or null): the input is in - in_minus. prep (or null): also prep = (masked out ? new out : 0), the
// output of an application of `out` prepared as launch_prep_out would.
template <typename T>
void launch_sweep(const T* in, T* out, int dim, const int Lin[3], const int Lout[3], int axis, const int* start,
                  const T* w, int E, bool add_to_out, const Geom* mask_in, const Geom* mask_out, cudaStream_t st,
                  const T* in_minus = nullptr, T* prep = nullptr);

// ---- exact coarsest-level solve (coarse_direct.cu) ----------------------------------------------
// dense tangent of a level on its free dofs (cidx: dof -> compact index or -1), accumulated into A
// (nfree x nfree, zeroed by the caller)
void launch_assemble_dense(int dim, int n, const CellArgs<double>& a, double* A, long long nfree, const int* cidx,
                           cudaStream_t st);
// blocked Gauss-Jordan inverse, ping-ponging between A and B; returns the buffer holding the inverse;
// flags a pivot <= 0 in err; work holds 32*32 + 64 n doubles
double* launch_gj_invert(double* A, double* B, long long n, double* work, unsigned* err, bool ff_arith,
                         cudaStream_t st);
// x[free_idx[i]] = sum_j A_ij b[free_idx[j]]
void launch_dense_gemv(const double* A, const double* b, double* x, long long n, const int* free_idx, cudaStream_t st);

}  // namespace hy
