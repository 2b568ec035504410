// Gauss-point state build, residual and diagonal kernels (all dims and degrees).
#include "setup_kernels.cuh"
#include "launch.cuh"

namespace hy {
namespace {
template <int DIM, int N, int VAR, typename T>
void launch_state(const CellArgs<double>& a, T* out, cudaStream_t st) {
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NPT = ipow(N, DIM);
  const int grid = (a.g.ncells + CB - 1) / CB;
  qp_state_kernel<DIM, N, VAR, T><<<grid, CB * NPT, 0, st>>>(a, out);
}
template <int DIM, int N>
void launch_residual(const CellArgs<double>& a, cudaStream_t st) {
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NPT = ipow(N, DIM);
  const int grid = (a.g.ncells + CB - 1) / CB;
  residual_kernel<DIM, N><<<grid, CB * NPT, 0, st>>>(a);
}
template <int DIM, int N, typename E, int SRC = 0>
void launch_diag(const CellArgs<double>& a, cudaStream_t st) {
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NPT = ipow(N, DIM);
  const int grid = (a.g.ncells + CB - 1) / CB;
  diag_kernel<DIM, N, E, SRC><<<grid, CB * NPT, 0, st>>>(a);
}

__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float to_f32(ff v) { return v.hi; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(ff v) { return (double)v.hi + (double)v.lo; }

// One thread per (cell, Gauss point): the FP32 cache entries of the point from the FP64 or double-float
// cache of the same state, each in its own cell-block layout. The same variant rounds every value to FP32 (the
// leading float of a double-float value is the FP64 value rounded to FP32), so the result equals what the
// FP32 state kernel writes. T2 from T4 keeps M and tau~ and recovers c1~ = JC~_0000 - JC~_0011 and
// c2~ = JC~_0011 (JC~ = c1~ S + c2~ I (x) I, Voigt entries (0, 0) and (0, 1)) in FP64 before rounding.
template <int DIM, int N, typename TS>
__global__ void derive_f32_kernel(const TS* __restrict__ src, int nvs, float* __restrict__ dst, int nvd, bool t4_to_t2,
                                  int ncells) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int CBS = layout_cells<TS>(DIM, N), BSS = layout_row<TS>(DIM, N);
  constexpr int CBD = layout_cells<float>(DIM, N), BSD = layout_row<float>(DIM, N);
  constexpr int NM = DIM * DIM + nsym(DIM);  // M and tau~
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)ncells * NPT) return;
  const int cell = (int)(i / NPT), p = (int)(i % NPT);
  const TS* s = src + (long long)(cell / CBS) * nvs * BSS + (cell % CBS) * NPT + p;
  float* d = dst + (long long)(cell / CBD) * nvd * BSD + (cell % CBD) * NPT + p;
  if (!t4_to_t2) {
    for (int v = 0; v < nvd; ++v) d[(long long)v * BSD] = to_f32(s[(long long)v * BSS]);
    return;
  }
#pragma unroll
  for (int v = 0; v < NM; ++v) d[(long long)v * BSD] = to_f32(s[(long long)v * BSS]);
  const double k00 = to_f64(s[(long long)NM * BSS]), k01 = to_f64(s[(long long)(NM + 1) * BSS]);
  d[(long long)NM * BSD] = (float)(k00 - k01);
  d[(long long)(NM + 1) * BSD] = (float)k01;
}

template <int DIM, int N>
void launch_derive(bool src_ff, const void* src, int nvs, float* dst, int nvd, bool t4_to_t2, int ncells,
                   cudaStream_t st) {
  const long long total = (long long)ncells * ipow(N, DIM);
  const int grid = (int)((total + 255) / 256);
  if (src_ff) derive_f32_kernel<DIM, N, ff><<<grid, 256, 0, st>>>(static_cast<const ff*>(src), nvs, dst, nvd, t4_to_t2, ncells);
  else derive_f32_kernel<DIM, N, double><<<grid, 256, 0, st>>>(static_cast<const double*>(src), nvs, dst, nvd, t4_to_t2, ncells);
}
}  // namespace

void launch_derive_f32(int dim, int n, bool src_ff, const void* src, int nvs, float* dst, int nvd, bool t4_to_t2,
                       int ncells, cudaStream_t st) {
  using Fn = void (*)(bool, const void*, int, float*, int, bool, int, cudaStream_t);
  static const Fn t[2][4] = {{launch_derive<2, 2>, launch_derive<2, 3>, launch_derive<2, 4>, launch_derive<2, 5>},
                             {launch_derive<3, 2>, launch_derive<3, 3>, launch_derive<3, 4>, launch_derive<3, 5>}};
  if (n < 2 || n > 5 || dim < 2 || dim > 3 || ncells <= 0) return;
  t[dim - 2][n - 2](src_ff, src, nvs, dst, nvd, t4_to_t2, ncells, st);
}

// indexed by Variant (0-4, VAR_NONE = 5, the general builds 6-8; double-float has no general build)
#define HY_SROW(D, N, T)                                                                                   \
  { launch_state<D, N, VAR_T4, T>, launch_state<D, N, VAR_T2, T>, launch_state<D, N, VAR_FC, T>,           \
    launch_state<D, N, VAR_SC, T>, launch_state<D, N, VAR_NC, T>, launch_state<D, N, VAR_NONE, T>,         \
    launch_state<D, N, VAR_FCG, T>, launch_state<D, N, VAR_SCG, T>, launch_state<D, N, VAR_NCG, T> }
#define HY_SROW_FF(D, N)                                                                                   \
  { launch_state<D, N, VAR_T4, ff>, launch_state<D, N, VAR_T2, ff>, launch_state<D, N, VAR_FC, ff>,         \
    launch_state<D, N, VAR_SC, ff>, launch_state<D, N, VAR_NC, ff>, launch_state<D, N, VAR_NONE, ff>,       \
    nullptr, nullptr, nullptr }

StateFn<double> state_fn_f64(int dim, int n, int var) {
  static const StateFn<double> t2[4][9] = {HY_SROW(2, 2, double), HY_SROW(2, 3, double), HY_SROW(2, 4, double),
                                           HY_SROW(2, 5, double)};
  static const StateFn<double> t3[4][9] = {HY_SROW(3, 2, double), HY_SROW(3, 3, double), HY_SROW(3, 4, double),
                                           HY_SROW(3, 5, double)};
  if (n < 2 || n > 5 || var < 0 || var > 8) return nullptr;
  return dim == 2 ? t2[n - 2][var] : dim == 3 ? t3[n - 2][var] : nullptr;
}
StateFn<float> state_fn_f32(int dim, int n, int var) {
  static const StateFn<float> t2[4][9] = {HY_SROW(2, 2, float), HY_SROW(2, 3, float), HY_SROW(2, 4, float),
                                          HY_SROW(2, 5, float)};
  static const StateFn<float> t3[4][9] = {HY_SROW(3, 2, float), HY_SROW(3, 3, float), HY_SROW(3, 4, float),
                                          HY_SROW(3, 5, float)};
  if (n < 2 || n > 5 || var < 0 || var > 8) return nullptr;
  return dim == 2 ? t2[n - 2][var] : dim == 3 ? t3[n - 2][var] : nullptr;
}
StateFn<ff> state_fn_ff(int dim, int n, int var) {
  static const StateFn<ff> t2[4][9] = {HY_SROW_FF(2, 2), HY_SROW_FF(2, 3), HY_SROW_FF(2, 4), HY_SROW_FF(2, 5)};
  static const StateFn<ff> t3[4][9] = {HY_SROW_FF(3, 2), HY_SROW_FF(3, 3), HY_SROW_FF(3, 4), HY_SROW_FF(3, 5)};
  if (n < 2 || n > 5 || var < 0 || var > 8) return nullptr;
  return dim == 2 ? t2[n - 2][var] : dim == 3 ? t3[n - 2][var] : nullptr;
}
#undef HY_SROW
#undef HY_SROW_FF

CellFn<double> residual_fn(int dim, int n) {
  static const CellFn<double> t[2][4] = {{launch_residual<2, 2>, launch_residual<2, 3>, launch_residual<2, 4>,
                                          launch_residual<2, 5>},
                                         {launch_residual<3, 2>, launch_residual<3, 3>, launch_residual<3, 4>,
                                          launch_residual<3, 5>}};
  if (n < 2 || n > 5 || dim < 2 || dim > 3) return nullptr;
  return t[dim - 2][n - 2];
}
CellFn<double> diag_fn(int dim, int n, bool ff_arith) {
  static const CellFn<double> t[2][2][4] = {
      {{launch_diag<2, 2, double>, launch_diag<2, 3, double>, launch_diag<2, 4, double>, launch_diag<2, 5, double>},
       {launch_diag<3, 2, double>, launch_diag<3, 3, double>, launch_diag<3, 4, double>, launch_diag<3, 5, double>}},
      {{launch_diag<2, 2, ff>, launch_diag<2, 3, ff>, launch_diag<2, 4, ff>, launch_diag<2, 5, ff>},
       {launch_diag<3, 2, ff>, launch_diag<3, 3, ff>, launch_diag<3, 4, ff>, launch_diag<3, 5, ff>}}};
  if (n < 2 || n > 5 || dim < 2 || dim > 3) return nullptr;
  return t[ff_arith ? 1 : 0][dim - 2][n - 2];
}
#define HY_DROW(E, S)                                                                                              \
  {{launch_diag<2, 2, E, S>, launch_diag<2, 3, E, S>, launch_diag<2, 4, E, S>, launch_diag<2, 5, E, S>},          \
   {launch_diag<3, 2, E, S>, launch_diag<3, 3, E, S>, launch_diag<3, 4, E, S>, launch_diag<3, 5, E, S>}}
CellFn<double> diag_cached_fn(int dim, int n, bool ff_arith, int var) {
  static const CellFn<double> t[2][2][2][4] = {{HY_DROW(double, 1), HY_DROW(double, 2)},
                                               {HY_DROW(ff, 1), HY_DROW(ff, 2)}};
  if (n < 2 || n > 5 || dim < 2 || dim > 3 || (var != VAR_T4 && var != VAR_T2)) return nullptr;
  return t[ff_arith ? 1 : 0][var == VAR_T4 ? 0 : 1][dim - 2][n - 2];
}
#undef HY_DROW
}  // namespace hy
