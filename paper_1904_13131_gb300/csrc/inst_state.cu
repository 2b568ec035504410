// Gauss-point state build, residual and diagonal kernels (all dims and degrees).
#include "cell_kernels.cuh"
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
template <int DIM, int N, typename E>
void launch_diag(const CellArgs<double>& a, cudaStream_t st) {
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NPT = ipow(N, DIM);
  const int grid = (a.g.ncells + CB - 1) / CB;
  diag_kernel<DIM, N, E><<<grid, CB * NPT, 0, st>>>(a);
}
}  // namespace

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
}  // namespace hy
