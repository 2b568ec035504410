// C ABI of libhyperelastic (include/hyperelastic.h): context, mesh hierarchy, Gauss-point state,
// tangent action, residual, geometric multigrid (Secs. 6-7), PCG and Newton (Secs. 3, 7).
// Host code orchestrates; every step on vectors runs in the kernels of this library.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hyperelastic.h"
#include "cell_kernels.cuh"
#include "launch.cuh"
#include "serve_internal.h"

using namespace hy;

constexpr int SETUP_PHASES = 5;  // carry down, state + diagonal, autotune, smoother estimates, coarse setup

namespace {

// Named NVTX range over a solver phase (linearisation, PCG, V-cycle, Newton load step) for profilers and
// tracers; without a tool attached, push and pop return at once.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// ---------------------------------------------------------------------------------------------
// 1D Q_k element tables from their definitions: Legendre recurrences for the GLL points (roots of
// P_k' plus the end points) and the Gauss points (roots of P_n), Newton iteration to full precision,
// Lagrange polynomials by their product formula.
void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0);
}

std::vector<double> gauss_points(int n, std::vector<double>& w) {
  std::vector<double> x(n);
  w.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double t = -std::cos(M_PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, t, p, dp);
      const double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double p, dp;
    legendre(n, t, p, dp);
    x[j] = 0.5 * (t + 1.0);
    w[j] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) on [-1,1], halved for [0,1]
  }
  std::sort(x.begin(), x.end());
  // weights are symmetric; recompute in sorted order
  for (int j = 0; j < n; ++j) {
    double p, dp;
    const double t = 2.0 * x[j] - 1.0;
    legendre(n, t, p, dp);
    w[j] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
  return x;
}

std::vector<double> gll_points(int k) {
  std::vector<double> x(k + 1);
  x[0] = 0.0;
  x[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double t = -std::cos(M_PI * j / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, t, p, dp);
      const double d2p = (2.0 * t * dp - k * (k + 1.0) * p) / (1.0 - t * t);  // Legendre ODE
      const double dt = dp / d2p;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[j] = 0.5 * (t + 1.0);
  }
  std::sort(x.begin(), x.end());
  return x;
}

double lagr(const std::vector<double>& nd, int j, double x) {
  double v = 1.0;
  for (size_t m = 0; m < nd.size(); ++m)
    if ((int)m != j) v *= (x - nd[m]) / (nd[j] - nd[m]);
  return v;
}
double dlagr(const std::vector<double>& nd, int j, double x) {
  double s = 0.0;
  for (size_t m = 0; m < nd.size(); ++m) {
    if ((int)m == j) continue;
    double t = 1.0 / (nd[j] - nd[m]);
    for (size_t l = 0; l < nd.size(); ++l)
      if ((int)l != j && l != m) t *= (x - nd[l]) / (nd[j] - nd[l]);
    s += t;
  }
  return s;
}

// Extreme eigenvalues of the symmetric tridiagonal (diag a, off-diagonal b) by Sturm-count bisection.
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double d = a[0] - x;
  if (d < 0) ++cnt;
  for (size_t i = 1; i < a.size(); ++i) {
    if (d == 0.0) d = 1e-300;
    d = a[i] - x - b[i - 1] * b[i - 1] / d;
    if (d < 0) ++cnt;
  }
  return cnt;
}
void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double& lmin, double& lmax) {
  const int n = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  double l = lo, h = hi;
  for (int it = 0; it < 200 && h - l > 1e-16 * std::max(std::fabs(h), std::fabs(l)); ++it) {
    const double mid = 0.5 * (l + h);
    if (sturm_count(a, b, mid) >= n) h = mid; else l = mid;
  }
  lmax = h;
  l = lo;
  h = hi;
  for (int it = 0; it < 200 && h - l > 1e-16 * std::max(std::fabs(h), std::fabs(l)); ++it) {
    const double mid = 0.5 * (l + h);
    if (sturm_count(a, b, mid) >= 1) h = mid; else l = mid;
  }
  lmin = h;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
struct Level {
  Geom g{};
  long long nnodes = 0, ndofs = 0, nqp = 0;
  uint8_t* d_mat = nullptr;
  Mat<double> mt64{};
  Mat<float> mt32{};
  Mat<ff> mtff{};
  bool mat_set = false;
  double* d_u64 = nullptr;
  float* d_u32 = nullptr;
  double* d_X64 = nullptr;  // nodal coordinates of a curved geometry (hy_set_geometry)
  double* d_c64 = nullptr;
  float* d_c32 = nullptr;
  size_t c64_len = 0, c32_len = 0;
  bool has64 = false, has32 = false;
  // the finest level's FP64 cache is allocated but built at its first use: with a double-float finest
  // action (fine_dtype) the solver itself never reads it
  bool lazy64 = false;
  double* d_diag = nullptr;
  double* d_dinv64 = nullptr;
  float* d_dinv32 = nullptr;
  double lmax = 0.0;
  ff* d_cff = nullptr;     // double-float cache of the finest level (solver parameter fine_dtype = HY_FF)
  size_t cff_len = 0;
  bool hasff = false;
  int form[3] = {-1, -1, -1};  // tangent-action kernel form per precision (FP64, FP32, double-float)
  int var[3] = {-1, -1, -1};   // tangent variant of the cache of each precision
  double* w64[5] = {};  // V-cycle vectors b, x, r, d, t
  float* w32[5] = {};
  double* d_Ainv = nullptr;  // exact coarse solve: dense free-dof tangent / its inverse (ping-pong pair)
  double* d_Awork = nullptr;
  double* d_inv_piv = nullptr;
  int* d_free_idx = nullptr;  // compact index -> dof
  int* d_cidx = nullptr;      // dof -> compact index or -1
  long long nfree = 0;
  double* d_Aresult = nullptr;  // whichever of the pair holds the inverse
  // the eigenvalue estimate's iterations as an executable graph, replayed while every argument its kernels
  // were captured with (the signature) is unchanged
  cudaGraphExec_t eig_exec = nullptr;
  std::vector<unsigned char> eig_sig;
  long long eig_nodes = 0;
  double* d_eigbuf = nullptr;  // this level's smoother estimate: scalars, coefficient history, dot partials
};

struct Transfer {  // level l-1 (coarse) <-> l (fine); the same 1D tables act along every axis
  int Lc = 0, Lf = 0, Ep = 0, Er = 0, Ei = 0;
  int *d_pstart = nullptr, *d_rstart = nullptr, *d_istart = nullptr;
  double *d_pw64 = nullptr, *d_rw64 = nullptr, *d_iw64 = nullptr;
  float *d_pw32 = nullptr, *d_rw32 = nullptr;
};

struct hy_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int dim = 0, k = 0, n = 0, nlev = 0;
  uint32_t fm[6] = {0, 0, 0, 0, 0, 0};
  std::vector<Level> lev;
  std::vector<Transfer> tr;
  Basis1D<double> b64{};
  Basis1D<float> b32{};
  Basis1D<ff> bff{};
  hy_solver_params sp{4, 1, 0.6, 1.2, 30, 0, 1e-3, 0, -1, HY_F64, -1, 0.0};
  int var = -1;
  int law = 0;  // volumetric function of the neo-Hooke law (hy_set_material_law)
  bool curved = false;  // a curved reference geometry is set (hy_set_geometry)
  bool mixed = false;
  bool state_ok = false;
  double coarse_lo = 0, coarse_hi = 0;
  int coarse_deg = 0;
  bool coarse_spd = false;
  unsigned* d_err = nullptr;
  unsigned long long* d_jmin = nullptr;
  double* d_partials = nullptr;
  double* d_scal = nullptr;
  double* d_face = nullptr;
  double* d_eig_scal = nullptr;  // eigenvalue-estimate scalars (8 doubles), then PCG_SCALARS of the graph PCG
  double* d_eig_hist = nullptr;  // alpha and beta history
  size_t eig_hist_len = 0;
  long long coarse_nfree = 0;    // free dofs of the coarsest level
  double *tmp64a = nullptr, *tmp64b = nullptr;
  float *tmp32a = nullptr, *tmp32b = nullptr, *tmp32c = nullptr;
  size_t tmp_len = 0;
  double* f64[12] = {};  // fine-level FP64 work vectors of PCG / Newton (10: graph-PCG iterate, 11: dead load)
  long long launches = 0;
  bool verbose = false;  // HY_VERBOSE=1: per-iteration diagnostics on stderr
  int prefetch = 0;      // L2 prefetch distance of the tangent action's cache chunks, in cell blocks
  size_t bytes = 0;      // device bytes currently owned
  // The V-cycle below the finest level's input/output copies is captured once per linearisation into a
  // CUDA graph and replayed (HY_GRAPHS=0 disables this and launches kernel by kernel).
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t vc_exec = nullptr;
  bool vc_valid = false;
  // one PCG iteration as a graph (captured once per linearisation), its scalars read back into pinned memory
  cudaGraphExec_t pcg_exec[2] = {nullptr, nullptr};
  long long pcg_nodes[2] = {0, 0};
  double* h_pcg_scal = nullptr;
  long long vc_nodes = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  // the exact coarse inverse is built on a side stream, overlapping the rest of the linearisation
  cudaStream_t side = nullptr;
  cudaEvent_t ev_side_fork = nullptr, ev_side_join = nullptr, ev_side_start = nullptr;
  // streams (and their end events) on which the levels' smoother estimates run side by side
  std::vector<cudaStream_t> eig_st;
  std::vector<cudaEvent_t> eig_ev;
  cudaEvent_t ev_eig_fork = nullptr;
  bool side_timed = false;
  // phase events of the last linearisation (PhaseTimer)
  cudaEvent_t ev_phase[6] = {};
  int phases_recorded = 0;
  unsigned* h_err_side = nullptr;  // pinned: the side stream's error word, read after the join
  bool side_pending = false;
  // reuse of the V-cycle setup (solver parameter setup_reuse): the coarsest level's displacement at the
  // last full setup, and whether that setup is still valid for this mesh, material and parameters
  double* d_usetup = nullptr;
  double* d_udiff = nullptr;
  bool setup_valid = false;
  bool last_setup_reused = false;
  // replacement of the outer PCG inside hy_newton_solve (the solve server's batched solves), or null
  hy_linear_solve_hook solve_hook = nullptr;
  void* solve_user = nullptr;
};

namespace {

#define HY_CK(call)                                                                                     \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                                     \
      return e_ == cudaErrorMemoryAllocation ? HY_ERR_OOM : HY_ERR_CUDA;                                \
    }                                                                                                   \
  } while (0)
#define HY_TRY(expr)                                                                                    \
  do {                                                                                                  \
    hy_status s_ = (expr);                                                                              \
    if (s_ != HY_OK) return s_;                                                                         \
  } while (0)

hy_status fail(hy_ctx* ctx, hy_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

// Device buffers are stream-ordered allocations on the context's stream, so that contexts working
// side by side (the solve server) never synchronise the whole device to allocate or free.
template <typename T>
hy_status dalloc(hy_ctx* ctx, T** p, size_t n) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  cudaError_t e = cudaMallocAsync(&q, bytes, ctx->stream);
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HY_ERR_OOM : HY_ERR_CUDA;
  }
  ctx->allocs.push_back({q, bytes});
  ctx->bytes += bytes;
  *p = (T*)q;
  return HY_OK;
}

void dfree(hy_ctx* ctx, void* p) {
  if (!p) return;
  for (auto it = ctx->allocs.begin(); it != ctx->allocs.end(); ++it)
    if (it->first == p) {
      ctx->bytes -= it->second;
      ctx->allocs.erase(it);
      break;
    }
  cudaFreeAsync(p, ctx->stream);
}

hy_status check_launch(hy_ctx* ctx, int nlaunch) {
  ctx->launches += nlaunch;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, HY_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return HY_OK;
}

void drop_graph(hy_ctx* ctx) {
  if (ctx->vc_exec) cudaGraphExecDestroy(ctx->vc_exec);
  ctx->vc_exec = nullptr;
  ctx->vc_valid = false;
  for (auto& e : ctx->pcg_exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
}

void free_mesh(hy_ctx* ctx) {
  if (ctx->side) cudaStreamSynchronize(ctx->side);  // a coarse setup in flight uses the level buffers
  for (cudaStream_t st : ctx->eig_st)
    if (st) cudaStreamSynchronize(st);
  ctx->side_pending = false;
  drop_graph(ctx);
  for (Level& L : ctx->lev)
    if (L.eig_exec) cudaGraphExecDestroy(L.eig_exec);
  for (auto& a : ctx->allocs) cudaFreeAsync(a.first, ctx->stream);
  ctx->allocs.clear();
  ctx->bytes = 0;
  ctx->lev.clear();
  ctx->tr.clear();
  ctx->d_err = nullptr;
  ctx->d_jmin = nullptr;
  ctx->d_partials = nullptr;
  ctx->d_scal = nullptr;
  ctx->d_face = nullptr;
  ctx->d_eig_scal = nullptr;
  ctx->d_eig_hist = nullptr;
  ctx->eig_hist_len = 0;
  ctx->d_usetup = ctx->d_udiff = nullptr;
  ctx->setup_valid = false;
  ctx->tmp64a = ctx->tmp64b = nullptr;
  ctx->tmp32a = ctx->tmp32b = ctx->tmp32c = nullptr;
  for (auto& p : ctx->f64) p = nullptr;
  ctx->state_ok = false;
  ctx->var = -1;
}

int lev_index(const hy_ctx* ctx, int level) { return level < 0 ? ctx->nlev - 1 : level; }

template <typename T>
CellArgs<T> cell_args(hy_ctx* ctx, Level& L) {
  CellArgs<T> a{};
  a.mat = L.d_mat;
  a.err = ctx->d_err;
  a.jmin_bits = ctx->d_jmin;
  a.g = L.g;
  a.nqp = L.nqp;
  if constexpr (std::is_same<T, double>::value) {
    a.mt = L.mt64;
    a.b = ctx->b64;
  } else if constexpr (std::is_same<T, float>::value) {
    a.mt = L.mt32;
    a.b = ctx->b32;
  } else {
    a.mt = L.mtff;
    a.b = ctx->bff;
  }
  a.mt.law = ctx->law;
  a.X64 = ctx->curved ? L.d_X64 : nullptr;
  return a;
}

// Per-precision views of a level: 0 FP64, 1 FP32, 2 double-float.
template <typename T> constexpr int prec_index() {
  return std::is_same<T, double>::value ? 0 : std::is_same<T, float>::value ? 1 : 2;
}
template <typename T> bool has_cache(const Level& L) {
  return prec_index<T>() == 0 ? L.has64 : prec_index<T>() == 1 ? L.has32 : L.hasff;
}
template <typename T> const T* cache_of(const Level& L);
template <> const double* cache_of<double>(const Level& L) { return L.d_c64; }
template <> const float* cache_of<float>(const Level& L) { return L.d_c32; }
template <> const ff* cache_of<ff>(const Level& L) { return L.d_cff; }
template <typename T> const vec_t<T>* ubar_of(const Level& L);
template <> const double* ubar_of<double>(const Level& L) { return L.d_u64; }
template <> const float* ubar_of<float>(const Level& L) { return L.d_u32; }
template <> const double* ubar_of<ff>(const Level& L) { return L.d_u64; }

ApplyFn<double> apply_fn(hy_ctx* ctx, double*, int var) {
  return ctx->dim == 2 ? apply_fn_f64_2d(ctx->n, var) : apply_fn_f64_3d(ctx->n, var);
}
ApplyFn<float> apply_fn(hy_ctx* ctx, float*, int var) {
  return ctx->dim == 2 ? apply_fn_f32_2d(ctx->n, var) : apply_fn_f32_3d(ctx->n, var);
}
ApplyFn<ff> apply_fn(hy_ctx* ctx, ff*, int var) {
  return ctx->dim == 2 ? apply_fn_ff_2d(ctx->n, var) : apply_fn_ff_3d(ctx->n, var);
}

// y = A~ x on level l in precision T (x zero on constrained dofs on read, y = x there). The vectors are
// of type vec_t<T> (FP64 for the double-float action).
// prepared: y already holds (constrained ? x : 0) (written by the kernel that produced x).
hy_status ensure_fp64_cache(hy_ctx* ctx, int l);

template <typename T>
hy_status vmult(hy_ctx* ctx, int l, const vec_t<T>* x, vec_t<T>* y, bool constrained_in = true, bool prepared = false) {
  using V = vec_t<T>;
  Level& L = ctx->lev[l];
  if constexpr (std::is_same<T, double>::value) {
    if (L.lazy64) HY_TRY(ensure_fp64_cache(ctx, l));
  }
  if (!has_cache<T>(L)) return fail(ctx, HY_ERR_STATE, "no Gauss-point cache of this precision on this level");
  CellArgs<T> a = cell_args<T>(ctx, L);
  a.x = x;
  a.y = y;
  a.cache = cache_of<T>(L);
  a.ubar = ubar_of<T>(L);
  a.pf = ctx->prefetch;
  if (constrained_in) {
    if (!prepared) launch_prep_out<V>(x, y, L.nnodes, ctx->dim, L.g, ctx->stream);
  } else {
    // raw operator rows of the free dofs applied to x including its constrained entries
    cudaMemsetAsync(y, 0, sizeof(V) * L.ndofs, ctx->stream);
    a.g.fm[0] = a.g.fm[1] = a.g.fm[2] = a.g.fm[3] = a.g.fm[4] = a.g.fm[5] = 0;
  }
  ApplyFn<T> fn = apply_fn(ctx, (T*)nullptr, L.var[prec_index<T>()]);
  if (!fn) return fail(ctx, HY_ERR_UNSUPPORTED, "no kernel for this dim/degree/variant");
  const int form = L.form[prec_index<T>()];
  fn(a, form < 0 ? FORM_POINT : form, ctx->stream);
  if (!constrained_in) launch_zero_constrained<V>(y, L.nnodes, ctx->dim, L.g, ctx->stream);
  return check_launch(ctx, prepared ? 1 : 2);
}

// The tangent action the solver uses on level l in the V-cycle precision T: on the finest level in FP64
// the double-float action when the solver parameter fine_dtype asks for it.
template <typename T>
hy_status level_apply(hy_ctx* ctx, int l, const T* x, T* y, bool prepared = false) {
  if constexpr (std::is_same<T, double>::value) {
    if (l == ctx->nlev - 1 && ctx->sp.fine_dtype == HY_FF && ctx->lev[l].hasff)
      return vmult<ff>(ctx, l, x, y, true, prepared);
  }
  return vmult<T>(ctx, l, x, y, true, prepared);
}

template <typename T>
hy_status dot(hy_ctx* ctx, const T* a, const T* b, long long n, double* out) {
  launch_dot<T>(a, b, n, ctx->d_partials, ctx->d_scal, ctx->stream);
  HY_TRY(check_launch(ctx, 2));
  HY_CK(cudaMemcpyAsync(out, ctx->d_scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  HY_CK(cudaStreamSynchronize(ctx->stream));
  return HY_OK;
}

template <typename T> T* wvec(Level& L, int i);
template <> double* wvec<double>(Level& L, int i) { return L.w64[i]; }
template <> float* wvec<float>(Level& L, int i) { return L.w32[i]; }
template <typename T> T* dinv_of(Level& L);
template <> double* dinv_of<double>(Level& L) { return L.d_dinv64; }
template <> float* dinv_of<float>(Level& L) { return L.d_dinv32; }
template <typename T> T* pw_of(Transfer& t);
template <> double* pw_of<double>(Transfer& t) { return t.d_pw64; }
template <> float* pw_of<float>(Transfer& t) { return t.d_pw32; }
template <typename T> T* rw_of(Transfer& t);
template <> double* rw_of<double>(Transfer& t) { return t.d_rw64; }
template <> float* rw_of<float>(Transfer& t) { return t.d_rw32; }
template <typename T> T* tmp_of(hy_ctx* c, int i);
template <> double* tmp_of<double>(hy_ctx* c, int i) { return i == 0 ? c->tmp64a : c->tmp64b; }
template <> float* tmp_of<float>(hy_ctx* c, int i) { return i == 0 ? c->tmp32a : c->tmp32b; }

// fine += P coarse (fine level l), constrained coarse entries read as zero, constrained fine rows zero.
// prep (or null): the last sweep also writes prep = (constrained ? new fine : 0), ready for an application
// of the new fine vector.
template <typename T>
hy_status prolongate_add(hy_ctx* ctx, int l, const T* coarse, T* fine, T* prep = nullptr) {
  Transfer& t = ctx->tr[l];
  const int d = ctx->dim;
  int Lin[3] = {t.Lc, t.Lc, t.Lc};
  const T* src = coarse;
  for (int ax = 0; ax < d; ++ax) {
    int Lout[3] = {Lin[0], Lin[1], Lin[2]};
    Lout[ax] = t.Lf;
    const bool last = ax == d - 1;
    T* dst = last ? fine : tmp_of<T>(ctx, ax & 1);
    launch_sweep<T>(src, dst, d, Lin, Lout, ax, t.d_pstart, pw_of<T>(t), t.Ep, last, ax == 0 ? &ctx->lev[l - 1].g : nullptr,
                    last ? &ctx->lev[l].g : nullptr, ctx->stream, nullptr, last ? prep : nullptr);
    src = dst;
    Lin[ax] = t.Lf;
  }
  return check_launch(ctx, d);
}

// coarse = P^T fine (fine level l), with the same constraint masks; with fine_minus, of fine - fine_minus
// (the residual formed inside the first sweep).
template <typename T>
hy_status restrict_to(hy_ctx* ctx, int l, const T* fine, T* coarse, const T* fine_minus = nullptr) {
  Transfer& t = ctx->tr[l];
  const int d = ctx->dim;
  int Lin[3] = {t.Lf, t.Lf, t.Lf};
  const T* src = fine;
  for (int ax = 0; ax < d; ++ax) {
    int Lout[3] = {Lin[0], Lin[1], Lin[2]};
    Lout[ax] = t.Lc;
    const bool last = ax == d - 1;
    T* dst = last ? coarse : tmp_of<T>(ctx, ax & 1);
    launch_sweep<T>(src, dst, d, Lin, Lout, ax, t.d_rstart, rw_of<T>(t), t.Er, false, ax == 0 ? &ctx->lev[l].g : nullptr,
                    last ? &ctx->lev[l - 1].g : nullptr, ctx->stream, ax == 0 ? fine_minus : nullptr);
    src = dst;
    Lin[ax] = t.Lc;
  }
  return check_launch(ctx, d);
}

// Level l-1 displacement = nodal interpolation of the level-l one (Sec. 6, carried down).
// (The same nodal interpolation carries a curved geometry's coordinates down: fine -> coarse of level l.)
hy_status interpolate_down_vec(hy_ctx* ctx, int l, const double* fine, double* coarse) {
  Transfer& t = ctx->tr[l];
  const int d = ctx->dim;
  int Lin[3] = {t.Lf, t.Lf, t.Lf};
  const double* src = fine;
  for (int ax = 0; ax < d; ++ax) {
    int Lout[3] = {Lin[0], Lin[1], Lin[2]};
    Lout[ax] = t.Lc;
    const bool last = ax == d - 1;
    double* dst = last ? coarse : tmp_of<double>(ctx, ax & 1);
    launch_sweep<double>(src, dst, d, Lin, Lout, ax, t.d_istart, t.d_iw64, t.Ei, false, nullptr, nullptr, ctx->stream);
    src = dst;
    Lin[ax] = t.Lc;
  }
  return check_launch(ctx, d);
}
hy_status interpolate_down(hy_ctx* ctx, int l) {
  return interpolate_down_vec(ctx, l, ctx->lev[l].d_u64, ctx->lev[l - 1].d_u64);
}

// Chebyshev iteration of the given degree on [lo, hi] for A~ x = b on level l (Saad, Alg. 12.1),
// Jacobi preconditioned; x0_zero starts from zero. Uses the level's r, d, t vectors. t_ready: t already holds
// (constrained ? x : 0), the output of the first application prepared; prep_x: the last update leaves t so
// prepared for an application of the final x.
template <typename T>
hy_status chebyshev(hy_ctx* ctx, int l, const T* b, T* x, bool x0_zero, int degree, double lo, double hi,
                    bool t_ready = false, bool prep_x = false) {
  Level& L = ctx->lev[l];
  T* r = wvec<T>(L, 2);
  T* dd = wvec<T>(L, 3);
  T* t = wvec<T>(L, 4);
  const T* dinv = dinv_of<T>(L);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (!x0_zero) HY_TRY(level_apply<T>(ctx, l, x, t, t_ready));
  // each update also prepares t for the next application of d, or after the last one of x (no separate
  // prep_out launch)
  launch_cheb_init<T>(b, t, dinv, r, dd, x, T(1.0 / theta), x0_zero, L.ndofs, degree > 1 || prep_x ? &L.g : nullptr,
                      ctx->dim, ctx->stream, degree == 1 && prep_x);
  HY_TRY(check_launch(ctx, 1));
  for (int j = 1; j < degree; ++j) {
    HY_TRY(level_apply<T>(ctx, l, dd, t, true));
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const bool last = j + 1 == degree;
    launch_cheb_step<T>(t, dinv, r, dd, x, T(rho_new * rho), T(2.0 * rho_new / delta), L.ndofs,
                        !last || prep_x ? &L.g : nullptr, ctx->dim, ctx->stream, last && prep_x);
    HY_TRY(check_launch(ctx, 1));
    rho = rho_new;
  }
  return HY_OK;
}

bool level_f32(const hy_ctx* ctx, int l) { return ctx->mixed && l > 0; }

// V-cycle on level l for the level's b (w[0]) into x (w[1]), zero initial guess (Sec. 6, Sec. 7).
hy_status vcycle_level(hy_ctx* ctx, int l);

template <typename T>
hy_status vcycle_typed(hy_ctx* ctx, int l) {
  Level& L = ctx->lev[l];
  T* b = wvec<T>(L, 0);
  T* x = wvec<T>(L, 1);
  const double lo = ctx->sp.cheb_lo * L.lmax, hi = ctx->sp.cheb_hi * L.lmax;
  // Every smoothing sweep leaves t prepared for the application of its x that follows it (the next sweep's
  // first one, or the residual's), and the prolongation leaves t prepared for the post-smoother's first one.
  for (int s = 0; s < ctx->sp.cheb_sweeps; ++s)
    HY_TRY(chebyshev<T>(ctx, l, b, x, s == 0, ctx->sp.cheb_degree, lo, hi, s > 0, true));
  T* t = wvec<T>(L, 4);
  HY_TRY(level_apply<T>(ctx, l, x, t, true));
  // the residual b - t is formed inside the restriction's first sweep
  Level& C = ctx->lev[l - 1];
  const bool cf32 = level_f32(ctx, l - 1);
  if ((sizeof(T) == 4) == cf32) {
    HY_TRY(restrict_to<T>(ctx, l, b, wvec<T>(C, 0), t));
  } else {  // float fine level above the FP64 coarsest level
    HY_TRY(restrict_to<T>(ctx, l, b, (T*)ctx->tmp32c, t));
    launch_convert<float, double>((const float*)ctx->tmp32c, C.w64[0], C.ndofs, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
  }
  HY_TRY(vcycle_level(ctx, l - 1));
  if ((sizeof(T) == 4) == cf32) {
    HY_TRY(prolongate_add<T>(ctx, l, wvec<T>(C, 1), x, t));
  } else {
    launch_convert<double, float>(C.w64[1], ctx->tmp32c, C.ndofs, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
    HY_TRY(prolongate_add<T>(ctx, l, (const T*)ctx->tmp32c, x, t));
  }
  for (int s = 0; s < ctx->sp.cheb_sweeps; ++s)
    HY_TRY(chebyshev<T>(ctx, l, b, x, false, ctx->sp.cheb_degree, lo, hi, true, s + 1 < ctx->sp.cheb_sweeps));
  return HY_OK;
}

hy_status vcycle_level(hy_ctx* ctx, int l) {
  if (l == 0) {
    Level& L = ctx->lev[0];
    if (ctx->sp.coarse_solver >= 1) {
      HY_CK(cudaMemsetAsync(L.w64[1], 0, sizeof(double) * L.ndofs, ctx->stream));
      if (L.nfree) launch_dense_gemv(L.d_Aresult, L.w64[0], L.w64[1], L.nfree, L.d_free_idx, ctx->stream);
      return check_launch(ctx, 1);
    }
    return chebyshev<double>(ctx, 0, L.w64[0], L.w64[1], true, ctx->coarse_deg, ctx->coarse_lo, ctx->coarse_hi);
  }
  return level_f32(ctx, l) ? vcycle_typed<float>(ctx, l) : vcycle_typed<double>(ctx, l);
}

// The V-cycle from the finest level's b to its x, replayed from a CUDA graph captured on a private
// stream the first time after each change of linearisation (the graph holds the Chebyshev
// coefficients and eigenvalue bounds as kernel arguments, so it is re-captured when they change).
hy_status vcycle_body(hy_ctx* ctx) {
  const int top = ctx->nlev - 1;
  if (!ctx->use_graphs) return vcycle_level(ctx, top);
  if (!ctx->vc_valid) {
    if (!ctx->cap_stream) HY_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    const long long l0 = ctx->launches;
    ctx->stream = ctx->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      ctx->stream = saved;
      return fail(ctx, HY_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    }
    const hy_status st = vcycle_level(ctx, top);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->stream = saved;
    ctx->vc_nodes = ctx->launches - l0;
    ctx->launches = l0;
    if (st != HY_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (st != HY_OK) return st;
      return fail(ctx, HY_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    drop_graph(ctx);
    e = cudaGraphInstantiate(&ctx->vc_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, HY_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    ctx->vc_valid = true;
  }
  HY_CK(cudaGraphLaunch(ctx->vc_exec, ctx->stream));
  ctx->launches += ctx->vc_nodes;
  return HY_OK;
}

// z = V r on the finest level (FP64 in/out).
hy_status vcycle_top(hy_ctx* ctx, const double* r, double* z) {
  if (!ctx->coarse_spd)
    return fail(ctx, HY_ERR_NOCONV,
                "coarsest-level tangent is not positive definite (smallest Ritz value " + std::to_string(ctx->coarse_lo) +
                    "); the Chebyshev coarse solver needs an SPD operator");
  const int top = ctx->nlev - 1;
  Level& L = ctx->lev[top];
  if (level_f32(ctx, top)) {
    launch_convert<double, float>(r, L.w32[0], L.ndofs, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
    HY_TRY(vcycle_body(ctx));
    launch_convert<float, double>(L.w32[1], z, L.ndofs, ctx->stream);
    return check_launch(ctx, 1);
  }
  HY_CK(cudaMemcpyAsync(L.w64[0], r, sizeof(double) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
  HY_TRY(vcycle_body(ctx));
  HY_CK(cudaMemcpyAsync(z, L.w64[1], sizeof(double) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
  return HY_OK;
}

constexpr int EIG_GRAPH_MAX_ITERS = 64;
// per level: 8 scalars, the alpha and beta history of a graph-length run, the dot partial sums
constexpr int EIG_BUF_LEN = 8 + 2 * EIG_GRAPH_MAX_ITERS + DOT_BLOCKS;

// Device buffers of one eigenvalue-estimate run.
struct EigBufs {
  double* sc;        // {rz, rz0, pq, rzn, alpha, beta, stopped, count}
  double* hist;      // alpha history [iters], then beta history [iters]; follows sc contiguously
  double* partials;  // dot partial sums
};
EigBufs ctx_eig_bufs(hy_ctx* ctx) { return {ctx->d_eig_scal, ctx->d_eig_hist, ctx->d_partials}; }
EigBufs level_eig_bufs(Level& L) {
  return {L.d_eigbuf, L.d_eigbuf + 8, L.d_eigbuf + 8 + 2 * EIG_GRAPH_MAX_ITERS};
}

// Enqueues `iters` Jacobi-PCG iterations on level l (Ritz values of D^{-1} A~ come from their coefficients),
// start vector from SplitMix64 with seed l, constrained entries zero (Sec. 7), on the context's current
// stream. A run of at most EIG_GRAPH_MAX_ITERS iterations with graphs enabled is enqueued without any host
// synchronisation; a longer one looks at the device-side stop flag now and then.
template <typename T>
hy_status eig_enqueue(hy_ctx* ctx, int l, int iters, const EigBufs& eb) {
  Level& L = ctx->lev[l];
  T* r = wvec<T>(L, 2);
  T* z = wvec<T>(L, 3);
  T* q = wvec<T>(L, 4);
  T* p = wvec<T>(L, 1);
  const T* dinv = dinv_of<T>(L);
  double* sc = eb.sc;
  double* hist = eb.hist;
  double* part = eb.partials;
  launch_splitmix<T>(r, L.ndofs, (unsigned long long)l, ctx->stream);
  launch_zero_constrained<T>(r, L.nnodes, ctx->dim, L.g, ctx->stream);
  launch_mul<T>(dinv, r, z, L.ndofs, ctx->stream);
  HY_CK(cudaMemcpyAsync(p, z, sizeof(T) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
  HY_CK(cudaMemsetAsync(sc, 0, sizeof(double) * 8, ctx->stream));
  launch_dot<T>(r, z, L.ndofs, part, sc + 0, ctx->stream);  // rz
  HY_CK(cudaMemcpyAsync(sc + 1, sc + 0, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));  // rz0
  HY_TRY(check_launch(ctx, 5));
  // CG iterations with every scalar on the device; the coefficient history comes back once at the end
  auto iteration = [&](int it) -> hy_status {
    HY_TRY(level_apply<T>(ctx, l, p, q));
    launch_dot<T>(p, q, L.ndofs, part, sc + 2, ctx->stream);  // pq
    launch_eig_alpha(sc, hist, it, ctx->stream);
    launch_axpy_dev<T>(sc + 4, -1.0, q, r, L.ndofs, ctx->stream);  // r -= alpha q
    launch_mul<T>(dinv, r, z, L.ndofs, ctx->stream);               // z = D^{-1} r
    launch_dot<T>(r, z, L.ndofs, part, sc + 3, ctx->stream);       // rzn
    launch_eig_beta(sc, hist, it, iters, ctx->stream);
    launch_xpay_dev<T>(z, sc + 5, p, p, L.ndofs, ctx->stream);     // p = z + beta p
    return check_launch(ctx, 9);
  };
  if (ctx->use_graphs && iters <= EIG_GRAPH_MAX_ITERS) {
    // A short run (the smoother estimates) is one CUDA graph: once the device-side stop flag is set the
    // remaining iterations change nothing. The graph is kept per level and replayed at later
    // linearisations as long as the arguments of its kernels are the same (the signature below: the
    // action's kernel arguments, form and precision, the vectors, scalars, iteration count).
    std::vector<unsigned char> sig;
    auto add = [&sig](const void* v, size_t bytes) {
      const unsigned char* b = static_cast<const unsigned char*>(v);
      sig.insert(sig.end(), b, b + bytes);
    };
    const bool ff_top = std::is_same<T, double>::value && l == ctx->nlev - 1 && ctx->sp.fine_dtype == HY_FF && L.hasff;
    if (ff_top) {
      CellArgs<ff> ca = cell_args<ff>(ctx, L);
      ca.cache = cache_of<ff>(L);
      ca.ubar = ubar_of<ff>(L);
      add(&ca, sizeof(ca));
      add(&L.form[2], sizeof(int));
      add(&L.var[2], sizeof(int));
    } else {
      CellArgs<T> ca = cell_args<T>(ctx, L);
      ca.cache = cache_of<T>(L);
      ca.ubar = ubar_of<T>(L);
      add(&ca, sizeof(ca));
      add(&L.form[prec_index<T>()], sizeof(int));
      add(&L.var[prec_index<T>()], sizeof(int));
    }
    const void* ptrs[9] = {r, z, q, p, dinv, sc, hist, part, ctx->d_err};
    add(ptrs, sizeof(ptrs));
    add(&iters, sizeof(iters));
    add(&ctx->prefetch, sizeof(ctx->prefetch));
    const int ptag = prec_index<T>() + (ff_top ? 8 : 0);
    add(&ptag, sizeof(ptag));
    if (!L.eig_exec || sig != L.eig_sig) {
      if (L.eig_exec) cudaGraphExecDestroy(L.eig_exec);
      L.eig_exec = nullptr;
      if (!ctx->cap_stream) HY_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      cudaStream_t saved = ctx->stream;
      const long long l0 = ctx->launches;
      ctx->stream = ctx->cap_stream;
      cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        ctx->stream = saved;
        return fail(ctx, HY_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
      }
      hy_status st = HY_OK;
      for (int it = 0; it < iters && st == HY_OK; ++it) st = iteration(it);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(ctx->cap_stream, &g);
      ctx->stream = saved;
      L.eig_nodes = ctx->launches - l0;
      ctx->launches = l0;
      if (st != HY_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st != HY_OK) return st;
        return fail(ctx, HY_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
      }
      e = cudaGraphInstantiate(&L.eig_exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        L.eig_exec = nullptr;
        return fail(ctx, HY_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
      L.eig_sig.swap(sig);
    }
    HY_CK(cudaGraphLaunch(L.eig_exec, ctx->stream));
    ctx->launches += L.eig_nodes;
  } else {
    for (int it = 0; it < iters; ++it) {
      HY_TRY(iteration(it));
      if ((it & 31) == 31 && it + 1 < iters) {  // look at the stop flag now and then (one host sync)
        double stopped = 0.0;
        HY_CK(cudaMemcpyAsync(&stopped, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        HY_CK(cudaStreamSynchronize(ctx->stream));
        if (stopped != 0.0) break;
      }
    }
  }
  return HY_OK;
}

// Extreme Ritz values from a finished run's scalars hs (8) and coefficient history hh (alpha [iters], then
// beta [iters]): the Lanczos tridiagonal of the CG coefficients, over the iterations taken up to and
// including the one whose residual met the stop test.
hy_status eig_extremes(hy_ctx* ctx, const double* hs, const double* hh, int iters, double& lmin, double& lmax) {
  int m = (int)hs[7];
  if (hs[6] == 0.0) m = iters;
  if (m == 0) return fail(ctx, HY_ERR_STATE, "eigenvalue estimate: no iterations");
  std::vector<double> diag(m), off(std::max(m - 1, 1));
  for (int j = 0; j < m; ++j) {
    diag[j] = 1.0 / hh[j] + (j > 0 ? hh[iters + j - 1] / hh[j - 1] : 0.0);
    if (j + 1 < m) off[j] = std::sqrt(hh[iters + j]) / hh[j];
  }
  tridiag_extremes(diag, off, lmin, lmax);
  return HY_OK;
}

// One run on the context's stream with the context's buffers, waited for.
template <typename T>
hy_status eig_estimate(hy_ctx* ctx, int l, int iters, double& lmin, double& lmax) {
  if ((long long)ctx->eig_hist_len < 2LL * iters) return fail(ctx, HY_ERR_STATE, "eigenvalue history too short");
  const EigBufs eb = ctx_eig_bufs(ctx);
  HY_TRY(eig_enqueue<T>(ctx, l, iters, eb));
  double hs[8];
  std::vector<double> hh((size_t)2 * iters);
  HY_CK(cudaMemcpyAsync(hs, eb.sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  HY_CK(cudaMemcpyAsync(hh.data(), eb.hist, sizeof(double) * 2 * iters, cudaMemcpyDeviceToHost, ctx->stream));
  HY_CK(cudaStreamSynchronize(ctx->stream));
  return eig_extremes(ctx, hs, hh.data(), iters, lmin, lmax);
}

// The smoother estimates of every level above the coarsest (the level precision of the V-cycle). A level's
// run reads only its own tangent and diagonal and writes only its own vectors and buffers, so with graphs
// the runs go side by side, each on a stream of its own: one fork, one join and one host synchronisation
// for all levels. Otherwise they run one after another.
hy_status smoother_eig_estimates(hy_ctx* ctx) {
  const int nl = ctx->nlev, iters = ctx->sp.eig_iters;
  if (!ctx->use_graphs || iters > EIG_GRAPH_MAX_ITERS) {
    for (int l = 1; l < nl; ++l) {
      double lmin, lmax;
      if (level_f32(ctx, l)) HY_TRY(eig_estimate<float>(ctx, l, iters, lmin, lmax));
      else HY_TRY(eig_estimate<double>(ctx, l, iters, lmin, lmax));
      ctx->lev[l].lmax = lmax;
    }
    return HY_OK;
  }
  if (nl < 2) return HY_OK;
  while ((int)ctx->eig_st.size() < nl) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    HY_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ctx->eig_st.push_back(st);
    HY_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ctx->eig_ev.push_back(ev);
  }
  if (!ctx->ev_eig_fork) HY_CK(cudaEventCreateWithFlags(&ctx->ev_eig_fork, cudaEventDisableTiming));
  HY_CK(cudaEventRecord(ctx->ev_eig_fork, ctx->stream));
  cudaStream_t main = ctx->stream;
  hy_status st = HY_OK;
  for (int l = 1; l < nl; ++l) {
    HY_CK(cudaStreamWaitEvent(ctx->eig_st[l], ctx->ev_eig_fork, 0));
    ctx->stream = ctx->eig_st[l];
    if (st == HY_OK)
      st = level_f32(ctx, l) ? eig_enqueue<float>(ctx, l, iters, level_eig_bufs(ctx->lev[l]))
                             : eig_enqueue<double>(ctx, l, iters, level_eig_bufs(ctx->lev[l]));
    ctx->stream = main;
    // joined even after a failure, so that nothing of the run outlives the call
    HY_CK(cudaEventRecord(ctx->eig_ev[l], ctx->eig_st[l]));
    HY_CK(cudaStreamWaitEvent(main, ctx->eig_ev[l], 0));
  }
  if (st != HY_OK) return st;
  const size_t per = 8 + 2 * (size_t)iters;  // scalars, then the history that follows them
  std::vector<double> h((size_t)nl * per);
  for (int l = 1; l < nl; ++l)
    HY_CK(cudaMemcpyAsync(h.data() + l * per, ctx->lev[l].d_eigbuf, sizeof(double) * per, cudaMemcpyDeviceToHost,
                          main));
  HY_CK(cudaStreamSynchronize(main));
  for (int l = 1; l < nl; ++l) {
    double lmin, lmax;
    HY_TRY(eig_extremes(ctx, h.data() + l * per, h.data() + l * per + 8, iters, lmin, lmax));
    ctx->lev[l].lmax = lmax;
  }
  return HY_OK;
}

hy_status ensure_level_vectors(hy_ctx* ctx, int l, bool f32) {
  Level& L = ctx->lev[l];
  for (int i = 0; i < 5; ++i) {
    if (f32) {
      if (!L.w32[i]) HY_TRY(dalloc(ctx, &L.w32[i], L.ndofs));
    } else {
      if (!L.w64[i]) HY_TRY(dalloc(ctx, &L.w64[i], L.ndofs));
    }
  }
  return HY_OK;
}

template <typename TOUT> TOUT*& cache_buf(Level& L);
template <> double*& cache_buf<double>(Level& L) { return L.d_c64; }
template <> float*& cache_buf<float>(Level& L) { return L.d_c32; }
template <> ff*& cache_buf<ff>(Level& L) { return L.d_cff; }
template <typename TOUT> size_t& cache_len(Level& L);
template <> size_t& cache_len<double>(Level& L) { return L.c64_len; }
template <> size_t& cache_len<float>(Level& L) { return L.c32_len; }
template <> size_t& cache_len<ff>(Level& L) { return L.cff_len; }

// Allocates level l's cache of element type TOUT for variant var and, unless only_allocate, launches the
// state kernel that fills it.
template <typename TOUT>
hy_status build_cache(hy_ctx* ctx, int l, int var, bool only_allocate = false) {
  Level& L = ctx->lev[l];
  const int cb = layout_cells<TOUT>(ctx->dim, ctx->n);
  const size_t nblocks = (size_t)((L.g.ncells + cb - 1) / cb);
  const size_t len = std::max<size_t>(1, (size_t)cache_values(var, ctx->dim) * layout_row<TOUT>(ctx->dim, ctx->n) * nblocks);
  TOUT*& buf = cache_buf<TOUT>(L);
  size_t& cur = cache_len<TOUT>(L);
  if (cur < len) {
    dfree(ctx, buf);
    buf = nullptr;
    HY_TRY(dalloc(ctx, &buf, len));
    cur = len;
  }
  if (only_allocate) return HY_OK;
  CellArgs<double> a = cell_args<double>(ctx, L);
  a.u64 = L.d_u64;
  StateFn<TOUT> fn;
  if constexpr (std::is_same<TOUT, double>::value) fn = state_fn_f64(ctx->dim, ctx->n, var);
  else if constexpr (std::is_same<TOUT, float>::value) fn = state_fn_f32(ctx->dim, ctx->n, var);
  else fn = state_fn_ff(ctx->dim, ctx->n, var);
  if (!fn) return fail(ctx, HY_ERR_UNSUPPORTED, "no state kernel");
  fn(a, buf, ctx->stream);
  return check_launch(ctx, 1);
}

hy_status check_error_word(hy_ctx* ctx, const char* where) {
  unsigned h = 0;
  HY_CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  HY_CK(cudaStreamSynchronize(ctx->stream));
  if (h) {
    HY_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
    if (h & ERRBIT_TIMEOUT) return fail(ctx, HY_ERR_TIMEOUT, std::string(where) + ": a bounded device wait gave up");
    return fail(ctx, HY_ERR_JNEG, std::string(where) + ((h & ERRBIT_NAN) ? ": NaN in J" : ": J <= 0 at a Gauss point"));
  }
  return HY_OK;
}

// Exact coarse solve: dense constrained tangent of level 0, inverted in place (Gauss-Jordan, SPD so no
// pivoting); a pivot <= 0 marks the level as not positive definite, like a negative Ritz value would.
hy_status coarse_direct_setup(hy_ctx* ctx) {
  Level& C = ctx->lev[0];
  if (C.ndofs > 6000) return fail(ctx, HY_ERR_UNSUPPORTED, "exact coarse solve needs a coarsest level of at most 6000 dofs");
  if (!C.d_Ainv) {
    // free-dof numbering of the coarsest level (host, from the face masks)
    std::vector<int> cidx(C.ndofs, -1), fidx;
    const int Lc = C.g.L;
    for (long long nd = 0; nd < C.nnodes; ++nd) {
      const int i0 = (int)(nd % Lc), i1 = (int)((nd / Lc) % Lc), i2 = ctx->dim == 3 ? (int)(nd / ((long long)Lc * Lc)) : 0;
      uint32_t cm = 0;
      if (i0 == 0) cm |= C.g.fm[0];
      if (i0 == Lc - 1) cm |= C.g.fm[1];
      if (i1 == 0) cm |= C.g.fm[2];
      if (i1 == Lc - 1) cm |= C.g.fm[3];
      if (ctx->dim == 3 && i2 == 0) cm |= C.g.fm[4];
      if (ctx->dim == 3 && i2 == Lc - 1) cm |= C.g.fm[5];
      for (int c = 0; c < ctx->dim; ++c)
        if (!((cm >> c) & 1u)) {
          cidx[nd * ctx->dim + c] = (int)fidx.size();
          fidx.push_back((int)(nd * ctx->dim + c));
        }
    }
    C.nfree = (long long)fidx.size();
    const size_t nf = (size_t)std::max<long long>(C.nfree, 1);
    HY_TRY(dalloc(ctx, &C.d_Ainv, nf * nf));
    HY_TRY(dalloc(ctx, &C.d_Awork, nf * nf));
    HY_TRY(dalloc(ctx, &C.d_inv_piv, 32 * 32 + 64 * nf));  // blocked Gauss-Jordan panels
    HY_TRY(dalloc(ctx, &C.d_free_idx, nf));
    HY_TRY(dalloc(ctx, &C.d_cidx, C.ndofs));
    if (C.nfree) HY_CK(cudaMemcpyAsync(C.d_free_idx, fidx.data(), sizeof(int) * C.nfree, cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(C.d_cidx, cidx.data(), sizeof(int) * C.ndofs, cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaStreamSynchronize(ctx->stream));
  }
  const long long n = C.nfree;
  ctx->coarse_lo = ctx->coarse_hi = 0.0;
  ctx->coarse_deg = 0;
  ctx->coarse_spd = true;
  if (n == 0) return HY_OK;
  // Assembly and inversion go to the side stream, after the work queued so far on the context's stream
  // (the carried-down coarse displacement): they need nothing else of the linearisation and overlap its
  // state builds, diagonals and eigenvalue estimates. coarse_direct_finish joins them.
  if (!ctx->side) {
    // the longest chain of the linearisation: its blocks go first, the main stream's work fills in around them
    int lo = 0, hi = 0;
    HY_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    HY_CK(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi));
    HY_CK(cudaEventCreateWithFlags(&ctx->ev_side_fork, cudaEventDisableTiming));
    HY_CK(cudaEventCreate(&ctx->ev_side_join));
    HY_CK(cudaEventCreate(&ctx->ev_side_start));
    HY_CK(cudaMallocHost((void**)&ctx->h_err_side, sizeof(unsigned)));
  }
  HY_CK(cudaEventRecord(ctx->ev_side_fork, ctx->stream));
  HY_CK(cudaStreamWaitEvent(ctx->side, ctx->ev_side_fork, 0));
  HY_CK(cudaEventRecord(ctx->ev_side_start, ctx->side));
  ctx->side_timed = true;
  unsigned* err = ctx->d_err + 1;
  HY_CK(cudaMemsetAsync(C.d_Ainv, 0, sizeof(double) * n * n, ctx->side));
  HY_CK(cudaMemsetAsync(err, 0, sizeof(unsigned), ctx->side));
  CellArgs<double> a = cell_args<double>(ctx, C);
  a.u64 = C.d_u64;
  a.err = err;
  launch_assemble_dense(ctx->dim, ctx->n, a, C.d_Ainv, n, C.d_cidx, ctx->side);
  HY_TRY(check_launch(ctx, 1));
  const bool ff_arith = ctx->sp.coarse_solver == 2;
  C.d_Aresult = launch_gj_invert(C.d_Ainv, C.d_Awork, n, C.d_inv_piv, err, ff_arith, ctx->side);
  HY_TRY(check_launch(ctx, (int)(3 * ((n + 31) / 32)) + 1 + (ff_arith ? 2 : 0)));
  HY_CK(cudaMemcpyAsync(ctx->h_err_side, err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->side));
  HY_CK(cudaEventRecord(ctx->ev_side_join, ctx->side));
  ctx->side_pending = true;
  return HY_OK;
}

// Join the coarse setup of the side stream: the context's stream waits for it, and its error word decides.
hy_status coarse_direct_finish(hy_ctx* ctx) {
  if (!ctx->side_pending) return HY_OK;
  ctx->side_pending = false;
  HY_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_side_join, 0));
  HY_CK(cudaEventSynchronize(ctx->ev_side_join));
  const unsigned h = *ctx->h_err_side;
  if (h & (ERRBIT_JNEG | ERRBIT_NAN)) return fail(ctx, HY_ERR_JNEG, "coarse level: J <= 0 at a Gauss point");
  ctx->coarse_spd = !(h & ERRBIT_NONSPD);
  return HY_OK;
}

// ---- autotuner of the tangent-action kernel form -----------------------------------------------------
// Key: (dim, degree, variant, precision, log2 of the level's cell count). Decisions are shared by every
// context of the process and, when HY_TUNE_FILE names a file, read from it at the first tuning and
// rewritten with every new decision, as a JSON array with one object per line:
//   {"dim": 3, "degree": 2, "variant": "NC", "precision": "f64", "cells_log2": 15, "threads_per_cell": "point"}
using TuneKey = std::tuple<int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
bool g_tune_loaded = false;
const char* const kVarNames[9] = {"T4", "T2", "FC", "SC", "NC", "none", "FCG", "SCG", "NCG"};
const char* const kFormNames[4] = {"point", "line", "line_persistent", "plane"};
const char* const kPrecNames[3] = {"f64", "f32", "ff"};

int name_index(const char* s, const char* const* names, int n) {
  for (int i = 0; i < n; ++i)
    if (std::strcmp(s, names[i]) == 0) return i;
  return -1;
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("HY_TUNE_FILE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    int d = 0, k = 0, b = 0;
    char var[8] = {}, prec[8] = {}, form[24] = {};
    if (std::sscanf(line, " {\"dim\": %d, \"degree\": %d, \"variant\": \"%7[^\"]\", \"precision\": \"%7[^\"]\", "
                          "\"cells_log2\": %d, \"threads_per_cell\": \"%23[^\"]\"",
                    &d, &k, var, prec, &b, form) != 6)
      continue;  // the brackets and anything unrecognised
    const int v = name_index(var, kVarNames, 9), fm = name_index(form, kFormNames, 4);
    const int p = name_index(prec, kPrecNames, 3);
    if (v >= 0 && fm >= 0 && p >= 0) g_tune[TuneKey{d, k, v, p, b}] = fm;
  }
  std::fclose(f);
}

void tune_save_locked() {
  const char* path = std::getenv("HY_TUNE_FILE");
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "[\n");
  size_t i = 0;
  for (const auto& kv : g_tune) {
    const TuneKey& t = kv.first;
    std::fprintf(f,
                 "  {\"dim\": %d, \"degree\": %d, \"variant\": \"%s\", \"precision\": \"%s\", \"cells_log2\": %d, "
                 "\"threads_per_cell\": \"%s\"}%s\n",
                 std::get<0>(t), std::get<1>(t), kVarNames[std::get<2>(t)], kPrecNames[std::get<3>(t)],
                 std::get<4>(t), kFormNames[kv.second], ++i < g_tune.size() ? "," : "");
  }
  std::fprintf(f, "]\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

template <typename T>
hy_status autotune_level(hy_ctx* ctx, int l) {
  using V = vec_t<T>;
  Level& L = ctx->lev[l];
  const int dt = prec_index<T>();
  if (ctx->sp.kernel_form >= 0) {
    L.form[dt] = ctx->sp.kernel_form;
    return HY_OK;
  }
  int bucket = 0;
  for (long long c = L.g.ncells; c > 1; c >>= 1) ++bucket;
  const TuneKey key{ctx->dim, ctx->k, L.var[dt], dt, bucket};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      L.form[dt] = it->second;
      return HY_OK;
    }
  }
  // time both forms on this level's cache: one warm-up application each, then three rounds that
  // alternate the forms, each timing four back-to-back applications (hides the host launch latency on
  // small levels); the best round of each form decides
  V* x = wvec<V>(L, 2);
  V* y = wvec<V>(L, 3);
  launch_splitmix<V>(x, L.ndofs, 12345ULL, ctx->stream);
  HY_TRY(check_launch(ctx, 1));
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  HY_CK(cudaEventCreate(&ev.a));
  HY_CK(cudaEventCreate(&ev.b));
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  // FP32 also has the persistent line form (next cache chunk copied in under the current block's work)
  // and, in 3D, the plane form
  const int nforms = std::is_same<T, float>::value ? (ctx->dim == 3 && ctx->n <= PLANE_MAX_N ? 4 : 3) : 2;
  float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
  for (int form = 0; form < nforms; ++form) {
    L.form[dt] = form;
    HY_TRY(vmult<T>(ctx, l, x, y));
  }
  for (int r = 0; r < 3; ++r) {
    for (int form = 0; form < nforms; ++form) {
      L.form[dt] = form;
      cudaEventRecord(e0, ctx->stream);
      for (int q = 0; q < 4; ++q) HY_TRY(vmult<T>(ctx, l, x, y));
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best[form] = std::min(best[form], 0.25f * ms);
    }
  }
  int choice = FORM_POINT;
  for (int form = 1; form < nforms; ++form)
    if (best[form] < best[choice]) choice = form;
  L.form[dt] = choice;
  if (ctx->verbose)
    std::fprintf(stderr,
                 "[hy] autotune dim %d k %d var %d %s cells 2^%d: point %.3f ms, line %.3f ms, persistent %.3f ms, "
                 "plane %.3f ms -> %s\n",
                 ctx->dim, ctx->k, L.var[dt], kPrecNames[dt], bucket, best[0], best[1], nforms > 2 ? best[2] : 0.f,
                 nforms > 3 ? best[3] : 0.f, kFormNames[choice]);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune.emplace(key, choice).second) tune_save_locked();
  return HY_OK;
}

// Builds the finest level's deferred FP64 cache (and picks its kernel form) on the first FP64 action that
// needs it. Not inside a stream capture: the build synchronises with the host.
hy_status ensure_fp64_cache(hy_ctx* ctx, int l) {
  Level& L = ctx->lev[l];
  if (!L.lazy64) return HY_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HY_CK(cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(ctx, HY_ERR_STATE, "FP64 cache needed inside a capture");
  HY_TRY(build_cache<double>(ctx, l, L.var[0]));
  HY_TRY(check_error_word(ctx, "FP64 state build"));
  L.lazy64 = false;
  L.has64 = true;
  return autotune_level<double>(ctx, l);
}

// Verbose phase timer of set_displacement (synchronises the stream, so only when HY_VERBOSE=1).
// Phase events of set_displacement: recorded on the context's stream at the start and after each phase (no
// synchronisation); setup_phases_ms reads them once the stream has been synchronised. With HY_VERBOSE=1 each
// phase is also synchronised and printed.
struct PhaseTimer {
  hy_ctx* ctx;
  int next = 0;
  std::chrono::steady_clock::time_point t;
  explicit PhaseTimer(hy_ctx* c) : ctx(c), t(std::chrono::steady_clock::now()) {
    if (!ctx->ev_phase[0])
      for (cudaEvent_t& e : ctx->ev_phase) cudaEventCreate(&e);
    ctx->phases_recorded = 0;
    record();
  }
  void record() {
    if (next < SETUP_PHASES + 1 && cudaEventRecord(ctx->ev_phase[next], ctx->stream) == cudaSuccess) {
      ++next;
      ctx->phases_recorded = next;
    }
  }
  void mark(const char* what) {
    record();
    if (!ctx->verbose) return;
    cudaStreamSynchronize(ctx->stream);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[hy] set_displacement %-14s %8.3f ms\n", what,
                 std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

// Device time of the phases of the last set_displacement (the stream must have reached its end): carry down,
// state and diagonal, autotune, smoother eigenvalue estimates, coarse setup (the join of the exact inverse or
// the coarse eigenvalue estimate), then the side stream's exact coarse inverse itself (0 if none).
void setup_phases_ms(hy_ctx* ctx, double out[SETUP_PHASES + 1]) {
  for (int i = 0; i <= SETUP_PHASES; ++i) out[i] = 0.0;
  for (int i = 0; i + 1 < ctx->phases_recorded; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_phase[i], ctx->ev_phase[i + 1]) == cudaSuccess) out[i] = ms;
  }
  if (ctx->side_timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_side_start, ctx->ev_side_join) == cudaSuccess) out[SETUP_PHASES] = ms;
  }
}

hy_status set_displacement(hy_ctx* ctx, const double* u, int var, bool mixed) {
  const Range range("set_displacement");
  if (ctx->nlev == 0) return fail(ctx, HY_ERR_STATE, "mesh not set up");
  PhaseTimer pt(ctx);
  for (int l = 0; l < ctx->nlev; ++l)
    if (!ctx->lev[l].mat_set) return fail(ctx, HY_ERR_STATE, "material not set on level " + std::to_string(l));
  if (var < 0 || var > 4) return fail(ctx, HY_ERR_ARG, "variant out of range");
  // Curved cells or the second law: FC, SC and NC run their general builds (the reference map per Gauss
  // point in the cache, the volumetric function chosen at run time); T4 and T2 fold both into their state.
  const bool general = ctx->curved || ctx->law != HY_LAW_LOG2;
  auto build_of = [general](int v) { return (general && v >= VAR_FC && v <= VAR_NC) ? v - VAR_FC + VAR_FCG : v; };
  if (general && ctx->sp.fine_dtype == HY_FF && var >= VAR_FC)
    return fail(ctx, HY_ERR_UNSUPPORTED,
                "the double-float action of FC/SC/NC is built for the lattice and the paper's law only");
  ctx->state_ok = false;
  drop_graph(ctx);
  ctx->var = var;
  ctx->mixed = mixed;
  {
    // coefficient history of the eigenvalue estimates: the longest run of this linearisation
    const long long coarse_it = ctx->sp.coarse_eig_iters > 0 ? std::min<long long>(ctx->coarse_nfree, ctx->sp.coarse_eig_iters)
                                                              : ctx->coarse_nfree;
    const long long need = 2 * std::max<long long>({ctx->nlev > 1 ? (long long)ctx->sp.eig_iters : 0,
                                                     ctx->sp.coarse_solver < 1 ? std::max<long long>(coarse_it, 1) : 0, 1});
    if ((long long)ctx->eig_hist_len < need) {
      dfree(ctx, ctx->d_eig_hist);
      ctx->d_eig_hist = nullptr;
      HY_TRY(dalloc(ctx, &ctx->d_eig_hist, (size_t)need));
      ctx->eig_hist_len = (size_t)need;
    }
  }
  const int top = ctx->nlev - 1;
  HY_CK(cudaMemcpyAsync(ctx->lev[top].d_u64, u, sizeof(double) * ctx->lev[top].ndofs, cudaMemcpyDeviceToDevice,
                        ctx->stream));
  for (int l = top; l >= 1; --l) HY_TRY(interpolate_down(ctx, l));
  pt.mark("carry down");
  // Setup reuse (setup_reuse > 0): keep the last full setup's eigenvalue estimates and coarse inverse while
  // the coarsest level's displacement stays within the tolerance of the one they were computed for.
  bool reuse = false;
  if (ctx->sp.setup_reuse > 0.0 && ctx->setup_valid) {
    Level& C = ctx->lev[0];
    launch_sub<double>(C.d_u64, ctx->d_usetup, ctx->d_udiff, C.ndofs, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
    double dd = 0.0, uu = 0.0;
    HY_TRY(dot<double>(ctx, ctx->d_udiff, ctx->d_udiff, C.ndofs, &dd));
    HY_TRY(dot<double>(ctx, C.d_u64, C.d_u64, C.ndofs, &uu));
    reuse = std::sqrt(dd) <= ctx->sp.setup_reuse * std::sqrt(uu);
  }
  ctx->setup_valid = false;
  ctx->last_setup_reused = reuse;
  ctx->side_timed = false;
  hy_status coarse_st = HY_OK;
  if (ctx->sp.coarse_solver >= 1 && !reuse) coarse_st = coarse_direct_setup(ctx);  // runs on the side stream
  if (coarse_st != HY_OK) return coarse_st;
  HY_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
  const unsigned long long one_bits = 0x7FF0000000000000ULL;  // +inf
  HY_CK(cudaMemcpyAsync(ctx->d_jmin, &one_bits, sizeof(one_bits), cudaMemcpyHostToDevice, ctx->stream));
  for (int l = 0; l < ctx->nlev; ++l) {
    Level& L = ctx->lev[l];
    const bool need64 = (l == top) || (l == 0) || !mixed;
    const bool need32 = mixed && (l > 0 || l == top);
    L.has64 = L.has32 = L.hasff = L.lazy64 = false;
    L.form[0] = L.form[1] = L.form[2] = -1;
    // the finest level's FP64 and double-float caches serve the outer CG: the given variant; the V-cycle's
    // level operators (every cache below the finest, and its FP32 cache) take the level variant
    const int lvar = build_of(ctx->sp.level_variant >= 0 ? ctx->sp.level_variant : var);
    L.var[0] = l == top ? build_of(var) : lvar;
    L.var[1] = lvar;
    L.var[2] = var;
    if (need64 && l == top && l > 0 && ctx->sp.fine_dtype == HY_FF) {
      HY_TRY(build_cache<double>(ctx, l, L.var[0], true));
      L.lazy64 = true;
    } else if (need64) {
      HY_TRY(build_cache<double>(ctx, l, L.var[0]));
      L.has64 = true;
    }
    if (l == top && ctx->sp.fine_dtype == HY_FF) {
      HY_TRY(build_cache<ff>(ctx, l, L.var[2]));
      L.hasff = true;
    }
    if (need32) {
      // The finest level's FP32 cache comes from its double-float or FP64 cache of the same state where the
      // variants allow (the same variant, or T2 from T4): one state evaluation instead of two.
      const bool from_ff = L.hasff, from64 = !from_ff && L.has64;
      const int vs = from_ff ? L.var[2] : L.var[0], vd = L.var[1];
      const bool t4_to_t2 = vs == VAR_T4 && vd == VAR_T2;
      // (A variant that caches nothing needs no FP32 build at all: the other build has checked J.)
      if (l == top && (from_ff || from64) && (vs == vd || t4_to_t2)) {
        HY_TRY(build_cache<float>(ctx, l, vd, true));
        if (cache_values(vd, ctx->dim) > 0) {
          launch_derive_f32(ctx->dim, ctx->n, from_ff,
                            from_ff ? (const void*)cache_of<ff>(L) : (const void*)cache_of<double>(L),
                            cache_values(vs, ctx->dim), cache_buf<float>(L), cache_values(vd, ctx->dim), t4_to_t2,
                            L.g.ncells, ctx->stream);
          HY_TRY(check_launch(ctx, 1));
        }
      } else {
        HY_TRY(build_cache<float>(ctx, l, L.var[1]));
      }
      if (!L.d_u32) HY_TRY(dalloc(ctx, &L.d_u32, L.ndofs));
      launch_convert<double, float>(L.d_u64, L.d_u32, L.ndofs, ctx->stream);
      HY_TRY(check_launch(ctx, 1));
      L.has32 = true;
    }
    // diagonal (FP64), inverse in the level precisions
    HY_CK(cudaMemsetAsync(L.d_diag, 0, sizeof(double) * L.ndofs, ctx->stream));
    CellArgs<double> a = cell_args<double>(ctx, L);
    a.u64 = L.d_u64;
    a.y = L.d_diag;
    // the state from the level's T4/T2 cache in the diagonal's arithmetic where there is one, else evaluated
    const bool ffa = ctx->sp.fine_dtype == HY_FF;
    const int cvar = ffa ? L.var[2] : L.var[0];
    const bool cached = (ffa ? L.hasff : L.has64) && (cvar == VAR_T4 || cvar == VAR_T2);
    CellFn<double> dfn = diag_fn(ctx->dim, ctx->n, ffa);
    if (cached) {
      a.cache = ffa ? reinterpret_cast<const double*>(cache_of<ff>(L)) : cache_of<double>(L);
      dfn = diag_cached_fn(ctx->dim, ctx->n, ffa, cvar);
    }
    dfn(a, ctx->stream);
    launch_set_constrained_one<double>(L.d_diag, L.nnodes, ctx->dim, L.g, ctx->stream);
    HY_TRY(check_launch(ctx, 2));
    if (need64) {
      if (!L.d_dinv64) HY_TRY(dalloc(ctx, &L.d_dinv64, L.ndofs));
      launch_invert<double>(L.d_diag, L.d_dinv64, L.ndofs, ctx->stream);
      HY_TRY(ensure_level_vectors(ctx, l, false));
    }
    if (need32) {
      if (!L.d_dinv32) HY_TRY(dalloc(ctx, &L.d_dinv32, L.ndofs));
      launch_invert<float>(L.d_diag, L.d_dinv32, L.ndofs, ctx->stream);
      HY_TRY(ensure_level_vectors(ctx, l, true));
    }
    HY_TRY(check_launch(ctx, (int)need64 + (int)need32));
  }
  HY_TRY(check_error_word(ctx, "set_displacement"));
  pt.mark("state+diag");
  for (int l = 0; l < ctx->nlev; ++l) {
    if (ctx->lev[l].has64) HY_TRY(autotune_level<double>(ctx, l));
    if (ctx->lev[l].has32) HY_TRY(autotune_level<float>(ctx, l));
    if (ctx->lev[l].hasff) HY_TRY(autotune_level<ff>(ctx, l));
  }
  pt.mark("autotune");
  // eigenvalue estimates (level precision of the V-cycle)
  if (!reuse) HY_TRY(smoother_eig_estimates(ctx));
  pt.mark("smoother eig");
  if (reuse) {
    // the last full setup's coarse inverse or Chebyshev coarse bounds stay
  } else if (ctx->sp.coarse_solver >= 1) {
    HY_TRY(coarse_direct_finish(ctx));
  } else {
    const long long nfree = ctx->coarse_nfree;
    int it = ctx->sp.coarse_eig_iters > 0 ? (int)std::min<long long>(nfree, ctx->sp.coarse_eig_iters) : (int)nfree;
    if (it < 1) it = 1;
    double lmin, lmax;
    HY_TRY(eig_estimate<double>(ctx, 0, it, lmin, lmax));
    ctx->coarse_lo = lmin;
    ctx->coarse_hi = ctx->sp.cheb_hi * lmax;
  }
  // The Chebyshev coarse solver needs an SPD coarsest level; an indefinite one (a tangent about an
  // unstable state) is reported when the V-cycle is used, not here, so that applications still work.
  if (ctx->sp.coarse_solver < 1 && !reuse) {
    ctx->coarse_spd = ctx->coarse_lo > 0.0;
    ctx->coarse_deg = 0;
    if (ctx->coarse_spd) {
      const double sig = (ctx->coarse_hi + ctx->coarse_lo) / (ctx->coarse_hi - ctx->coarse_lo);
      ctx->coarse_deg = std::max(1, (int)std::ceil(std::acosh(1.0 / ctx->sp.coarse_reduction) / std::acosh(sig) - 1e-12));
    }
  }
  pt.mark("coarse setup");
  if (ctx->verbose) {
    for (int l = 1; l < ctx->nlev; ++l) std::fprintf(stderr, "[hy] level %d lmax %.6e\n", l, ctx->lev[l].lmax);
    std::fprintf(stderr, "[hy] coarse lo %.6e hi %.6e degree %d\n", ctx->coarse_lo, ctx->coarse_hi, ctx->coarse_deg);
  }
  if (!reuse) {  // this full setup is the reference of later reuse
    HY_CK(cudaMemcpyAsync(ctx->d_usetup, ctx->lev[0].d_u64, sizeof(double) * ctx->lev[0].ndofs,
                          cudaMemcpyDeviceToDevice, ctx->stream));
  }
  ctx->setup_valid = true;
  ctx->state_ok = true;
  return HY_OK;
}

// f = sum over faces of t_face * int_face N_a dA (dead tractions, host array [6][3]); true if any is nonzero.
hy_status face_load(hy_ctx* ctx, const double (*traction)[3], double* f, bool* any) {
  Level& L = ctx->lev[ctx->nlev - 1];
  HY_CK(cudaMemsetAsync(f, 0, sizeof(double) * L.ndofs, ctx->stream));
  FaceLoad fl{};
  fl.k = ctx->k;
  for (int a = 0; a < ctx->n; ++a) {
    double s = 0.0;
    for (int q = 0; q < ctx->n; ++q) s += ctx->b64.w[q] * ctx->b64.S[q][a];
    fl.w1[a] = s;
  }
  *any = false;
  for (int face = 0; face < 2 * ctx->dim; ++face) {
    bool nz = false;
    for (int c = 0; c < ctx->dim; ++c) {
      fl.t[c] = traction[face][c];
      nz = nz || traction[face][c] != 0.0;
    }
    if (!nz) continue;
    *any = true;
    launch_face_load(f, ctx->dim, L.g, face, fl, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
  }
  return HY_OK;
}

hy_status residual(hy_ctx* ctx, const double* u, double* r) {
  Level& L = ctx->lev[ctx->nlev - 1];
  HY_CK(cudaMemsetAsync(r, 0, sizeof(double) * L.ndofs, ctx->stream));
  CellArgs<double> a = cell_args<double>(ctx, L);
  a.u64 = u;
  a.y = r;
  residual_fn(ctx->dim, ctx->n)(a, ctx->stream);
  return check_launch(ctx, 1);
}

hy_status jacobian_ok(hy_ctx* ctx, const double* u, bool& ok) {
  Level& L = ctx->lev[ctx->nlev - 1];
  CellArgs<double> a = cell_args<double>(ctx, L);
  a.u64 = u;
  HY_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
  state_fn_f64(ctx->dim, ctx->n, VAR_NONE)(a, nullptr, ctx->stream);
  HY_TRY(check_launch(ctx, 1));
  unsigned h = 0;
  HY_CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  HY_CK(cudaStreamSynchronize(ctx->stream));
  HY_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
  ok = (h == 0);
  return HY_OK;
}

hy_status pcg_host(hy_ctx* ctx, const double* b, double* x, double rtol, int max_iter, int* its_out) {
  Level& L = ctx->lev[ctx->nlev - 1];
  const long long n = L.ndofs;
  double *r = ctx->f64[0], *z = ctx->f64[1], *p = ctx->f64[2], *q = ctx->f64[3];
  if (its_out) *its_out = 0;
  HY_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  HY_CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  double bb;
  HY_TRY(dot<double>(ctx, b, b, n, &bb));
  const double nb = std::sqrt(bb);
  if (nb == 0.0) return HY_OK;
  if (!(nb == nb)) return fail(ctx, HY_ERR_ARG, "pcg: right-hand side has NaN");
  HY_TRY(vcycle_top(ctx, r, z));
  HY_CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  double rz;
  HY_TRY(dot<double>(ctx, r, z, n, &rz));
  for (int it = 1; it <= max_iter; ++it) {
    HY_TRY(level_apply<double>(ctx, ctx->nlev - 1, p, q));
    double pq;
    HY_TRY(dot<double>(ctx, p, q, n, &pq));
    if (ctx->verbose) std::fprintf(stderr, "[hy] pcg it %d rz %.3e pAp %.3e\n", it, rz, pq);
    if (!(pq > 0.0)) return fail(ctx, HY_ERR_NOCONV, "pcg: p^T A p <= 0 (operator not SPD)");
    const double alpha = rz / pq;
    launch_axpby<double>(alpha, p, 1.0, x, n, ctx->stream);
    launch_axpby<double>(-alpha, q, 1.0, r, n, ctx->stream);
    HY_TRY(check_launch(ctx, 2));
    double rr;
    HY_TRY(dot<double>(ctx, r, r, n, &rr));
    if (its_out) *its_out = it;
    if (std::sqrt(rr) <= rtol * nb) return HY_OK;
    HY_TRY(vcycle_top(ctx, r, z));
    double rzn;
    HY_TRY(dot<double>(ctx, r, z, n, &rzn));
    launch_xpay<double>(z, rzn / rz, p, p, n, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
    rz = rzn;
  }
  return fail(ctx, HY_ERR_NOCONV, "pcg: iteration cap reached");
}

}  // namespace

// =============================================================================================
// Work-list batches: several problems of the same dim and degree applied (and solved) together. The
// finest-level tangent actions of all problems run as ONE launch over a list of per-problem arguments;
// the rest of a preconditioned CG iteration runs as one branch per problem of a CUDA graph, captured once
// per resident set (the problems not yet converged), so that one graph launch and one host
// synchronisation advance every resident problem by one iteration.
struct hy_batch {
  int device = 0;
  int dim = 0, n = 0;
  std::vector<hy_ctx*> ctx;
  cudaStream_t s0 = nullptr;              // the batch's own stream
  std::vector<cudaStream_t> branch;       // one per problem: graph branches
  std::vector<cudaEvent_t> ev;            // one per problem: joins
  cudaEvent_t ev_fork = nullptr, ev_done = nullptr, ev_upload = nullptr;
  void* d_list = nullptr;                 // per-problem kernel arguments (CellArgs<double> or <float>)
  int* d_start = nullptr;                 // first thread block of each problem, then the total
  double* d_scal = nullptr;               // PCG_SCALARS doubles per problem
  void* h_list = nullptr;                 // pinned staging of the uploads
  int* h_start = nullptr;
  double* h_scal_in = nullptr;            // pinned: initial scalars
  double* h_scal_out = nullptr;           // pinned: scalars read back after each iteration
  int form[3] = {-1, -1, -1};             // tuned kernel form of the list launch per precision
  std::vector<const void*> up_x, up_y;    // what the uploaded list describes
  int up_dt = -1, up_blocks = 0;
  long long up_max_nodes = 0;
  std::string err;
  long long launches = 0;
};

namespace {

hy_status bfail(hy_batch* b, hy_status s, const std::string& msg) {
  b->err = msg;
  return s;
}
#define HB_CK(call)                                                                                     \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return bfail(b, e_ == cudaErrorMemoryAllocation ? HY_ERR_OOM : HY_ERR_CUDA,   \
                                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

constexpr size_t BATCH_ARG_BYTES = sizeof(CellArgs<double>) > sizeof(CellArgs<float>) ? sizeof(CellArgs<double>)
                                                                                      : sizeof(CellArgs<float>);

ApplyListFn<double> list_fn(int dim, int n, int var, double*) {
  return dim == 2 ? apply_list_fn_f64_2d(n, var) : apply_list_fn_f64_3d(n, var);
}
ApplyListFn<float> list_fn(int dim, int n, int var, float*) {
  return dim == 2 ? apply_list_fn_f32_2d(n, var) : apply_list_fn_f32_3d(n, var);
}
ApplyListFn<ff> list_fn(int dim, int n, int var, ff*) {
  return dim == 2 ? apply_list_fn_ff_2d(n, var) : apply_list_fn_ff_3d(n, var);
}

// Upload the argument list of the finest-level actions y_j = A_j x_j of the problems idx (skipped when
// the device copy already describes exactly these vectors).
template <typename T>
hy_status upload_list(hy_batch* b, const std::vector<int>& idx, const std::vector<const void*>& x,
                      const std::vector<const void*>& y) {
  const int dt = prec_index<T>();
  if (b->up_dt == dt && b->up_x == x && b->up_y == y) return HY_OK;
  HB_CK(cudaEventSynchronize(b->ev_upload));  // the staging buffer is free again
  CellArgs<T>* h = static_cast<CellArgs<T>*>(b->h_list);
  const int cb = apply_cells_per_block<T>(b->dim, b->n);
  long long blocks = 0, max_nodes = 0;
  for (size_t j = 0; j < idx.size(); ++j) {
    hy_ctx* c = b->ctx[idx[j]];
    Level& L = c->lev[c->nlev - 1];
    max_nodes = std::max(max_nodes, L.nnodes);
    CellArgs<T> a = cell_args<T>(c, L);
    a.x = static_cast<const vec_t<T>*>(x[j]);
    a.y = static_cast<vec_t<T>*>(const_cast<void*>(y[j]));
    a.cache = cache_of<T>(L);
    a.ubar = ubar_of<T>(L);
    a.pf = c->prefetch;
    h[j] = a;
    b->h_start[j] = (int)blocks;
    blocks += (L.g.ncells + cb - 1) / cb;
  }
  if (blocks > 0x7fffffffLL) return bfail(b, HY_ERR_ARG, "batch: too many thread blocks for one launch");
  b->h_start[idx.size()] = (int)blocks;
  HB_CK(cudaMemcpyAsync(b->d_list, h, sizeof(CellArgs<T>) * idx.size(), cudaMemcpyHostToDevice, b->s0));
  HB_CK(cudaMemcpyAsync(b->d_start, b->h_start, sizeof(int) * (idx.size() + 1), cudaMemcpyHostToDevice, b->s0));
  HB_CK(cudaEventRecord(b->ev_upload, b->s0));
  b->up_x = x;
  b->up_y = y;
  b->up_dt = dt;
  b->up_blocks = (int)blocks;
  b->up_max_nodes = max_nodes;
  return HY_OK;
}

// prep_out of every listed problem (one launch) followed by the list launch, on stream st; x and y are
// the vectors the uploaded list describes.
template <typename T>
hy_status list_apply(hy_batch* b, const std::vector<int>& idx, const std::vector<const void*>& x,
                     const std::vector<const void*>& y, int form, cudaStream_t st) {
  hy_ctx* c0 = b->ctx[idx[0]];
  const int var = c0->lev[c0->nlev - 1].var[prec_index<T>()];
  ApplyListFn<T> fn = list_fn(b->dim, b->n, var, (T*)nullptr);
  if (!fn) return bfail(b, HY_ERR_UNSUPPORTED, "batch: no kernel for this dim/degree/variant");
  (void)x;
  (void)y;
  launch_prep_out_list<T>(static_cast<const CellArgs<T>*>(b->d_list), (int)idx.size(), b->dim, b->up_max_nodes, st);
  fn(static_cast<const CellArgs<T>*>(b->d_list), b->d_start, (int)idx.size(), b->up_blocks, form, st);
  b->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, HY_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return HY_OK;
}

// Pick the faster kernel form for the list launch of this batch and precision (timed on the real list:
// one warm-up each, then three alternating rounds of four launches, the best round of each decides).
template <typename T>
hy_status tune_list(hy_batch* b, const std::vector<int>& idx, const std::vector<const void*>& x,
                    const std::vector<const void*>& y) {
  const int dt = prec_index<T>();
  if (b->form[dt] >= 0) return HY_OK;
  const int forced = b->ctx[idx[0]]->sp.kernel_form;
  if (forced >= 0) {
    b->form[dt] = forced;
    return HY_OK;
  }
  cudaEvent_t e0, e1;
  HB_CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfail(b, HY_ERR_CUDA, "cudaEventCreate");
  }
  float best[2] = {1e30f, 1e30f};
  hy_status st = HY_OK;
  for (int f = 0; f < 2 && st == HY_OK; ++f) st = list_apply<T>(b, idx, x, y, f, b->s0);
  for (int r = 0; r < 3 && st == HY_OK; ++r)
    for (int f = 0; f < 2 && st == HY_OK; ++f) {
      cudaEventRecord(e0, b->s0);
      for (int q = 0; q < 4 && st == HY_OK; ++q) st = list_apply<T>(b, idx, x, y, f, b->s0);
      cudaEventRecord(e1, b->s0);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best[f] = std::min(best[f], 0.25f * ms);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != HY_OK) return st;
  b->form[dt] = best[1] < best[0] ? FORM_LINE : FORM_POINT;
  if (b->ctx[idx[0]]->verbose)
    std::fprintf(stderr, "[hy] batch of %zu: list launch %s point %.3f ms, line %.3f ms\n", idx.size(),
                 kPrecNames[dt], best[0], best[1]);
  return HY_OK;
}

// s0 waits for the work already queued on every context's stream.
hy_status join_in(hy_batch* b) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    HB_CK(cudaEventRecord(b->ev[i], b->ctx[i]->stream));
    HB_CK(cudaStreamWaitEvent(b->s0, b->ev[i], 0));
  }
  return HY_OK;
}
// every context's stream waits for the batch's work.
hy_status join_out(hy_batch* b) {
  HB_CK(cudaEventRecord(b->ev_done, b->s0));
  for (hy_ctx* c : b->ctx) HB_CK(cudaStreamWaitEvent(c->stream, b->ev_done, 0));
  return HY_OK;
}

// The V-cycle of vcycle_top issued kernel by kernel on ctx->stream (for capture inside a batch graph).
hy_status vcycle_top_ops(hy_ctx* ctx, const double* r, double* z) {
  const int top = ctx->nlev - 1;
  Level& L = ctx->lev[top];
  if (level_f32(ctx, top)) {
    launch_convert<double, float>(r, L.w32[0], L.ndofs, ctx->stream);
    HY_TRY(check_launch(ctx, 1));
    HY_TRY(vcycle_level(ctx, top));
    launch_convert<float, double>(L.w32[1], z, L.ndofs, ctx->stream);
    return check_launch(ctx, 1);
  }
  HY_CK(cudaMemcpyAsync(L.w64[0], r, sizeof(double) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
  HY_TRY(vcycle_level(ctx, top));
  HY_CK(cudaMemcpyAsync(z, L.w64[1], sizeof(double) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
  return HY_OK;
}

// One PCG iteration of one problem after q = A p: alpha = rz/pq; x += alpha p; r -= alpha q;
// converged = |r| <= tol; z = V r; beta = rzn/rz; p = z + beta p (scalars sc on the device).
// first half (after q = A p): alpha, x += alpha p, r -= alpha q, |r|^2 and the convergence test
hy_status pcg_update(hy_ctx* c, double* sc, double* x) {
  const long long nd = c->lev[c->nlev - 1].ndofs;
  double *r = c->f64[0], *p = c->f64[2], *q = c->f64[3];
  cudaStream_t st = c->stream;
  launch_dot<double>(p, q, nd, c->d_partials, sc + 1, st);
  launch_pcg_scalar(sc, 0, st);
  launch_axpy_dev<double>(sc + 2, 1.0, p, x, nd, st);
  launch_axpy_dev<double>(sc + 2, -1.0, q, r, nd, st);
  launch_dot<double>(r, r, nd, c->d_partials, sc + 3, st);
  launch_pcg_scalar(sc, 1, st);
  return check_launch(c, 8);
}
// second half: z = V r, beta, p = z + beta p
hy_status pcg_direction(hy_ctx* c, double* sc) {
  const long long nd = c->lev[c->nlev - 1].ndofs;
  double *r = c->f64[0], *z = c->f64[1], *p = c->f64[2];
  cudaStream_t st = c->stream;
  HY_TRY(vcycle_top_ops(c, r, z));
  launch_dot<double>(r, z, nd, c->d_partials, sc + 4, st);
  launch_pcg_scalar(sc, 2, st);
  launch_xpay_dev<double>(z, sc + 5, p, p, nd, st);
  return check_launch(c, 4);
}
hy_status pcg_branch(hy_ctx* c, double* sc, double* x) {
  HY_TRY(pcg_update(c, sc, x));
  return pcg_direction(c, sc);
}

// One PCG iteration of every resident problem R, captured into a graph on s0: the list launch
// q_i = A_i p_i, then one branch per problem (pcg_branch), then a copy of all scalars to pinned host
// memory. *kernels = kernels one replay launches.
template <typename TL>
hy_status capture_iteration(hy_batch* b, const std::vector<int>& R, double* const* xsol, int form,
                            cudaGraphExec_t* exec, long long* kernels) {
  std::vector<const void*> ps, qs;
  for (int i : R) {
    ps.push_back(b->ctx[i]->f64[2]);
    qs.push_back(b->ctx[i]->f64[3]);
  }
  HY_TRY(upload_list<TL>(b, R, ps, qs));
  std::vector<cudaStream_t> saved(R.size());
  std::vector<long long> l0(R.size());
  for (size_t j = 0; j < R.size(); ++j) {
    saved[j] = b->ctx[R[j]]->stream;
    l0[j] = b->ctx[R[j]]->launches;
  }
  const long long b0 = b->launches;
  HB_CK(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal));
  hy_status st = list_apply<TL>(b, R, ps, qs, form, b->s0);
  if (st == HY_OK && cudaEventRecord(b->ev_fork, b->s0) != cudaSuccess) st = bfail(b, HY_ERR_CUDA, "cudaEventRecord");
  for (size_t j = 0; j < R.size() && st == HY_OK; ++j) {
    const int i = R[j];
    hy_ctx* c = b->ctx[i];
    cudaStream_t bs = b->branch[i];
    if (cudaStreamWaitEvent(bs, b->ev_fork, 0) != cudaSuccess) {
      st = bfail(b, HY_ERR_CUDA, "cudaStreamWaitEvent");
      break;
    }
    c->stream = bs;
    st = pcg_branch(c, b->d_scal + (size_t)i * PCG_SCALARS, xsol[i]);
    c->stream = saved[j];
    if (st != HY_OK) {
      b->err = c->err;
      break;
    }
    if (cudaEventRecord(b->ev[i], bs) != cudaSuccess || cudaStreamWaitEvent(b->s0, b->ev[i], 0) != cudaSuccess)
      st = bfail(b, HY_ERR_CUDA, "branch join");
  }
  if (st == HY_OK &&
      cudaMemcpyAsync(b->h_scal_out, b->d_scal, sizeof(double) * PCG_SCALARS * b->ctx.size(), cudaMemcpyDeviceToHost,
                      b->s0) != cudaSuccess)
    st = bfail(b, HY_ERR_CUDA, "cudaMemcpyAsync of the scalars");
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->s0, &g);
  long long nk = b->launches - b0;
  for (size_t j = 0; j < R.size(); ++j) {
    hy_ctx* c = b->ctx[R[j]];
    c->stream = saved[j];
    nk += c->launches - l0[j];
    c->launches = l0[j];
  }
  b->launches = b0;
  if (st != HY_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != HY_OK) return st;
    return bfail(b, HY_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, HY_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  *kernels = nk;
  return HY_OK;
}

hy_status batch_check(hy_batch* b) {
  for (hy_ctx* c : b->ctx) {
    if (c->nlev == 0 || c->dim != b->dim || c->n != b->n)
      return bfail(b, HY_ERR_STATE, "batch: a context's mesh changed since the batch was created");
    if (!c->state_ok) return bfail(b, HY_ERR_STATE, "batch: set_displacement on every context first");
    const Level& L = c->lev[c->nlev - 1];
    const Level& L0 = b->ctx[0]->lev[b->ctx[0]->nlev - 1];
    if (L.var[0] != L0.var[0] || L.var[1] != L0.var[1] || L.var[2] != L0.var[2])
      return bfail(b, HY_ERR_ARG, "batch: the contexts must use the same variants");
  }
  return HY_OK;
}

template <typename T>
hy_status batch_apply(hy_batch* b, const void* const* x, void* const* y) {
  const int cnt = (int)b->ctx.size();
  std::vector<int> R(cnt);
  std::vector<const void*> xs(cnt), ys(cnt);
  for (int i = 0; i < cnt; ++i) {
    hy_ctx* c = b->ctx[i];
    const Level& L = c->lev[c->nlev - 1];
    if constexpr (std::is_same<T, double>::value) {
      if (L.lazy64 && ensure_fp64_cache(c, c->nlev - 1) != HY_OK) return bfail(b, HY_ERR_STATE, "batch: " + c->err);
    }
    if (!has_cache<T>(L)) return bfail(b, HY_ERR_STATE, "batch: a context has no finest-level cache of this precision");
    if (!x[i] || !y[i] || x[i] == y[i]) return bfail(b, HY_ERR_ARG, "batch: null or aliased vectors");
    R[i] = i;
    xs[i] = x[i];
    ys[i] = y[i];
  }
  HY_TRY(join_in(b));
  HY_TRY(upload_list<T>(b, R, xs, ys));
  HY_TRY(tune_list<T>(b, R, xs, ys));
  HY_TRY(list_apply<T>(b, R, xs, ys, b->form[prec_index<T>()], b->s0));
  return join_out(b);
}

hy_status batch_pcg(hy_batch* b, const double* const* rhs, double* const* xs, double rtol, int max_iter, int* its,
                    hy_status* sts) {
  const int cnt = (int)b->ctx.size();
  std::vector<int> R;
  for (int i = 0; i < cnt; ++i) {
    its[i] = 0;
    sts[i] = HY_OK;
    if (!rhs[i] || !xs[i]) return bfail(b, HY_ERR_ARG, "batch: null vectors");
  }
  for (int i = 0; i < cnt; ++i) {
    hy_ctx* c = b->ctx[i];
    if (!c->coarse_spd) {
      sts[i] = fail(c, HY_ERR_NOCONV, "coarsest-level tangent is not positive definite");
      continue;
    }
    const long long nd = c->lev[c->nlev - 1].ndofs;
    double *r = c->f64[0], *z = c->f64[1], *p = c->f64[2];
    hy_status st = HY_OK;
    double bb = 0.0;
    if (cudaMemsetAsync(xs[i], 0, sizeof(double) * nd, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(r, rhs[i], sizeof(double) * nd, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      st = fail(c, HY_ERR_CUDA, "batch pcg: initial copies");
    if (st == HY_OK) st = dot<double>(c, rhs[i], rhs[i], nd, &bb);
    const double nb = std::sqrt(bb);
    if (st == HY_OK && nb == 0.0) continue;
    if (st == HY_OK && !(nb == nb)) st = fail(c, HY_ERR_ARG, "pcg: right-hand side has NaN");
    if (st == HY_OK) st = vcycle_top(c, r, z);
    if (st == HY_OK && cudaMemcpyAsync(p, z, sizeof(double) * nd, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      st = fail(c, HY_ERR_CUDA, "batch pcg: copy");
    if (st == HY_OK) {
      double* hs = b->h_scal_in + (size_t)i * PCG_SCALARS;
      for (int k = 0; k < PCG_SCALARS; ++k) hs[k] = 0.0;
      hs[6] = rtol * nb;
      if (cudaMemcpyAsync(b->d_scal + (size_t)i * PCG_SCALARS, hs, sizeof(double) * PCG_SCALARS,
                          cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        st = fail(c, HY_ERR_CUDA, "batch pcg: scalars");
    }
    if (st == HY_OK) {
      launch_dot<double>(r, z, nd, c->d_partials, b->d_scal + (size_t)i * PCG_SCALARS, c->stream);
      st = check_launch(c, 2);
    }
    if (st != HY_OK) {
      sts[i] = st;
      continue;
    }
    R.push_back(i);
  }
  // the finest-level action of the outer CG: double-float when every problem asks for it (fine_dtype)
  bool use_ff = true;
  for (hy_ctx* c : b->ctx) use_ff = use_ff && c->sp.fine_dtype == HY_FF && c->lev[c->nlev - 1].hasff;
  if (!use_ff)
    for (int i : R)
      if (ensure_fp64_cache(b->ctx[i], b->ctx[i]->nlev - 1) != HY_OK) return bfail(b, HY_ERR_STATE, "batch: " + b->ctx[i]->err);
  HY_TRY(join_in(b));
  hy_status result = HY_OK;
  if (!R.empty()) {
    std::vector<const void*> ps, qs;
    for (int i : R) {
      ps.push_back(b->ctx[i]->f64[2]);
      qs.push_back(b->ctx[i]->f64[3]);
    }
    if (use_ff) {
      result = upload_list<ff>(b, R, ps, qs);
      if (result == HY_OK) result = tune_list<ff>(b, R, ps, qs);
    } else {
      result = upload_list<double>(b, R, ps, qs);
      if (result == HY_OK) result = tune_list<double>(b, R, ps, qs);
    }
  }
  // R: problems in the current graph; live: those still iterating. A finished problem stays in the graph
  // as a no-op (alpha = beta = 0 on the device) until a quarter of the graph's problems have finished,
  // then the graph is captured again for the live ones.
  cudaGraphExec_t exec = nullptr;
  long long nk = 0;
  bool rebuild = true;
  std::vector<char> live(cnt, 0);
  for (int i : R) live[i] = 1;
  size_t n_live = R.size();
  double t_capture = 0.0, t_replay = 0.0;
  int n_capture = 0, n_replay = 0;
  while (result == HY_OK && n_live > 0) {
    if (rebuild) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      std::vector<int> keep;
      for (int i : R)
        if (live[i]) keep.push_back(i);
      R.swap(keep);
      const auto t0 = std::chrono::steady_clock::now();
      result = use_ff ? capture_iteration<ff>(b, R, xs, b->form[2], &exec, &nk)
                      : capture_iteration<double>(b, R, xs, b->form[0], &exec, &nk);
      t_capture += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      ++n_capture;
      if (result != HY_OK) break;
      rebuild = false;
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGraphLaunch(exec, b->s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s0);
    t_replay += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ++n_replay;
    if (e != cudaSuccess) {
      result = bfail(b, HY_ERR_CUDA, std::string("batch pcg iteration: ") + cudaGetErrorString(e));
      break;
    }
    b->launches += nk;
    size_t finished_in_graph = 0;
    for (int i : R) {
      if (!live[i]) {
        ++finished_in_graph;
        continue;
      }
      const double* h = b->h_scal_out + (size_t)i * PCG_SCALARS;
      bool done = true;
      if (h[8] != 0.0) {
        sts[i] = fail(b->ctx[i], HY_ERR_NOCONV, "pcg: p^T A p <= 0 (operator not SPD)");
      } else {
        ++its[i];
        if (h[7] == 0.0) {
          if (its[i] >= max_iter) {
            sts[i] = fail(b->ctx[i], HY_ERR_NOCONV, "pcg: iteration cap reached");
            // mark it finished on the device too, so that replays before the next capture leave it alone
            double* one = b->h_scal_in + (size_t)i * PCG_SCALARS + 7;
            *one = 1.0;
            if (cudaMemcpyAsync(b->d_scal + (size_t)i * PCG_SCALARS + 7, one, sizeof(double), cudaMemcpyHostToDevice,
                                b->s0) != cudaSuccess)
              result = bfail(b, HY_ERR_CUDA, "batch pcg: finish flag");
          } else {
            done = false;
          }
        }
      }
      if (done) {
        live[i] = 0;
        --n_live;
        ++finished_in_graph;
      }
    }
    if (n_live > 0 && 4 * finished_in_graph >= R.size()) rebuild = true;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (b->ctx[0]->verbose)
    std::fprintf(stderr, "[hy] batch pcg of %d: %d captures %.2f ms, %d replays %.2f ms\n", cnt, n_capture, t_capture,
                 n_replay, t_replay);
  const hy_status jo = join_out(b);
  if (result == HY_OK && jo == HY_OK)
    for (int i = 0; i < cnt; ++i)
      if (sts[i] == HY_OK) sts[i] = check_error_word(b->ctx[i], "batch pcg");
  return result != HY_OK ? result : jo;
}

// Capture what `body` issues on ctx->stream into an executable graph (private capture stream); kernel
// counts recorded during the capture go to *nodes instead of the context's counter.
template <typename F>
hy_status capture_exec(hy_ctx* ctx, F&& body, cudaGraphExec_t* exec, long long* nodes) {
  if (!ctx->cap_stream) HY_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->stream;
  const long long l0 = ctx->launches;
  ctx->stream = ctx->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    ctx->stream = saved;
    return fail(ctx, HY_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  const hy_status st = body();
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ctx->cap_stream, &g);
  ctx->stream = saved;
  *nodes = ctx->launches - l0;
  ctx->launches = l0;
  if (st != HY_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != HY_OK) return st;
    return fail(ctx, HY_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, HY_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return HY_OK;
}

// PCG of one problem with every CG scalar on the device. An iteration is two graphs, captured once per
// linearisation: A = {q = A p; alpha; x += alpha p; r -= alpha q; |r|^2; convergence test; scalars to pinned
// host memory} and B = {z = V r; beta; p = z + beta p}. The host waits once per iteration, after A, and
// launches B only if the problem has not converged; the iterate lives in a work vector and is copied out.
// Same arithmetic as pcg_host (the scalars are formed on the device instead of the host).
hy_status pcg_graph(hy_ctx* ctx, const double* b, double* x_out, double rtol, int max_iter, int* its_out) {
  const int top = ctx->nlev - 1;
  const long long n = ctx->lev[top].ndofs;
  double *r = ctx->f64[0], *z = ctx->f64[1], *p = ctx->f64[2], *q = ctx->f64[3], *x = ctx->f64[10];
  double* sc = ctx->d_eig_scal + 8;
  if (its_out) *its_out = 0;
  if (!ctx->h_pcg_scal) HY_CK(cudaMallocHost((void**)&ctx->h_pcg_scal, 2 * sizeof(double) * PCG_SCALARS));
  double* h_in = ctx->h_pcg_scal;
  double* h_out = ctx->h_pcg_scal + PCG_SCALARS;
  HY_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  HY_CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  double bb;
  HY_TRY(dot<double>(ctx, b, b, n, &bb));  // synchronises: h_in is free again
  const double nb = std::sqrt(bb);
  auto copy_out = [&]() { return cudaMemcpyAsync(x_out, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream); };
  if (nb == 0.0) {
    HY_CK(copy_out());
    return HY_OK;
  }
  if (!(nb == nb)) return fail(ctx, HY_ERR_ARG, "pcg: right-hand side has NaN");
  HY_TRY(vcycle_top(ctx, r, z));
  HY_CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  for (int k = 0; k < PCG_SCALARS; ++k) h_in[k] = 0.0;
  h_in[6] = rtol * nb;
  HY_CK(cudaMemcpyAsync(sc, h_in, sizeof(double) * PCG_SCALARS, cudaMemcpyHostToDevice, ctx->stream));
  launch_dot<double>(r, z, n, ctx->d_partials, sc, ctx->stream);  // rz
  HY_TRY(check_launch(ctx, 2));
  if (!ctx->pcg_exec[0]) {
    HY_TRY(capture_exec(ctx, [&]() -> hy_status {
      HY_TRY(level_apply<double>(ctx, top, p, q));
      HY_TRY(pcg_update(ctx, sc, x));
      HY_CK(cudaMemcpyAsync(h_out, sc, sizeof(double) * PCG_SCALARS, cudaMemcpyDeviceToHost, ctx->stream));
      return HY_OK;
    }, &ctx->pcg_exec[0], &ctx->pcg_nodes[0]));
    HY_TRY(capture_exec(ctx, [&]() -> hy_status { return pcg_direction(ctx, sc); }, &ctx->pcg_exec[1],
                        &ctx->pcg_nodes[1]));
  }
  for (int it = 1; it <= max_iter; ++it) {
    HY_CK(cudaGraphLaunch(ctx->pcg_exec[0], ctx->stream));
    HY_CK(cudaStreamSynchronize(ctx->stream));
    ctx->launches += ctx->pcg_nodes[0];
    if (h_out[8] != 0.0) {
      HY_CK(copy_out());
      return fail(ctx, HY_ERR_NOCONV, "pcg: p^T A p <= 0 (operator not SPD)");
    }
    if (its_out) *its_out = it;
    if (h_out[7] != 0.0) {
      HY_CK(copy_out());
      return HY_OK;
    }
    HY_CK(cudaGraphLaunch(ctx->pcg_exec[1], ctx->stream));
    ctx->launches += ctx->pcg_nodes[1];
  }
  HY_CK(copy_out());
  return fail(ctx, HY_ERR_NOCONV, "pcg: iteration cap reached");
}

hy_status pcg(hy_ctx* ctx, const double* b, double* x, double rtol, int max_iter, int* its_out) {
  const Range range("pcg");
  return ctx->use_graphs ? pcg_graph(ctx, b, x, rtol, max_iter, its_out) : pcg_host(ctx, b, x, rtol, max_iter, its_out);
}

void batch_free(hy_batch* b) {
  if (b->s0) cudaStreamSynchronize(b->s0);
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->ev_fork, b->ev_done, b->ev_upload})
    if (e) cudaEventDestroy(e);
  if (b->d_list) cudaFree(b->d_list);
  if (b->d_start) cudaFree(b->d_start);
  if (b->d_scal) cudaFree(b->d_scal);
  if (b->h_list) cudaFreeHost(b->h_list);
  if (b->h_start) cudaFreeHost(b->h_start);
  if (b->h_scal_in) cudaFreeHost(b->h_scal_in);
  if (b->h_scal_out) cudaFreeHost(b->h_scal_out);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
}

}  // namespace

// =============================================================================================
extern "C" {

const char* hy_status_str(hy_status s) {
  switch (s) {
    case HY_OK: return "HY_OK";
    case HY_ERR_ARG: return "HY_ERR_ARG";
    case HY_ERR_STATE: return "HY_ERR_STATE";
    case HY_ERR_OOM: return "HY_ERR_OOM";
    case HY_ERR_CUDA: return "HY_ERR_CUDA";
    case HY_ERR_JNEG: return "HY_ERR_JNEG";
    case HY_ERR_NOCONV: return "HY_ERR_NOCONV";
    case HY_ERR_TIMEOUT: return "HY_ERR_TIMEOUT";
    case HY_ERR_UNSUPPORTED: return "HY_ERR_UNSUPPORTED";
  }
  return "HY_ERR_UNKNOWN";
}

const char* hy_last_error(const hy_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hy_status hy_create(hy_ctx** out, int device, void* stream) {
  if (!out) return HY_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HY_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return HY_ERR_CUDA;
  hy_ctx* ctx = new (std::nothrow) hy_ctx();
  if (!ctx) return HY_ERR_OOM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  const char* v = std::getenv("HY_VERBOSE");
  ctx->verbose = v && v[0] == '1';
  if (const char* pf = std::getenv("HY_PREFETCH")) ctx->prefetch = std::max(0, std::atoi(pf));
  const char* gr = std::getenv("HY_GRAPHS");
  ctx->use_graphs = !(gr && gr[0] == '0');
  *out = ctx;
  return HY_OK;
}

void hy_destroy(hy_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  free_mesh(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_side_fork) cudaEventDestroy(ctx->ev_side_fork);
  if (ctx->ev_side_join) cudaEventDestroy(ctx->ev_side_join);
  if (ctx->ev_side_start) cudaEventDestroy(ctx->ev_side_start);
  for (cudaStream_t st : ctx->eig_st)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : ctx->eig_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_eig_fork) cudaEventDestroy(ctx->ev_eig_fork);
  for (cudaEvent_t e : ctx->ev_phase)
    if (e) cudaEventDestroy(e);
  if (ctx->h_pcg_scal) cudaFreeHost(ctx->h_pcg_scal);
  if (ctx->h_err_side) cudaFreeHost(ctx->h_err_side);
  delete ctx;
}

hy_status hy_mesh_setup(hy_ctx* ctx, int dim, int degree, int m, int n_levels, const uint32_t* face_masks) {
  if (!ctx) return HY_ERR_ARG;
  if (dim != 2 && dim != 3) return fail(ctx, HY_ERR_ARG, "dim must be 2 or 3");
  if (degree < 1) return fail(ctx, HY_ERR_ARG, "degree must be >= 1");
  if (degree > 4) return fail(ctx, HY_ERR_UNSUPPORTED, "degree > 4 is not built");
  if (m < 1 || n_levels < 1 || !face_masks) return fail(ctx, HY_ERR_ARG, "bad mesh size or masks");
  {
    int mm = m;
    for (int l = 1; l < n_levels; ++l) {
      if (mm % 2) return fail(ctx, HY_ERR_ARG, "cells per direction must stay even while coarsening");
      mm /= 2;
    }
  }
  for (int f = 0; f < 2 * dim; ++f)
    if (face_masks[f] >> dim) return fail(ctx, HY_ERR_ARG, "face mask has bits beyond dim");
  const double Ldof = std::pow((double)degree * m + 1.0, dim) * dim;
  if (Ldof > 2.0e9) return fail(ctx, HY_ERR_ARG, "mesh too large");
  HY_CK(cudaSetDevice(ctx->device));
  if (ctx->stream) HY_CK(cudaStreamSynchronize(ctx->stream));
  free_mesh(ctx);
  ctx->dim = dim;
  ctx->k = degree;
  ctx->n = degree + 1;
  ctx->nlev = n_levels;
  for (int f = 0; f < 6; ++f) ctx->fm[f] = f < 2 * dim ? face_masks[f] : 0;
  // 1D tables
  {
    const int k = degree, n = degree + 1;
    std::vector<double> wg;
    const std::vector<double> xg = gauss_points(n, wg);
    const std::vector<double> gl = gll_points(k);
    Basis1D<double>& b = ctx->b64;
    std::memset(&b, 0, sizeof(b));
    for (int q = 0; q < n; ++q) {
      b.w[q] = wg[q];
      for (int a = 0; a < n; ++a) {
        b.S[q][a] = lagr(gl, a, xg[q]);
        b.Sd[q][a] = dlagr(gl, a, xg[q]);
        b.D[q][a] = dlagr(xg, a, xg[q]);
      }
    }
    for (int i = 0; i < MAXN; ++i) {
      ctx->b32.w[i] = (float)b.w[i];
      ctx->bff.w[i] = ff(b.w[i]);
      for (int j = 0; j < MAXN; ++j) {
        ctx->b32.S[i][j] = (float)b.S[i][j];
        ctx->b32.D[i][j] = (float)b.D[i][j];
        ctx->b32.Sd[i][j] = (float)b.Sd[i][j];
        ctx->bff.S[i][j] = ff(b.S[i][j]);
        ctx->bff.D[i][j] = ff(b.D[i][j]);
        ctx->bff.Sd[i][j] = ff(b.Sd[i][j]);
      }
    }
  }
  ctx->lev.assign(n_levels, Level());
  long long max_nd = 0;
  for (int l = 0; l < n_levels; ++l) {
    Level& L = ctx->lev[l];
    const int ml = m >> (n_levels - 1 - l);
    L.g.m = ml;
    L.g.L = degree * ml + 1;
    L.g.ncells = 1;
    for (int i = 0; i < dim; ++i) L.g.ncells *= ml;
    for (int f = 0; f < 6; ++f) L.g.fm[f] = ctx->fm[f];
    L.g.h = 1.0 / ml;
    L.g.inv_h = (double)ml;
    L.nnodes = 1;
    for (int i = 0; i < dim; ++i) L.nnodes *= L.g.L;
    L.ndofs = L.nnodes * dim;
    L.nqp = (long long)L.g.ncells * ipow(degree + 1, dim);
    HY_TRY(dalloc(ctx, &L.d_u64, L.ndofs));
    HY_TRY(dalloc(ctx, &L.d_diag, L.ndofs));
    HY_TRY(dalloc(ctx, &L.d_mat, L.g.ncells));
    max_nd = std::max(max_nd, L.ndofs);
  }
  {
    const Level& C = ctx->lev[0];
    const int Lc = C.g.L;
    long long nf = 0;
    for (long long nd = 0; nd < C.nnodes; ++nd) {
      const int i0 = (int)(nd % Lc), i1 = (int)((nd / Lc) % Lc), i2 = dim == 3 ? (int)(nd / ((long long)Lc * Lc)) : 0;
      uint32_t cm = 0;
      if (i0 == 0) cm |= C.g.fm[0];
      if (i0 == Lc - 1) cm |= C.g.fm[1];
      if (i1 == 0) cm |= C.g.fm[2];
      if (i1 == Lc - 1) cm |= C.g.fm[3];
      if (dim == 3 && i2 == 0) cm |= C.g.fm[4];
      if (dim == 3 && i2 == Lc - 1) cm |= C.g.fm[5];
      for (int c = 0; c < dim; ++c) nf += ((cm >> c) & 1u) ? 0 : 1;
    }
    ctx->coarse_nfree = nf;
  }
  // transfer tables
  ctx->tr.assign(n_levels, Transfer());
  size_t tmp_len = 1;
  const std::vector<double> gl = gll_points(degree);
  for (int l = 1; l < n_levels; ++l) {
    Transfer& t = ctx->tr[l];
    const int k = degree, n = degree + 1;
    const int mc = ctx->lev[l - 1].g.m;
    t.Lc = ctx->lev[l - 1].g.L;
    t.Lf = ctx->lev[l].g.L;
    // prolongation: fine node i in fine cell cf = coarse cell cf/2 at local position ((cf%2) + x_j)/2
    std::vector<double> P((size_t)t.Lf * t.Lc, 0.0);
    std::vector<int> pstart(t.Lf);
    std::vector<double> pw((size_t)t.Lf * n, 0.0);
    for (int i = 0; i < t.Lf; ++i) {
      const int cf = std::min(i / k, 2 * mc - 1);
      const int j = i - k * cf;
      const int c = cf / 2;
      const double xi = ((cf % 2) + gl[j]) / 2.0;
      pstart[i] = k * c;
      for (int e = 0; e < n; ++e) {
        double v = lagr(gl, e, xi);
        if (std::fabs(v) < 1e-15) v = 0.0;
        pw[(size_t)i * n + e] = v;
        P[(size_t)i * t.Lc + k * c + e] = v;
      }
    }
    t.Ep = n;
    // restriction = P^T: for coarse node J the fine rows with a nonzero entry form a contiguous range
    t.Er = std::min(4 * k + 1, t.Lf);
    std::vector<int> rstart(t.Lc);
    std::vector<double> rw((size_t)t.Lc * t.Er, 0.0);
    for (int J = 0; J < t.Lc; ++J) {
      int first = -1;
      for (int i = 0; i < t.Lf; ++i)
        if (P[(size_t)i * t.Lc + J] != 0.0) { first = i; break; }
      if (first < 0) first = 0;
      first = std::min(first, t.Lf - t.Er);
      rstart[J] = first;
      for (int e = 0; e < t.Er; ++e) rw[(size_t)J * t.Er + e] = P[(size_t)(first + e) * t.Lc + J];
    }
    // interpolation down: coarse node J at coarse-cell position x_j lies in fine cell 2c (x_j < 1/2)
    // or 2c+1, at fine-cell position 2 x_j or 2 x_j - 1
    t.Ei = n;
    std::vector<int> istart(t.Lc);
    std::vector<double> iw((size_t)t.Lc * n, 0.0);
    for (int J = 0; J < t.Lc; ++J) {
      const int c = std::min(J / k, mc - 1);
      const int j = J - k * c;
      const int f = gl[j] < 0.5 ? 2 * c : 2 * c + 1;
      const double xi = gl[j] < 0.5 ? 2.0 * gl[j] : 2.0 * gl[j] - 1.0;
      istart[J] = k * f;
      for (int e = 0; e < n; ++e) {
        double v = lagr(gl, e, xi);
        if (std::fabs(v) < 1e-15) v = 0.0;
        iw[(size_t)J * n + e] = v;
      }
    }
    std::vector<float> pw32(pw.begin(), pw.end()), rw32(rw.begin(), rw.end());
    HY_TRY(dalloc(ctx, &t.d_pstart, t.Lf));
    HY_TRY(dalloc(ctx, &t.d_rstart, t.Lc));
    HY_TRY(dalloc(ctx, &t.d_istart, t.Lc));
    HY_TRY(dalloc(ctx, &t.d_pw64, pw.size()));
    HY_TRY(dalloc(ctx, &t.d_rw64, rw.size()));
    HY_TRY(dalloc(ctx, &t.d_iw64, iw.size()));
    HY_TRY(dalloc(ctx, &t.d_pw32, pw.size()));
    HY_TRY(dalloc(ctx, &t.d_rw32, rw.size()));
    HY_CK(cudaMemcpyAsync(t.d_pstart, pstart.data(), sizeof(int) * t.Lf, cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_rstart, rstart.data(), sizeof(int) * t.Lc, cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_istart, istart.data(), sizeof(int) * t.Lc, cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_pw64, pw.data(), sizeof(double) * pw.size(), cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_rw64, rw.data(), sizeof(double) * rw.size(), cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_iw64, iw.data(), sizeof(double) * iw.size(), cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_pw32, pw32.data(), sizeof(float) * pw32.size(), cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaMemcpyAsync(t.d_rw32, rw32.data(), sizeof(float) * rw32.size(), cudaMemcpyHostToDevice, ctx->stream));
    HY_CK(cudaStreamSynchronize(ctx->stream));  // the host tables go out of scope
    size_t inter = (size_t)t.Lf * dim;
    for (int i = 1; i < dim; ++i) inter *= t.Lf;  // bounds every intermediate of the sweeps
    tmp_len = std::max(tmp_len, inter);
  }
  ctx->tmp_len = tmp_len;
  HY_TRY(dalloc(ctx, &ctx->tmp64a, tmp_len));
  HY_TRY(dalloc(ctx, &ctx->tmp64b, tmp_len));
  HY_TRY(dalloc(ctx, &ctx->tmp32a, tmp_len));
  HY_TRY(dalloc(ctx, &ctx->tmp32b, tmp_len));
  HY_TRY(dalloc(ctx, &ctx->tmp32c, tmp_len));
  HY_TRY(dalloc(ctx, &ctx->d_err, 2));  // [0] the context's stream, [1] the side stream of the coarse setup
  HY_TRY(dalloc(ctx, &ctx->d_jmin, 1));
  HY_TRY(dalloc(ctx, &ctx->d_partials, DOT_BLOCKS));
  HY_TRY(dalloc(ctx, &ctx->d_scal, 4));
  HY_TRY(dalloc(ctx, &ctx->d_face, 18));
  HY_TRY(dalloc(ctx, &ctx->d_eig_scal, 8 + PCG_SCALARS));
  for (int l = 1; l < n_levels; ++l) HY_TRY(dalloc(ctx, &ctx->lev[l].d_eigbuf, EIG_BUF_LEN));
  HY_TRY(dalloc(ctx, &ctx->d_usetup, ctx->lev[0].ndofs));
  HY_TRY(dalloc(ctx, &ctx->d_udiff, ctx->lev[0].ndofs));
  for (int i = 0; i < 12; ++i) HY_TRY(dalloc(ctx, &ctx->f64[i], ctx->lev[n_levels - 1].ndofs));
  HY_CK(cudaMemsetAsync(ctx->d_err, 0, 2 * sizeof(unsigned), ctx->stream));
  HY_CK(cudaStreamSynchronize(ctx->stream));
  return HY_OK;
}

hy_status hy_num_dofs(const hy_ctx* ctx, int level, int64_t* n) {
  if (!ctx || !n) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return HY_ERR_ARG;
  *n = ctx->lev[l].ndofs;
  return HY_OK;
}

hy_status hy_set_material(hy_ctx* ctx, int level, const uint8_t* cell_mat, const double* mu, const double* lambda,
                          int n_mat) {
  if (!ctx) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "level out of range");
  if (!cell_mat || !mu || !lambda || n_mat < 1 || n_mat > MAXMAT) return fail(ctx, HY_ERR_ARG, "bad material arrays");
  Level& L = ctx->lev[l];
  for (int i = 0; i < L.g.ncells; ++i)
    if (cell_mat[i] >= n_mat) return fail(ctx, HY_ERR_ARG, "material id out of range");
  for (int i = 0; i < n_mat; ++i)
    if (!(mu[i] > 0.0) || !(lambda[i] > -2.0 / 3.0 * mu[i]) || !std::isfinite(lambda[i]))
      return fail(ctx, HY_ERR_ARG, "material parameters out of range");
  HY_CK(cudaSetDevice(ctx->device));
  HY_CK(cudaMemcpyAsync(L.d_mat, cell_mat, L.g.ncells, cudaMemcpyHostToDevice, ctx->stream));
  HY_CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < MAXMAT; ++i) {
    L.mt64.mu[i] = i < n_mat ? mu[i] : 0.0;
    L.mt64.lam[i] = i < n_mat ? lambda[i] : 0.0;
    L.mt32.mu[i] = (float)L.mt64.mu[i];
    L.mt32.lam[i] = (float)L.mt64.lam[i];
    L.mtff.mu[i] = ff(L.mt64.mu[i]);
    L.mtff.lam[i] = ff(L.mt64.lam[i]);
  }
  L.mat_set = true;
  ctx->state_ok = false;
  ctx->setup_valid = false;
  return HY_OK;
}

hy_status hy_set_displacement(hy_ctx* ctx, const double* u_dev, hy_variant variant, hy_dtype level_dtype) {
  if (!ctx || !u_dev) return HY_ERR_ARG;
  if (level_dtype != HY_F64 && level_dtype != HY_F32) return fail(ctx, HY_ERR_ARG, "bad dtype");
  HY_CK(cudaSetDevice(ctx->device));
  return set_displacement(ctx, u_dev, (int)variant, level_dtype == HY_F32);
}

hy_status hy_vmult(hy_ctx* ctx, int level, const void* x, void* y, hy_dtype dtype) {
  if (!ctx || !x || !y) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "level out of range");
  if (!ctx->state_ok) return fail(ctx, HY_ERR_STATE, "set_displacement first");
  if (x == y) return fail(ctx, HY_ERR_ARG, "x and y must not alias");
  HY_CK(cudaSetDevice(ctx->device));
  if (dtype == HY_F64) return vmult<double>(ctx, l, (const double*)x, (double*)y);
  if (dtype == HY_F32) return vmult<float>(ctx, l, (const float*)x, (float*)y);
  if (dtype == HY_FF) return vmult<ff>(ctx, l, (const double*)x, (double*)y);
  return fail(ctx, HY_ERR_ARG, "bad dtype");
}

hy_status hy_apply_tangent(hy_ctx* ctx, const void* x, void* y, hy_dtype dtype) {
  if (!ctx) return HY_ERR_ARG;
  return hy_vmult(ctx, -1, x, y, dtype);
}

hy_status hy_residual(hy_ctx* ctx, const double* u, double* r) {
  if (!ctx || !u || !r) return HY_ERR_ARG;
  if (ctx->nlev == 0) return fail(ctx, HY_ERR_STATE, "mesh not set up");
  if (!ctx->lev[ctx->nlev - 1].mat_set) return fail(ctx, HY_ERR_STATE, "material not set");
  HY_CK(cudaSetDevice(ctx->device));
  const Range range("residual");
  HY_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
  HY_TRY(residual(ctx, u, r));
  return check_error_word(ctx, "residual");
}

hy_status hy_diagonal(hy_ctx* ctx, int level, void* d, hy_dtype dtype) {
  if (!ctx || !d) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "level out of range");
  if (!ctx->state_ok) return fail(ctx, HY_ERR_STATE, "set_displacement first");
  HY_CK(cudaSetDevice(ctx->device));
  Level& L = ctx->lev[l];
  if (dtype == HY_F64) {
    HY_CK(cudaMemcpyAsync(d, L.d_diag, sizeof(double) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
    return HY_OK;
  }
  if (dtype == HY_F32) {
    launch_convert<double, float>(L.d_diag, (float*)d, L.ndofs, ctx->stream);
    return check_launch(ctx, 1);
  }
  return fail(ctx, HY_ERR_ARG, "bad dtype");
}

hy_status hy_gmg_vcycle(hy_ctx* ctx, const double* r, double* z) {
  if (!ctx || !r || !z) return HY_ERR_ARG;
  if (!ctx->state_ok) return fail(ctx, HY_ERR_STATE, "set_displacement first");
  HY_CK(cudaSetDevice(ctx->device));
  const Range range("gmg_vcycle");
  return vcycle_top(ctx, r, z);
}

hy_status hy_set_solver_params(hy_ctx* ctx, const hy_solver_params* p) {
  if (!ctx || !p) return HY_ERR_ARG;
  if (p->cheb_degree < 1 || p->cheb_sweeps < 1 || !(p->cheb_lo > 0) || !(p->cheb_hi > p->cheb_lo) ||
      p->kernel_form < -1 || p->kernel_form > 3 || (p->fine_dtype != HY_F64 && p->fine_dtype != HY_FF) ||
      p->level_variant < -1 || p->level_variant > 4 ||
      p->eig_iters < 1 || p->coarse_eig_iters < 0 || !(p->coarse_reduction > 0 && p->coarse_reduction < 1) ||
      p->coarse_solver < 0 || p->coarse_solver > 2 || !(p->setup_reuse >= 0.0))
    return fail(ctx, HY_ERR_ARG, "solver parameters out of range");
  ctx->sp = *p;
  ctx->state_ok = false;
  ctx->setup_valid = false;
  drop_graph(ctx);
  return HY_OK;
}

hy_status hy_get_solver_params(const hy_ctx* ctx, hy_solver_params* p) {
  if (!ctx || !p) return HY_ERR_ARG;
  *p = ctx->sp;
  return HY_OK;
}

hy_status hy_level_info(const hy_ctx* ctx, int level, double* lmax, double* clo, double* chi, int* cdeg) {
  if (!ctx) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return HY_ERR_ARG;
  if (lmax) *lmax = ctx->lev[l].lmax;
  if (clo) *clo = ctx->coarse_lo;
  if (chi) *chi = ctx->coarse_hi;
  if (cdeg) *cdeg = ctx->coarse_deg;
  return HY_OK;
}

hy_status hy_set_level_info(hy_ctx* ctx, int level, double lmax, double clo, double chi) {
  if (!ctx) return HY_ERR_ARG;
  drop_graph(ctx);
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "level out of range");
  if (l == 0) {
    if (!(chi > clo && clo > 0)) return fail(ctx, HY_ERR_ARG, "bad coarse interval");
    ctx->coarse_lo = clo;
    ctx->coarse_hi = chi;
    ctx->coarse_spd = true;
    const double sig = (chi + clo) / (chi - clo);
    ctx->coarse_deg = std::max(1, (int)std::ceil(std::acosh(1.0 / ctx->sp.coarse_reduction) / std::acosh(sig) - 1e-12));
  } else {
    if (!(lmax > 0)) return fail(ctx, HY_ERR_ARG, "bad lmax");
    ctx->lev[l].lmax = lmax;
  }
  return HY_OK;
}

hy_status hy_face_load(hy_ctx* ctx, const double traction[6][3], double* f) {
  if (!ctx || !traction || !f) return HY_ERR_ARG;
  if (ctx->nlev == 0) return fail(ctx, HY_ERR_STATE, "mesh not set up");
  HY_CK(cudaSetDevice(ctx->device));
  bool any = false;
  return face_load(ctx, traction, f, &any);
}

hy_status hy_set_geometry(hy_ctx* ctx, const double* X) {
  if (!ctx) return HY_ERR_ARG;
  if (ctx->nlev == 0) return fail(ctx, HY_ERR_STATE, "mesh not set up");
  HY_CK(cudaSetDevice(ctx->device));
  ctx->state_ok = false;
  ctx->setup_valid = false;
  drop_graph(ctx);
  if (!X) {
    ctx->curved = false;
    return HY_OK;
  }
  const int top = ctx->nlev - 1;
  for (int l = 0; l < ctx->nlev; ++l)
    if (!ctx->lev[l].d_X64) HY_TRY(dalloc(ctx, &ctx->lev[l].d_X64, ctx->lev[l].ndofs));
  HY_CK(cudaMemcpyAsync(ctx->lev[top].d_X64, X, sizeof(double) * ctx->lev[top].ndofs, cudaMemcpyDeviceToDevice,
                        ctx->stream));
  for (int l = top; l >= 1; --l) HY_TRY(interpolate_down_vec(ctx, l, ctx->lev[l].d_X64, ctx->lev[l - 1].d_X64));
  ctx->curved = true;
  return HY_OK;
}

hy_status hy_check_bounded_wait(hy_ctx* ctx, double limit_s) {
  if (!ctx) return HY_ERR_ARG;
  if (!ctx->d_err) return fail(ctx, HY_ERR_STATE, "check_bounded_wait: no mesh");
  if (!(limit_s >= 1e-3 && limit_s <= 10.0)) return fail(ctx, HY_ERR_ARG, "check_bounded_wait: limit_s outside [1e-3, 10]");
  launch_bounded_wait_check(ctx->d_err, (unsigned long long)(limit_s * 1e9), ctx->stream);
  HY_TRY(check_launch(ctx, 1));
  return check_error_word(ctx, "check_bounded_wait");
}

hy_status hy_set_material_law(hy_ctx* ctx, int law) {
  if (!ctx) return HY_ERR_ARG;
  if (law != HY_LAW_LOG2 && law != HY_LAW_J2) return fail(ctx, HY_ERR_ARG, "unknown material law");
  ctx->law = law;
  ctx->state_ok = false;
  ctx->setup_valid = false;
  drop_graph(ctx);
  return HY_OK;
}

hy_status hy_kernel_form(const hy_ctx* ctx, int level, hy_dtype dtype, int* form) {
  if (!ctx || !form || (dtype != HY_F64 && dtype != HY_F32 && dtype != HY_FF)) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return HY_ERR_ARG;
  const Level& L = ctx->lev[l];
  const bool have = dtype == HY_F64 ? L.has64 : dtype == HY_F32 ? L.has32 : L.hasff;
  *form = have ? L.form[dtype == HY_F64 ? 0 : dtype == HY_F32 ? 1 : 2] : -1;
  return HY_OK;
}

hy_status hy_level_displacement(const hy_ctx* cctx, int level, double* u) {
  hy_ctx* ctx = const_cast<hy_ctx*>(cctx);
  if (!ctx || !u) return HY_ERR_ARG;
  const int l = lev_index(ctx, level);
  if (l < 0 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "level out of range");
  HY_CK(cudaSetDevice(ctx->device));
  HY_CK(cudaMemcpyAsync(u, ctx->lev[l].d_u64, sizeof(double) * ctx->lev[l].ndofs, cudaMemcpyDeviceToDevice, ctx->stream));
  return HY_OK;
}

hy_status hy_prolongate_add(hy_ctx* ctx, int fine_level, const void* coarse, void* fine, hy_dtype dtype) {
  if (!ctx || !coarse || !fine) return HY_ERR_ARG;
  const int l = lev_index(ctx, fine_level);
  if (l < 1 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "fine level must be >= 1");
  HY_CK(cudaSetDevice(ctx->device));
  if (dtype == HY_F64) return prolongate_add<double>(ctx, l, (const double*)coarse, (double*)fine);
  if (dtype == HY_F32) return prolongate_add<float>(ctx, l, (const float*)coarse, (float*)fine);
  return fail(ctx, HY_ERR_ARG, "bad dtype");
}

hy_status hy_restrict(hy_ctx* ctx, int fine_level, const void* fine, void* coarse, hy_dtype dtype) {
  if (!ctx || !coarse || !fine) return HY_ERR_ARG;
  const int l = lev_index(ctx, fine_level);
  if (l < 1 || l >= ctx->nlev) return fail(ctx, HY_ERR_ARG, "fine level must be >= 1");
  HY_CK(cudaSetDevice(ctx->device));
  if (dtype == HY_F64) return restrict_to<double>(ctx, l, (const double*)fine, (double*)coarse);
  if (dtype == HY_F32) return restrict_to<float>(ctx, l, (const float*)fine, (float*)coarse);
  return fail(ctx, HY_ERR_ARG, "bad dtype");
}

hy_status hy_pcg(hy_ctx* ctx, const double* b, double* x, double rtol, int max_iter, int* iterations) {
  if (!ctx || !b || !x || !(rtol > 0) || max_iter < 1) return HY_ERR_ARG;
  if (!ctx->state_ok) return fail(ctx, HY_ERR_STATE, "set_displacement first");
  HY_CK(cudaSetDevice(ctx->device));
  return pcg(ctx, b, x, rtol, max_iter, iterations);
}

void hy_newton_default_params(hy_newton_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->load_steps = 5;
  p->max_newton = 25;
  p->newton_rtol = 1e-10;
  p->newton_atol = 1e-14;
  p->cg_rtol = 1e-8;
  p->cg_max_iter = 1000;
  p->variant = HY_T4;
  p->level_dtype = HY_F64;
}

hy_status hy_newton_solve(hy_ctx* ctx, const hy_newton_params* p, double* u, hy_newton_report* rep) {
  if (!ctx || !p || !u) return HY_ERR_ARG;
  if (p->load_steps < 1 || p->max_newton < 1 || !(p->newton_rtol > 0) || !(p->cg_rtol > 0) || p->cg_max_iter < 1)
    return fail(ctx, HY_ERR_ARG, "newton parameters out of range");
  const int s_first = p->first_step > 0 ? p->first_step : 1;
  const int s_last = p->last_step > 0 ? p->last_step : p->load_steps;
  if (p->first_step < 0 || p->last_step < 0 || s_first > s_last || s_last > p->load_steps)
    return fail(ctx, HY_ERR_ARG, "newton: need 1 <= first_step <= last_step <= load_steps");
  if (ctx->nlev == 0) return fail(ctx, HY_ERR_STATE, "mesh not set up");
  const Range range_solve("hy_newton_solve");
  HY_CK(cudaSetDevice(ctx->device));
  hy_newton_report rl;
  std::memset(&rl, 0, sizeof(rl));
  Level& L = ctx->lev[ctx->nlev - 1];
  const long long n = L.ndofs;
  double *R = ctx->f64[4], *du0 = ctx->f64[5], *rhs = ctx->f64[6], *du = ctx->f64[7], *trial = ctx->f64[8],
         *t = ctx->f64[9], *fext = ctx->f64[11];
  HY_CK(cudaMemcpyAsync(ctx->d_face, p->face_values, sizeof(double) * 18, cudaMemcpyHostToDevice, ctx->stream));
  bool loaded = false;  // dead tractions: R = R_int - factor * f_ext (the tangent is unchanged)
  HY_TRY(face_load(ctx, p->face_traction, fext, &loaded));
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t0) { return std::chrono::duration<double, std::milli>(clk::now() - t0).count(); };
  const clk::time_point t_start = clk::now();
  hy_status st = HY_OK;
  for (int s = s_first; s <= s_last && st == HY_OK; ++s) {
    const Range range_step("load step");
    const double factor = (double)s / p->load_steps;
    double ref = -1.0;
    int its = 0;
    while (true) {
      launch_lift(u, du0, factor, ctx->d_face, L.nnodes, ctx->dim, L.g, ctx->stream);
      HY_TRY(check_launch(ctx, 1));
      double lift2;
      HY_TRY(dot<double>(ctx, du0, du0, n, &lift2));
      HY_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
      HY_TRY(residual(ctx, u, R));
      if ((st = check_error_word(ctx, "newton residual")) != HY_OK) break;
      if (loaded) {
        launch_axpby<double>(-factor, fext, 1.0, R, n, ctx->stream);
        launch_zero_constrained<double>(R, L.nnodes, ctx->dim, L.g, ctx->stream);
        HY_TRY(check_launch(ctx, 2));
      }
      if (its > 0 && lift2 == 0.0) {
        double rr;
        HY_TRY(dot<double>(ctx, R, R, n, &rr));
        rl.final_residual = std::sqrt(rr);
        if (ctx->verbose) std::fprintf(stderr, "[hy] step %d it %d |R| %.3e ref %.3e\n", s, its, std::sqrt(rr), ref);
        if (std::sqrt(rr) <= std::max(p->newton_rtol * ref, p->newton_atol)) break;
      }
      if (its >= p->max_newton) {
        st = fail(ctx, HY_ERR_NOCONV, "newton: iteration cap in load step " + std::to_string(s));
        break;
      }
      const clk::time_point t_setup = clk::now();
      if ((st = set_displacement(ctx, u, (int)p->variant, p->level_dtype == HY_F32)) != HY_OK) break;
      HY_CK(cudaStreamSynchronize(ctx->stream));
      rl.setup_ms_total += ms_since(t_setup);
      if (ctx->last_setup_reused) rl.setups_reused++;
      {
        double ph[SETUP_PHASES + 1];
        setup_phases_ms(ctx, ph);
        for (int i = 0; i <= SETUP_PHASES; ++i) rl.setup_phase_ms[i] += ph[i];
      }
      // rhs = -R - Z A du0 (lifting of the prescribed increment into the first solve)
      HY_CK(cudaMemcpyAsync(rhs, R, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
      if (lift2 > 0.0) {
        // in the finest-level action of the outer CG (double-float when fine_dtype asks for it)
        if (ctx->sp.fine_dtype == HY_FF && ctx->lev[ctx->nlev - 1].hasff) HY_TRY(vmult<ff>(ctx, ctx->nlev - 1, du0, t, false));
        else HY_TRY(vmult<double>(ctx, ctx->nlev - 1, du0, t, false));
        launch_axpby<double>(-1.0, t, -1.0, rhs, n, ctx->stream);  // rhs = -A du0 - R
      } else {
        launch_axpby<double>(0.0, R, -1.0, rhs, n, ctx->stream);   // rhs = -R
      }
      HY_TRY(check_launch(ctx, 1));
      double rr;
      HY_TRY(dot<double>(ctx, rhs, rhs, n, &rr));
      if (ref < 0) ref = std::sqrt(rr);
      rl.final_residual = std::sqrt(rr);
      if (ctx->verbose) std::fprintf(stderr, "[hy] step %d it %d |rhs| %.3e lift2 %.3e\n", s, its, std::sqrt(rr), lift2);
      int cg_its = 0;
      HY_CK(cudaStreamSynchronize(ctx->stream));
      const clk::time_point t_solve = clk::now();
      st = ctx->solve_hook ? ctx->solve_hook(ctx->solve_user, ctx, rhs, du, p->cg_rtol, p->cg_max_iter, &cg_its)
                           : pcg(ctx, rhs, du, p->cg_rtol, p->cg_max_iter, &cg_its);
      HY_CK(cudaStreamSynchronize(ctx->stream));
      if (rl.n_solves < 256) {
        rl.solve_ms[rl.n_solves] = ms_since(t_solve);
        rl.solve_cg_iterations[rl.n_solves] = cg_its;
      }
      rl.n_solves++;
      if (st != HY_OK) break;
      rl.cg_iterations_total += cg_its;
      if (ctx->verbose) std::fprintf(stderr, "[hy] step %d it %d cg %d\n", s, its, cg_its);
      rl.cg_iterations_max = std::max(rl.cg_iterations_max, cg_its);
      launch_axpby<double>(1.0, du0, 1.0, du, n, ctx->stream);  // du = delta + du0
      HY_TRY(check_launch(ctx, 1));
      double step = 1.0;
      bool ok = false;
      for (int h = 0; h < 6; ++h) {
        launch_xpay<double>(u, step, du, trial, n, ctx->stream);
        HY_TRY(check_launch(ctx, 1));
        HY_TRY(jacobian_ok(ctx, trial, ok));
        if (ok) break;
        step *= 0.5;
        rl.backtracks++;
      }
      if (!ok) {
        st = fail(ctx, HY_ERR_JNEG, "newton: J <= 0 after 5 halvings");
        break;
      }
      HY_CK(cudaMemcpyAsync(u, trial, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
      ++its;
    }
    if (s <= 64) rl.newton_iterations[s - 1] = its;
    if (st == HY_OK) rl.load_steps_done = s;
  }
  HY_CK(cudaStreamSynchronize(ctx->stream));
  rl.total_ms = ms_since(t_start);
  if (rep) *rep = rl;
  return st;
}

hy_status hy_dot(hy_ctx* ctx, const double* a, const double* b, int64_t n, double* result) {
  if (!ctx || !a || !b || !result || n < 0) return HY_ERR_ARG;
  if (!ctx->d_partials) return fail(ctx, HY_ERR_STATE, "mesh not set up (scratch not allocated)");
  HY_CK(cudaSetDevice(ctx->device));
  return dot<double>(ctx, a, b, (long long)n, result);
}

// Device bytes a context needs for a problem, mirroring the allocations of hy_mesh_setup and
// hy_set_displacement (requested sizes; the allocator's own rounding comes on top).
hy_status hy_footprint(int dim, int degree, int m, int n_levels, hy_variant variant, hy_dtype level_dtype,
                       const hy_solver_params* sp, const uint32_t* face_masks, int64_t* bytes) {
  return hy_footprint_general(dim, degree, m, n_levels, variant, level_dtype, sp, face_masks, false, bytes);
}

}  // extern "C"

hy_status hy_footprint_general(int dim, int degree, int m, int n_levels, hy_variant variant, hy_dtype level_dtype,
                               const hy_solver_params* sp, const uint32_t* face_masks, bool general,
                               int64_t* bytes) {
  if (!bytes || (dim != 2 && dim != 3) || degree < 1 || degree > 4 || m < 1 || n_levels < 1) return HY_ERR_ARG;
  const int coarse_solver = sp ? sp->coarse_solver : 0;
  const hy_dtype fine_dtype = sp ? sp->fine_dtype : HY_F64;
  const int level_variant = sp ? sp->level_variant : -1;
  if (fine_dtype != HY_F64 && fine_dtype != HY_FF) return HY_ERR_ARG;
  if (coarse_solver < 0 || coarse_solver > 2 || level_variant < -1 || level_variant > 4) return HY_ERR_ARG;
  if ((int)variant < 0 || (int)variant > 4) return HY_ERR_ARG;
  auto al = [](size_t n, size_t sz) { return std::max<size_t>(n, 1) * sz; };
  const int n = degree + 1;
  const bool mixed = level_dtype == HY_F32;
  size_t total = 0, tmp_len = 1;
  std::vector<long long> nd(n_levels), L1(n_levels), nc(n_levels);
  for (int l = 0; l < n_levels; ++l) {
    const long long ml = (long long)m >> (n_levels - 1 - l);
    if (ml < 1) return HY_ERR_ARG;
    L1[l] = degree * ml + 1;
    nc[l] = 1;
    long long nn = 1;
    for (int i = 0; i < dim; ++i) {
      nc[l] *= ml;
      nn *= L1[l];
    }
    nd[l] = nn * dim;
    total += al(nd[l], 8) * 2 + al(nc[l], 1);  // u64, diag, materials
  }
  for (int l = 1; l < n_levels; ++l) {
    const long long Lc = L1[l - 1], Lf = L1[l];
    const long long Er = std::min<long long>(4 * degree + 1, Lf);
    total += al(Lf, 4) + 2 * al(Lc, 4) + al(Lf * n, 8) + al(Lc * Er, 8) + al(Lc * n, 8) + al(Lf * n, 4) + al(Lc * Er, 4);
    size_t inter = (size_t)Lf * dim;
    for (int i = 1; i < dim; ++i) inter *= Lf;
    tmp_len = std::max(tmp_len, inter);
  }
  total += 2 * al(tmp_len, 8) + 3 * al(tmp_len, 4);
  total += al(2, 4) + al(1, 8) + al(DOT_BLOCKS, 8) + al(4, 8) + al(18, 8) + al(8 + PCG_SCALARS, 8);
  total += (size_t)(n_levels - 1) * al(EIG_BUF_LEN, 8);  // the smoother estimates' per-level buffers
  total += 2 * al(nd[0], 8);  // coarsest-level displacement of the last full setup, and a difference
  total += 12 * al(nd[n_levels - 1], 8);
  const int top = n_levels - 1;
  for (int l = 0; l < n_levels; ++l) {
    const bool need64 = (l == top) || (l == 0) || !mixed;
    const bool need32 = mixed && (l > 0 || l == top);
    const int cb64 = layout_cells<double>(dim, n), cb32 = layout_cells<float>(dim, n);
    // as set_displacement assigns them
    auto build_of = [general](int v) { return (general && v >= VAR_FC && v <= VAR_NC) ? v - VAR_FC + VAR_FCG : v; };
    const int lvar = build_of(level_variant >= 0 ? level_variant : (int)variant);
    const int var64 = l == top ? build_of((int)variant) : lvar;
    const size_t clen64 = std::max<size_t>(1, (size_t)cache_values(var64, dim) * layout_row<double>(dim, n) *
                                                  (size_t)((nc[l] + cb64 - 1) / cb64));
    const size_t clen32 = std::max<size_t>(1, (size_t)cache_values(lvar, dim) * layout_row<float>(dim, n) *
                                                  (size_t)((nc[l] + cb32 - 1) / cb32));
    if (need64) total += al(clen64, 8) + al(nd[l], 8) + 5 * al(nd[l], 8);
    if (l == top && fine_dtype == HY_FF) total += al(clen64, 8);  // double-float cache: the FP64 layout, variant
    if (need32) total += al(clen32, 4) + al(nd[l], 4) + al(nd[l], 4) + 5 * al(nd[l], 4);
  }
  // free dofs of the coarsest level (all dofs bound them when no masks are given)
  size_t nf = (size_t)nd[0];
  {
    if (face_masks) {
      nf = 0;
      const long long Lc = L1[0];
      const long long nn = nd[0] / dim;
      for (long long q = 0; q < nn; ++q) {
        const long long i0 = q % Lc, i1 = (q / Lc) % Lc, i2 = dim == 3 ? q / (Lc * Lc) : 0;
        uint32_t cm = 0;
        if (i0 == 0) cm |= face_masks[0];
        if (i0 == Lc - 1) cm |= face_masks[1];
        if (i1 == 0) cm |= face_masks[2];
        if (i1 == Lc - 1) cm |= face_masks[3];
        if (dim == 3 && i2 == 0) cm |= face_masks[4];
        if (dim == 3 && i2 == Lc - 1) cm |= face_masks[5];
        for (int c = 0; c < dim; ++c) nf += ((cm >> c) & 1u) ? 0 : 1;
      }
    }
  }
  if (coarse_solver >= 1) total += 2 * al(nf * nf, 8) + al(32 * 32 + 64 * nf, 8) + al(nf, 4) + al(nd[0], 4);
  // eigenvalue-estimate history for the default solver parameters (30 smoother iterations, all free
  // coarse dofs for the Chebyshev coarse solver)
  total += al((size_t)(2 * std::max<long long>({n_levels > 1 ? 30LL : 0LL,
                                                coarse_solver < 1 ? std::max<long long>((long long)nf, 1) : 0LL, 1LL})),
              8);
  *bytes = (int64_t)total;
  return HY_OK;
}

extern "C" {

hy_status hy_ctx_bytes(const hy_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return HY_ERR_ARG;
  *bytes = (int64_t)ctx->bytes;
  return HY_OK;
}

hy_status hy_kernel_launches(const hy_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return HY_ERR_ARG;
  *count = ctx->launches;
  return HY_OK;
}

hy_status hy_batch_create(hy_batch** out, hy_ctx* const* ctxs, int count) {
  if (!out) return HY_ERR_ARG;
  *out = nullptr;
  if (!ctxs || count < 1 || count > HY_BATCH_MAX) return HY_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || ctxs[i]->nlev == 0) return HY_ERR_STATE;
    if (ctxs[i]->device != ctxs[0]->device || ctxs[i]->dim != ctxs[0]->dim || ctxs[i]->n != ctxs[0]->n)
      return HY_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return HY_ERR_ARG;
  }
  if (cudaSetDevice(ctxs[0]->device) != cudaSuccess) return HY_ERR_CUDA;
  hy_batch* b = new (std::nothrow) hy_batch();
  if (!b) return HY_ERR_OOM;
  b->device = ctxs[0]->device;
  b->dim = ctxs[0]->dim;
  b->n = ctxs[0]->n;
  b->ctx.assign(ctxs, ctxs + count);
  b->branch.assign(count, nullptr);
  b->ev.assign(count, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < count && ok; ++i)
    ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_upload, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_list, BATCH_ARG_BYTES * count) == cudaSuccess &&
       cudaMalloc((void**)&b->d_start, sizeof(int) * (count + 1)) == cudaSuccess &&
       cudaMalloc((void**)&b->d_scal, sizeof(double) * PCG_SCALARS * count) == cudaSuccess &&
       cudaMallocHost(&b->h_list, BATCH_ARG_BYTES * count) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_start, sizeof(int) * (count + 1)) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_scal_in, sizeof(double) * PCG_SCALARS * count) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_scal_out, sizeof(double) * PCG_SCALARS * count) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    return HY_ERR_OOM;
  }
  *out = b;
  return HY_OK;
}

void hy_batch_destroy(hy_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  batch_free(b);
}

const char* hy_batch_last_error(const hy_batch* b) { return b ? b->err.c_str() : "null batch"; }

hy_status hy_batch_apply(hy_batch* b, const void* const* x, void* const* y, hy_dtype dtype) {
  if (!b || !x || !y) return HY_ERR_ARG;
  HB_CK(cudaSetDevice(b->device));
  HY_TRY(batch_check(b));
  if (dtype == HY_F64) return batch_apply<double>(b, x, y);
  if (dtype == HY_F32) return batch_apply<float>(b, x, y);
  if (dtype == HY_FF) return batch_apply<ff>(b, x, y);
  return bfail(b, HY_ERR_ARG, "bad dtype");
}

hy_status hy_batch_pcg(hy_batch* b, const double* const* rhs, double* const* x, double rtol, int max_iter,
                       int* iterations, hy_status* status) {
  if (!b || !rhs || !x || !iterations || !status || !(rtol > 0) || max_iter < 1) return HY_ERR_ARG;
  HB_CK(cudaSetDevice(b->device));
  HY_TRY(batch_check(b));
  return batch_pcg(b, rhs, x, rtol, max_iter, iterations, status);
}

hy_status hy_batch_kernel_launches(const hy_batch* b, int64_t* count) {
  if (!b || !count) return HY_ERR_ARG;
  *count = b->launches;
  return HY_OK;
}

hy_status hy_batch_kernel_form(const hy_batch* b, hy_dtype dtype, int* form) {
  if (!b || !form || (dtype != HY_F64 && dtype != HY_F32 && dtype != HY_FF)) return HY_ERR_ARG;
  *form = b->form[(int)dtype];
  return HY_OK;
}

}  // extern "C"

// ---- internal interface of the solve server (serve_internal.h) ----------------------------------
void hy_ctx_set_solve_hook(hy_ctx* ctx, hy_linear_solve_hook hook, void* user) {
  if (!ctx) return;
  ctx->solve_hook = hook;
  ctx->solve_user = user;
}

long long hy_ctx_batch_key(const hy_ctx* c) {
  if (!c || c->nlev == 0) return -1;
  const Level& L = c->lev[c->nlev - 1];
  const bool ff_action = c->sp.fine_dtype == HY_FF && L.hasff;
  long long key = c->dim;
  key = key * 8 + c->n;
  for (int d = 0; d < 3; ++d) key = key * 8 + (L.var[d] + 1);
  return key * 2 + (ff_action ? 1 : 0);
}

hy_status hy_batch_create_empty(hy_batch** out, int device, int capacity) {
  if (!out || capacity < 1 || capacity > HY_BATCH_MAX) return HY_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return HY_ERR_CUDA;
  hy_batch* b = new (std::nothrow) hy_batch();
  if (!b) return HY_ERR_OOM;
  b->device = device;
  b->branch.assign(capacity, nullptr);
  b->ev.assign(capacity, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < capacity && ok; ++i)
    ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_upload, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_list, BATCH_ARG_BYTES * capacity) == cudaSuccess &&
       cudaMalloc((void**)&b->d_start, sizeof(int) * (capacity + 1)) == cudaSuccess &&
       cudaMalloc((void**)&b->d_scal, sizeof(double) * PCG_SCALARS * capacity) == cudaSuccess &&
       cudaMallocHost(&b->h_list, BATCH_ARG_BYTES * capacity) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_start, sizeof(int) * (capacity + 1)) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_scal_in, sizeof(double) * PCG_SCALARS * capacity) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_scal_out, sizeof(double) * PCG_SCALARS * capacity) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    return HY_ERR_OOM;
  }
  *out = b;
  return HY_OK;
}

// New members: the uploaded argument list no longer describes them, and the list launch takes the kernel
// form that the autotuner chose for the largest member's finest level (it dominates the launch).
hy_status hy_batch_bind(hy_batch* b, hy_ctx* const* ctxs, int count) {
  if (!b || !ctxs || count < 1 || count > (int)b->branch.size()) return HY_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || ctxs[i]->nlev == 0) return HY_ERR_STATE;
    if (ctxs[i]->device != b->device || ctxs[i]->dim != ctxs[0]->dim || ctxs[i]->n != ctxs[0]->n)
      return HY_ERR_ARG;
  }
  HB_CK(cudaSetDevice(b->device));
  HB_CK(cudaEventSynchronize(b->ev_upload));  // the pinned staging of the previous members is free
  b->ctx.assign(ctxs, ctxs + count);
  b->dim = ctxs[0]->dim;
  b->n = ctxs[0]->n;
  b->up_dt = -1;
  b->up_x.clear();
  b->up_y.clear();
  const hy_ctx* big = ctxs[0];
  for (int i = 1; i < count; ++i)
    if (ctxs[i]->lev[ctxs[i]->nlev - 1].ndofs > big->lev[big->nlev - 1].ndofs) big = ctxs[i];
  for (int d = 0; d < 3; ++d) b->form[d] = big->lev[big->nlev - 1].form[d];
  return HY_OK;
}
