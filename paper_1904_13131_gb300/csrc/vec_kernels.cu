// Vector kernels of the solvers: Dirichlet handling, Chebyshev and CG updates, precision
// conversion, deterministic dot products, and the separable transfer sweeps of the multigrid.
// All are bandwidth-bound streams over lattice vectors; grids cover the vector with 256-thread
// blocks (grid-stride loops capped at a multiple of the SM count).
#include <algorithm>

#include "cell_kernels.cuh"
#include "launch.cuh"

namespace hy {
namespace {

constexpr int TPB = 256;

inline int grid_for(long long n) {
  long long g = (n + TPB - 1) / TPB;
  const long long cap = 152LL * 16;  // 16 resident blocks of 256 threads per SM, 152 SMs
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <int DIM>
__device__ __forceinline__ uint32_t cmask_of(const Geom& g, long long node) {
  const int i0 = (int)(node % g.L);
  const int i1 = (int)((node / g.L) % g.L);
  const int i2 = DIM == 3 ? (int)(node / ((long long)g.L * g.L)) : 0;
  return node_cmask<DIM>(g, i0, i1, i2);
}

template <typename T, int DIM>
__global__ void prep_out_kernel(const T* __restrict__ x, T* __restrict__ y, long long n_nodes, Geom g) {
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n_nodes; nd += (long long)gridDim.x * blockDim.x) {
    const uint32_t cm = cmask_of<DIM>(g, nd);
#pragma unroll
    for (int c = 0; c < DIM; ++c) y[nd * DIM + c] = ((cm >> c) & 1u) ? x[nd * DIM + c] : T(0);
  }
}

// prep_out of every problem of a work list: blockIdx.y = problem, x and y and the lattice from its arguments
template <typename T, int DIM>
__global__ void prep_out_list_kernel(const CellArgs<T>* __restrict__ list) {
  const CellArgs<T>& a = list[blockIdx.y];
  const long long n_nodes = (long long)a.g.L * a.g.L * (DIM == 3 ? a.g.L : 1);
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n_nodes; nd += (long long)gridDim.x * blockDim.x) {
    const uint32_t cm = cmask_of<DIM>(a.g, nd);
#pragma unroll
    for (int c = 0; c < DIM; ++c) a.y[nd * DIM + c] = ((cm >> c) & 1u) ? a.x[nd * DIM + c] : vec_t<T>(0);
  }
}

// f += t * int_face N_a dA for the lattice nodes of one face (the dead-load term of Eq. weak_form).
// On a cell face N_a is a product of 1D GLL-basis functions, so the integral is a product of 1D weights:
// along an in-face axis lattice index j gets h w1[j % k] from the cell it starts (if any) plus h w1[k] from
// the cell it ends (if any), with w1[i] the integral of basis function i over the unit interval.
template <int DIM>
__global__ void face_load_kernel(double* __restrict__ f, Geom g, int axis, int side, FaceLoad fl) {
  const long long L = g.L;
  const long long nface = DIM == 3 ? L * L : L;
  const int K = fl.k;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nface;
       idx += (long long)gridDim.x * blockDim.x) {
    long long j[3] = {0, 0, 0};
    long long rest = idx;
    double w = 1.0;
    for (int i = 0; i < DIM; ++i) {
      if (i == axis) {
        j[i] = side ? L - 1 : 0;
        continue;
      }
      j[i] = rest % L;
      rest /= L;
      const long long c = j[i] / K;
      const int r = (int)(j[i] % K);
      double wi = 0.0;
      if (c < g.m) wi += fl.w1[r];
      if (r == 0 && c > 0) wi += fl.w1[K];
      w *= wi * g.h;
    }
    const long long node = j[0] + L * (j[1] + (DIM == 3 ? L * j[2] : 0));
#pragma unroll
    for (int c = 0; c < DIM; ++c) f[node * DIM + c] += w * fl.t[c];
  }
}

template <typename T, int DIM>
__global__ void set_constrained_kernel(T* __restrict__ y, long long n_nodes, Geom g, T val) {
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n_nodes; nd += (long long)gridDim.x * blockDim.x) {
    const uint32_t cm = cmask_of<DIM>(g, nd);
    if (cm) {
#pragma unroll
      for (int c = 0; c < DIM; ++c)
        if ((cm >> c) & 1u) y[nd * DIM + c] = val;
    }
  }
}

template <int DIM>
__global__ void lift_kernel(const double* __restrict__ u, double* __restrict__ du0, double factor,
                            const double* __restrict__ fv, long long n_nodes, Geom g) {
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n_nodes; nd += (long long)gridDim.x * blockDim.x) {
    const int i[3] = {(int)(nd % g.L), (int)((nd / g.L) % g.L), DIM == 3 ? (int)(nd / ((long long)g.L * g.L)) : 0};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      // the prescribed value of the highest-numbered face constraining this component at this node
      int face = -1;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        if (i[a] == 0 && ((g.fm[2 * a] >> c) & 1u)) face = 2 * a;
        if (i[a] == g.L - 1 && ((g.fm[2 * a + 1] >> c) & 1u)) face = 2 * a + 1;
      }
      // the target is rounded on its own (no FMA contraction) so that u + du0 reproduces it exactly
      du0[nd * DIM + c] = face < 0 ? 0.0 : __dsub_rn(__dmul_rn(factor, fv[face * 3 + c]), u[nd * DIM + c]);
    }
  }
}

template <typename T>
__global__ void invert_kernel(const double* __restrict__ d, T* __restrict__ dinv, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dinv[i] = T(1.0 / d[i]);
}

template <typename TA, typename TB>
__global__ void convert_kernel(const TA* __restrict__ a, TB* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = TB(a[i]);
}

template <typename T>
__global__ void axpby_kernel(T a, const T* x, T b, T* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

template <typename T>
__global__ void xpay_kernel(const T* __restrict__ x, T a, const T* y, T* z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = x[i] + a * y[i];
}

template <typename T>
__global__ void mul_kernel(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = a[i] * b[i];
}

// SplitMix64 (Steele, Lea & Flood 2014) at counter i + 1, top 53 bits mapped to [-1, 1).
template <typename T>
__global__ void splitmix_kernel(T* __restrict__ out, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    out[i] = T(2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
  }
}

template <typename T>
__global__ void sub_kernel(const T* __restrict__ b, const T* __restrict__ t, T* __restrict__ r, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - t[i];
}

// PREP: also write t = (constrained ? d : 0), the output vector of the next application of d prepared as
// prep_out would (t is read first at the same index, so the overwrite is safe).
template <typename T, int PREP>
__global__ void cheb_init_kernel(const T* __restrict__ b, T* __restrict__ t, const T* __restrict__ dinv,
                                 T* __restrict__ r, T* __restrict__ d, T* __restrict__ x, T inv_theta, bool x0_zero,
                                 long long n, Geom g, bool prep_x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T ri = x0_zero ? b[i] : b[i] - t[i];
    const T di = dinv[i] * ri * inv_theta;
    r[i] = ri;
    d[i] = di;
    const T xi = x0_zero ? di : x[i] + di;
    x[i] = xi;
    if constexpr (PREP > 0) t[i] = ((cmask_of<PREP>(g, i / PREP) >> (i % PREP)) & 1u) ? (prep_x ? xi : di) : T(0);
  }
}

template <typename T, int PREP>
__global__ void cheb_step_kernel(T* __restrict__ t, const T* __restrict__ dinv, T* __restrict__ r,
                                 T* __restrict__ d, T* __restrict__ x, T cd, T cr, long long n, Geom g, bool prep_x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T ri = r[i] - t[i];
    const T di = cd * d[i] + cr * dinv[i] * ri;
    r[i] = ri;
    d[i] = di;
    const T xi = x[i] + di;
    x[i] = xi;
    if constexpr (PREP > 0) t[i] = ((cmask_of<PREP>(g, i / PREP) >> (i % PREP)) & 1u) ? (prep_x ? xi : di) : T(0);
  }
}

// y += sign * (*alpha) x and z = x + (*beta) y with the coefficient read from device memory, so that an
// iteration's scalars never travel to the host.
template <typename T>
__global__ void axpy_dev_kernel(const double* __restrict__ alpha, double sign, const T* __restrict__ x, T* y,
                                long long n) {
  const T a = T(sign * alpha[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
template <typename T>
__global__ void xpay_dev_kernel(const T* __restrict__ x, const double* __restrict__ beta, const T* y, T* z, long long n) {
  const T b = T(beta[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = x[i] + b * y[i];
}

// Scalars of one CG step of the eigenvalue estimate, kept on the device. s = {rz, rz0, pq, rzn, alpha,
// beta, stopped, count}; hist = alpha[iters] followed by beta[iters].
__global__ void eig_alpha_kernel(double* s, double* hist, int it) {
  const bool stopped = s[6] != 0.0;
  const double alpha = stopped ? 0.0 : s[0] / s[2];
  s[4] = alpha;
  if (!stopped) hist[it] = alpha;
}
// Scalars of one preconditioned CG step, kept on the device (the batched solve). s = {rz, pq, alpha, rr,
// rzn, beta, tol, converged, not_spd}. op 0: alpha = rz / pq (0 and not_spd set when pq <= 0);
// op 1: converged = sqrt(rr) <= tol; op 2: beta = rzn / rz, rz = rzn. Once converged or not_spd is set it
// stays set and alpha = beta = 0: later iterations of a finished problem leave x and r unchanged.
__global__ void pcg_scalar_kernel(double* s, int op) {
  const bool finished = s[7] != 0.0 || s[8] != 0.0;
  if (op == 0) {
    const double pq = s[1];
    if (finished) {
      s[2] = 0.0;
    } else if (pq > 0.0) {
      s[2] = s[0] / pq;
    } else {
      s[2] = 0.0;
      s[8] = 1.0;
    }
  } else if (op == 1) {
    if (!finished && sqrt(s[3]) <= s[6]) s[7] = 1.0;
  } else {
    if (finished) {
      s[5] = 0.0;
    } else {
      s[5] = s[4] / s[0];
      s[0] = s[4];
    }
  }
}
__global__ void eig_beta_kernel(double* s, double* hist, int it, int iters) {
  if (s[6] != 0.0) {
    s[5] = 0.0;
    return;
  }
  const double beta = s[3] / s[0];
  hist[iters + it] = beta;
  s[7] = it + 1;
  s[5] = beta;
  s[0] = s[3];
  if (s[3] <= 1e-28 * s[1]) s[6] = 1.0;
}

// Deterministic two-stage reduction: each of DOT_BLOCKS blocks sums a fixed strided subset in a
// fixed tree order; one block then sums the partials in index order.
template <typename T>
__global__ void dot_partial_kernel(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                   double* __restrict__ partials) {
  __shared__ double sh[TPB];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)TPB + threadIdx.x; i < n; i += (long long)DOT_BLOCKS * TPB)
    s = fma((double)a[i], (double)b[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sh[TPB];
  double s = 0.0;
  for (int i = threadIdx.x; i < DOT_BLOCKS; i += TPB) s += partials[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

template <typename T, int DIM>
__global__ void sweep_kernel(const T* __restrict__ in, const T* __restrict__ in_minus, T* __restrict__ out,
                             T* __restrict__ prep, int Li0, int Li1, int Lo0, int Lo1, int Lo2, int axis,
                             const int* __restrict__ start, const T* __restrict__ w, int E, bool add, bool use_mask_in,
                             Geom gin, bool use_mask_out, Geom gout) {
  const long long n_out = (long long)Lo0 * Lo1 * (DIM == 3 ? Lo2 : 1) * DIM;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n_out;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % DIM);
    const long long nd = idx / DIM;
    int o[3] = {(int)(nd % Lo0), (int)((nd / Lo0) % Lo1), DIM == 3 ? (int)(nd / ((long long)Lo0 * Lo1)) : 0};
    const int oa = o[axis];
    const int s0 = start[oa];
    T acc = T(0);
    for (int e = 0; e < E; ++e) {
      o[axis] = s0 + e;
      const long long ni = o[0] + (long long)Li0 * (o[1] + (long long)Li1 * o[2]);
      T v = in[ni * DIM + c];
      if (in_minus) v = v - in_minus[ni * DIM + c];
      if (use_mask_in && ((node_cmask<DIM>(gin, o[0], o[1], o[2]) >> c) & 1u)) v = T(0);
      acc = fma(w[(long long)oa * E + e], v, acc);
    }
    o[axis] = oa;
    const bool masked = use_mask_out && ((node_cmask<DIM>(gout, o[0], o[1], o[2]) >> c) & 1u);
    if (masked) acc = T(0);
    const T v = add ? out[idx] + acc : acc;
    out[idx] = v;
    if (prep) prep[idx] = masked ? v : T(0);
  }
}

}  // namespace

template <typename T>
void launch_prep_out(const T* x, T* y, long long n_nodes, int dim, const Geom& g, cudaStream_t st) {
  if (dim == 2) prep_out_kernel<T, 2><<<grid_for(n_nodes), TPB, 0, st>>>(x, y, n_nodes, g);
  else prep_out_kernel<T, 3><<<grid_for(n_nodes), TPB, 0, st>>>(x, y, n_nodes, g);
}
template <typename T>
void launch_prep_out_list(const CellArgs<T>* list, int count, int dim, long long max_nodes, cudaStream_t st) {
  if (count <= 0) return;
  long long gx = (max_nodes + TPB - 1) / TPB;
  const long long cap = std::max<long long>(1, 152LL * 16 / count);  // about one wave over all problems
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  const dim3 grid((unsigned)gx, (unsigned)count);
  if (dim == 2) prep_out_list_kernel<T, 2><<<grid, TPB, 0, st>>>(list);
  else prep_out_list_kernel<T, 3><<<grid, TPB, 0, st>>>(list);
}
template <typename T>
void launch_zero_constrained(T* y, long long n_nodes, int dim, const Geom& g, cudaStream_t st) {
  if (dim == 2) set_constrained_kernel<T, 2><<<grid_for(n_nodes), TPB, 0, st>>>(y, n_nodes, g, T(0));
  else set_constrained_kernel<T, 3><<<grid_for(n_nodes), TPB, 0, st>>>(y, n_nodes, g, T(0));
}
template <typename T>
void launch_set_constrained_one(T* y, long long n_nodes, int dim, const Geom& g, cudaStream_t st) {
  if (dim == 2) set_constrained_kernel<T, 2><<<grid_for(n_nodes), TPB, 0, st>>>(y, n_nodes, g, T(1));
  else set_constrained_kernel<T, 3><<<grid_for(n_nodes), TPB, 0, st>>>(y, n_nodes, g, T(1));
}
template <typename T>
void launch_invert(const double* d, T* dinv, long long n, cudaStream_t st) {
  invert_kernel<T><<<grid_for(n), TPB, 0, st>>>(d, dinv, n);
}
template <typename TA, typename TB>
void launch_convert(const TA* a, TB* b, long long n, cudaStream_t st) {
  convert_kernel<TA, TB><<<grid_for(n), TPB, 0, st>>>(a, b, n);
}
template <typename T>
void launch_axpby(T a, const T* x, T b, T* y, long long n, cudaStream_t st) {
  axpby_kernel<T><<<grid_for(n), TPB, 0, st>>>(a, x, b, y, n);
}
template <typename T>
void launch_xpay(const T* x, T a, const T* y, T* z, long long n, cudaStream_t st) {
  xpay_kernel<T><<<grid_for(n), TPB, 0, st>>>(x, a, y, z, n);
}
template <typename T>
void launch_mul(const T* a, const T* b, T* z, long long n, cudaStream_t st) {
  mul_kernel<T><<<grid_for(n), TPB, 0, st>>>(a, b, z, n);
}
template <typename T>
void launch_splitmix(T* out, long long n, unsigned long long seed, cudaStream_t st) {
  splitmix_kernel<T><<<grid_for(n), TPB, 0, st>>>(out, n, seed);
}
template <typename T>
void launch_axpy_dev(const double* alpha, double sign, const T* x, T* y, long long n, cudaStream_t st) {
  axpy_dev_kernel<T><<<grid_for(n), TPB, 0, st>>>(alpha, sign, x, y, n);
}
template <typename T>
void launch_xpay_dev(const T* x, const double* beta, const T* y, T* z, long long n, cudaStream_t st) {
  xpay_dev_kernel<T><<<grid_for(n), TPB, 0, st>>>(x, beta, y, z, n);
}
void launch_pcg_scalar(double* s, int op, cudaStream_t st) { pcg_scalar_kernel<<<1, 1, 0, st>>>(s, op); }
void launch_eig_alpha(double* s, double* hist, int it, cudaStream_t st) { eig_alpha_kernel<<<1, 1, 0, st>>>(s, hist, it); }
void launch_eig_beta(double* s, double* hist, int it, int iters, cudaStream_t st) {
  eig_beta_kernel<<<1, 1, 0, st>>>(s, hist, it, iters);
}
template <typename T>
void launch_sub(const T* b, const T* t, T* r, long long n, cudaStream_t st) {
  sub_kernel<T><<<grid_for(n), TPB, 0, st>>>(b, t, r, n);
}
template <typename T>
void launch_cheb_init(const T* b, T* t, const T* dinv, T* r, T* d, T* x, T inv_theta, bool x0_zero, long long n,
                      const Geom* prep, int dim, cudaStream_t st, bool prep_x) {
  const Geom g = prep ? *prep : Geom{};
  if (!prep) cheb_init_kernel<T, 0><<<grid_for(n), TPB, 0, st>>>(b, t, dinv, r, d, x, inv_theta, x0_zero, n, g, prep_x);
  else if (dim == 2)
    cheb_init_kernel<T, 2><<<grid_for(n), TPB, 0, st>>>(b, t, dinv, r, d, x, inv_theta, x0_zero, n, g, prep_x);
  else cheb_init_kernel<T, 3><<<grid_for(n), TPB, 0, st>>>(b, t, dinv, r, d, x, inv_theta, x0_zero, n, g, prep_x);
}
template <typename T>
void launch_cheb_step(T* t, const T* dinv, T* r, T* d, T* x, T cd, T cr, long long n, const Geom* prep, int dim,
                      cudaStream_t st, bool prep_x) {
  const Geom g = prep ? *prep : Geom{};
  if (!prep) cheb_step_kernel<T, 0><<<grid_for(n), TPB, 0, st>>>(t, dinv, r, d, x, cd, cr, n, g, prep_x);
  else if (dim == 2) cheb_step_kernel<T, 2><<<grid_for(n), TPB, 0, st>>>(t, dinv, r, d, x, cd, cr, n, g, prep_x);
  else cheb_step_kernel<T, 3><<<grid_for(n), TPB, 0, st>>>(t, dinv, r, d, x, cd, cr, n, g, prep_x);
}
void launch_face_load(double* f, int dim, const Geom& g, int face, const FaceLoad& fl, cudaStream_t st) {
  const long long L = g.L;
  const long long nface = dim == 3 ? L * L : L;
  if (dim == 2) face_load_kernel<2><<<grid_for(nface), TPB, 0, st>>>(f, g, face / 2, face % 2, fl);
  else face_load_kernel<3><<<grid_for(nface), TPB, 0, st>>>(f, g, face / 2, face % 2, fl);
}
void launch_lift(const double* u, double* du0, double factor, const double* fv, long long n_nodes, int dim,
                 const Geom& g, cudaStream_t st) {
  if (dim == 2) lift_kernel<2><<<grid_for(n_nodes), TPB, 0, st>>>(u, du0, factor, fv, n_nodes, g);
  else lift_kernel<3><<<grid_for(n_nodes), TPB, 0, st>>>(u, du0, factor, fv, n_nodes, g);
}
template <typename T>
void launch_dot(const T* a, const T* b, long long n, double* partials, double* out, cudaStream_t st) {
  dot_partial_kernel<T><<<DOT_BLOCKS, TPB, 0, st>>>(a, b, n, partials);
  dot_final_kernel<<<1, TPB, 0, st>>>(partials, out);
}
template <typename T>
void launch_sweep(const T* in, T* out, int dim, const int Lin[3], const int Lout[3], int axis, const int* start,
                  const T* w, int E, bool add, const Geom* mask_in, const Geom* mask_out, cudaStream_t st,
                  const T* in_minus, T* prep) {
  long long n_out = (long long)Lout[0] * Lout[1] * (dim == 3 ? Lout[2] : 1) * dim;
  Geom gi = mask_in ? *mask_in : Geom{};
  Geom go = mask_out ? *mask_out : Geom{};
  if (dim == 2)
    sweep_kernel<T, 2><<<grid_for(n_out), TPB, 0, st>>>(in, in_minus, out, prep, Lin[0], Lin[1], Lout[0], Lout[1],
                                                        Lout[2], axis, start, w, E, add, mask_in != nullptr, gi,
                                                        mask_out != nullptr, go);
  else
    sweep_kernel<T, 3><<<grid_for(n_out), TPB, 0, st>>>(in, in_minus, out, prep, Lin[0], Lin[1], Lout[0], Lout[1],
                                                        Lout[2], axis, start, w, E, add, mask_in != nullptr, gi,
                                                        mask_out != nullptr, go);
}

#define HY_INST(T)                                                                                              \
  template void launch_prep_out<T>(const T*, T*, long long, int, const Geom&, cudaStream_t);                    \
  template void launch_zero_constrained<T>(T*, long long, int, const Geom&, cudaStream_t);                      \
  template void launch_set_constrained_one<T>(T*, long long, int, const Geom&, cudaStream_t);                   \
  template void launch_invert<T>(const double*, T*, long long, cudaStream_t);                                   \
  template void launch_axpby<T>(T, const T*, T, T*, long long, cudaStream_t);                                   \
  template void launch_xpay<T>(const T*, T, const T*, T*, long long, cudaStream_t);                             \
  template void launch_sub<T>(const T*, const T*, T*, long long, cudaStream_t);                                 \
  template void launch_mul<T>(const T*, const T*, T*, long long, cudaStream_t);                                 \
  template void launch_axpy_dev<T>(const double*, double, const T*, T*, long long, cudaStream_t);               \
  template void launch_xpay_dev<T>(const T*, const double*, const T*, T*, long long, cudaStream_t);             \
  template void launch_splitmix<T>(T*, long long, unsigned long long, cudaStream_t);                            \
  template void launch_cheb_init<T>(const T*, T*, const T*, T*, T*, T*, T, bool, long long, const Geom*, int,     \
                                    cudaStream_t, bool);                                                        \
  template void launch_cheb_step<T>(T*, const T*, T*, T*, T*, T, T, long long, const Geom*, int, cudaStream_t,     \
                                    bool);                                                                      \
  template void launch_dot<T>(const T*, const T*, long long, double*, double*, cudaStream_t);                   \
  template void launch_sweep<T>(const T*, T*, int, const int*, const int*, int, const int*, const T*, int, bool, \
                                const Geom*, const Geom*, cudaStream_t, const T*, T*);
HY_INST(double)
HY_INST(float)
#undef HY_INST
template void launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, cudaStream_t);

template void launch_prep_out_list<double>(const CellArgs<double>*, int, int, long long, cudaStream_t);
template void launch_prep_out_list<float>(const CellArgs<float>*, int, int, long long, cudaStream_t);
template void launch_prep_out_list<ff>(const CellArgs<ff>*, int, int, long long, cudaStream_t);
// One thread block waits on an mbarrier that nothing arrives on: the bounded wait has to give up by itself
// after limit_ns and flag ERRBIT_TIMEOUT. A check of the failure path that every bulk-copy wait takes.
__global__ void bounded_wait_check_kernel(unsigned* err, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0) atomicOr(err, ERRBIT_TIMEOUT);
}

void launch_bounded_wait_check(unsigned* err, unsigned long long limit_ns, cudaStream_t st) {
  bounded_wait_check_kernel<<<1, 32, 0, st>>>(err, limit_ns);
}

}  // namespace hy
