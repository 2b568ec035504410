// Exact coarsest-level solve (option; the paper's coarse solver is Chebyshev to a 1e-3 reduction,
// Sec. 7): the constrained coarse tangent is assembled as a dense FP64 matrix, inverted in place by
// Gauss-Jordan elimination (SPD, so no pivoting), and every V-cycle applies the inverse with one
// matrix-vector product. Worth it because the coarsest level is tiny (a few thousand dofs) while its
// Chebyshev solve needs hundreds of dependent, latency-bound applications per V-cycle.
#include "cell_kernels.cuh"
#include "launch.cuh"

namespace hy {
namespace {

// One block per cell, one thread per row (node a, component c) of the element matrix.
//   A_{ac,be} = sum_q W [ d_ce g_a.tau.g_b + c1/2 (d_ce g_a.g_b + g_{a,e} g_{b,c}) + c2 g_{a,c} g_{b,e} ]
// with g_a = F^{-T} Grad N_a: the geometric and material parts of Eq. algebraic_tangent with the
// neo-Hooke action of Eq. simplified_action (c1 = 2(mu - 2 lambda ln J), c2 = 2 lambda, W = w_q h^d).
template <int DIM, int N>
__global__ void assemble_dense_kernel(const CellArgs<double> a, double* __restrict__ Aout, long long ndof) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int NS = nsym(DIM);
  constexpr int NR = NPT * DIM;
  __shared__ double S[MAXN][MAXN], D[MAXN][MAXN], Sd[MAXN][MAXN], W[NPT];
  __shared__ double u0[DIM][NPT], u1[DIM][NPT];
  __shared__ double Mq[DIM * DIM][NPT], tq[NS][NPT], c1q[NPT], c2q[NPT];
  __shared__ long long gdof[NR];
  __shared__ unsigned char cons[NR];
  __shared__ double mu_s, lam_s;
  const int t = threadIdx.x;
  const int cell = blockIdx.x;
  for (int i = t; i < MAXN * MAXN; i += blockDim.x) {  // blocks can be smaller than the tables (Q1, 2D)
    S[i / MAXN][i % MAXN] = a.b.S[i / MAXN][i % MAXN];
    D[i / MAXN][i % MAXN] = a.b.D[i / MAXN][i % MAXN];
    Sd[i / MAXN][i % MAXN] = a.b.Sd[i / MAXN][i % MAXN];
  }
  if (t == 0) {
    const int id = a.mat[cell];
    mu_s = a.mt.mu[id];
    lam_s = a.mt.lam[id];
  }
  int pc[3] = {0, 0, 0};
  if (t < NPT) {
    pc[0] = t % N;
    pc[1] = (t / N) % N;
    pc[2] = DIM == 3 ? t / (N * N) : 0;
    double w = a.b.w[pc[0]] * a.b.w[pc[1]];
    double hd = a.g.h * a.g.h;
    if (DIM == 3) {
      w *= a.b.w[pc[2]];
      hd *= a.g.h;
    }
    W[t] = w * hd;
    const int m = a.g.m, K = N - 1;
    const int c0 = cell % m, c1 = (cell / m) % m, c2 = DIM == 3 ? cell / (m * m) : 0;
    const int i0 = K * c0 + pc[0], i1 = K * c1 + pc[1], i2 = K * c2 + pc[2];
    const long long node = i0 + (long long)a.g.L * (i1 + (DIM == 3 ? (long long)a.g.L * i2 : 0));
    const uint32_t cm = node_cmask<DIM>(a.g, i0, i1, i2);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      u0[c][t] = a.u64[node * DIM + c];
      gdof[t * DIM + c] = node * DIM + c;
      cons[t * DIM + c] = (cm >> c) & 1u;
    }
  }
  __syncthreads();
  // forward sweeps of the displacement to the Gauss points (threads t < NPT compute)
  double (*src)[NPT] = u0;
  double (*dst)[NPT] = u1;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    if (t < NPT) {
      const int stride = ax == 0 ? 1 : (ax == 1 ? N : N * N);
      const int base = t - pc[ax] * stride;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) v = fma(S[pc[ax]][j], src[c][base + j * stride], v);
        dst[c][t] = v;
      }
    }
    __syncthreads();
    double (*tmp)[NPT] = src;
    src = dst;
    dst = tmp;
  }
  if (t < NPT) {
    double F[DIM][DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int J = 0; J < DIM; ++J) {
        const int stride = J == 0 ? 1 : (J == 1 ? N : N * N);
        const int base = t - pc[J] * stride;
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) v = fma(D[pc[J]][j], src[c][base + j * stride], v);
        F[c][J] = (c == J ? 1.0 : 0.0) + v * a.g.inv_h;
      }
    double M[DIM][DIM], tau[NS], c1, c2;
    const double J = neo_hooke_state<DIM>(F, mu_s, lam_s, W[t], a.g.inv_h, false, 0.0, M, tau, c1, c2);
    if (!(J > 0.0)) atomicOr(a.err, J != J ? ERRBIT_NAN : ERRBIT_JNEG);
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) Mq[i][t] = M[i / DIM][i % DIM];
#pragma unroll
    for (int i = 0; i < NS; ++i) tq[i][t] = tau[i];
    c1q[t] = c1;
    c2q[t] = c2;
  }
  __syncthreads();
  if (t >= NR || cons[t]) return;
  const int an = t / DIM, c = t % DIM;
  const int apc[3] = {an % N, (an / N) % N, DIM == 3 ? an / (N * N) : 0};
  for (int col = 0; col < NR; ++col) {
    if (cons[col]) continue;
    const int bn = col / DIM, e = col % DIM;
    const int bpc[3] = {bn % N, (bn / N) % N, DIM == 3 ? bn / (N * N) : 0};
    double acc = 0.0;
    for (int q = 0; q < NPT; ++q) {
      const int qc[3] = {q % N, (q / N) % N, DIM == 3 ? q / (N * N) : 0};
      double gra[DIM], grb[DIM];  // d N / d xi at q
#pragma unroll
      for (int J = 0; J < DIM; ++J) {
        double va = 1.0, vb = 1.0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          va *= (i == J ? Sd : S)[qc[i]][apc[i]];
          vb *= (i == J ? Sd : S)[qc[i]][bpc[i]];
        }
        gra[J] = va;
        grb[J] = vb;
      }
      double ga[DIM], gb[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int J = 0; J < DIM; ++J) {
          sa = fma(gra[J], Mq[J * DIM + j][q], sa);
          sb = fma(grb[J], Mq[J * DIM + j][q], sb);
        }
        ga[j] = sa;
        gb[j] = sb;
      }
      double v = 0.0;
      if (c == e) {
        double geo = 0.0, dotab = 0.0;
#pragma unroll
        for (int al = 0; al < NS; ++al) {
          const int i = vi<DIM>(al), j = vj<DIM>(al);
          geo = fma(tq[al][q], (i == j) ? ga[i] * gb[i] : ga[i] * gb[j] + ga[j] * gb[i], geo);
        }
#pragma unroll
        for (int j = 0; j < DIM; ++j) dotab = fma(ga[j], gb[j], dotab);
        v = geo + 0.5 * c1q[q] * dotab;
      }
      v = fma(0.5 * c1q[q], ga[e] * gb[c], v);
      v = fma(c2q[q], ga[c] * gb[e], v);
      acc += v;
    }
    atomicAdd(&Aout[gdof[t] * ndof + gdof[col]], acc);
  }
}

template <int DIM, int N>
void launch_assemble(const CellArgs<double>& a, double* A, long long ndof, cudaStream_t st) {
  assemble_dense_kernel<DIM, N><<<a.g.ncells, ipow(N, DIM) * DIM, 0, st>>>(a, A, ndof);
}

// Constrained dofs: identity rows and columns (the matrix is zero there before this).
template <int DIM>
__global__ void dense_constrained_identity(double* __restrict__ A, long long n_nodes, long long ndof, Geom g) {
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n_nodes; nd += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)(nd % g.L), i1 = (int)((nd / g.L) % g.L), i2 = DIM == 3 ? (int)(nd / ((long long)g.L * g.L)) : 0;
    const uint32_t cm = node_cmask<DIM>(g, i0, i1, i2);
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if ((cm >> c) & 1u) A[(nd * DIM + c) * ndof + nd * DIM + c] = 1.0;
  }
}

// Gauss-Jordan step k (in place): R = row k / pivot (R_k = 1 / pivot), C = column k.
__global__ void gj_prep(const double* __restrict__ A, long long n, long long k, double* __restrict__ R,
                        double* __restrict__ C, unsigned* err) {
  const double piv = A[k * n + k];
  if (blockIdx.x == 0 && threadIdx.x == 0 && !(piv > 0.0)) atomicOr(err, ERRBIT_NONSPD);
  const double inv = 1.0 / piv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    C[i] = A[i * n + k];
    R[i] = (i == k ? 1.0 : A[k * n + i]) * inv;
  }
}
// A_ij <- A_ij - C_i R_j for i != k (column k starts from zero), row k <- R.
__global__ void gj_update(double* __restrict__ A, long long n, long long k, const double* __restrict__ R,
                          const double* __restrict__ C) {
  const long long total = n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx / n, j = idx % n;
    if (i == k) A[idx] = R[j];
    else A[idx] = (j == k ? 0.0 : A[idx]) - C[i] * R[j];
  }
}

// x = A b, one warp per row, fixed summation order.
__global__ void dense_gemv(const double* __restrict__ A, const double* __restrict__ b, double* __restrict__ x,
                           long long n) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (warp >= n) return;
  const double* row = A + warp * n;
  double s = 0.0;
  for (long long j = lane; j < n; j += 32) s = fma(row[j], b[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[warp] = s;
}

}  // namespace

void launch_assemble_dense(int dim, int n, const CellArgs<double>& a, double* A, long long ndof, cudaStream_t st) {
  using Fn = void (*)(const CellArgs<double>&, double*, long long, cudaStream_t);
  static const Fn t2[4] = {launch_assemble<2, 2>, launch_assemble<2, 3>, launch_assemble<2, 4>, launch_assemble<2, 5>};
  static const Fn t3[4] = {launch_assemble<3, 2>, launch_assemble<3, 3>, launch_assemble<3, 4>, launch_assemble<3, 5>};
  (dim == 2 ? t2 : t3)[n - 2](a, A, ndof, st);
}

void launch_dense_constrained_identity(double* A, long long n_nodes, long long ndof, int dim, const Geom& g,
                                       cudaStream_t st) {
  const int grid = (int)std::min<long long>((n_nodes + 255) / 256, 1024);
  if (dim == 2) dense_constrained_identity<2><<<grid, 256, 0, st>>>(A, n_nodes, ndof, g);
  else dense_constrained_identity<3><<<grid, 256, 0, st>>>(A, n_nodes, ndof, g);
}

void launch_gj_step(double* A, long long n, long long k, double* R, double* C, unsigned* err, cudaStream_t st) {
  gj_prep<<<(int)std::min<long long>((n + 255) / 256, 64), 256, 0, st>>>(A, n, k, R, C, err);
  gj_update<<<(int)std::min<long long>((n * n + 255) / 256, 152LL * 16), 256, 0, st>>>(A, n, k, R, C);
}

void launch_dense_gemv(const double* A, const double* b, double* x, long long n, cudaStream_t st) {
  const long long threads = n * 32;
  dense_gemv<<<(int)((threads + 255) / 256), 256, 0, st>>>(A, b, x, n);
}

}  // namespace hy
