// Exact coarsest-level solve (option; the paper's coarse solver is Chebyshev to a 1e-3 reduction,
// Sec. 7): the coarse tangent restricted to the free dofs is assembled as a dense FP64 matrix, inverted by
// Gauss-Jordan elimination (SPD, so no pivoting), and every V-cycle applies the inverse with one
// matrix-vector product. Worth it because the coarsest level is tiny (a few thousand dofs) while its
// Chebyshev solve needs hundreds of dependent, latency-bound applications per V-cycle.
#include "cell_kernels.cuh"
#include "launch.cuh"

namespace hy {
namespace {

// One block per cell; the work items are the cell's node pairs (a, b), each forming a DIM x DIM block of
// the element matrix:
//   A_{ac,be} = sum_q W [ d_ce g_a.tau.g_b + c1/2 (d_ce g_a.g_b + g_{a,e} g_{b,c}) + c2 g_{a,c} g_{b,e} ]
// with g_a = F^{-T} Grad N_a: the geometric and material parts of Eq. algebraic_tangent with the
// neo-Hooke action of Eq. simplified_action (c1 = 2(mu - 2 lambda ln J), c2 = 2 lambda, W = w_q h^d).
// CH = 0: one block per cell, g_a(q) of every node of the cell in shared memory. CH > 0 (elements whose
// table NPT^2 DIM doubles exceeds shared memory: Q4 in 3D): the block (cell, blockIdx.y) holds g_a(q) for the
// CH nodes a of its chunk only; thread b forms g_b(q) itself and accumulates the pairs (a, b) of the chunk.
template <int DIM, int N, int CH>
__global__ void assemble_dense_kernel(const CellArgs<double> a, double* __restrict__ Aout, long long nfree,
                                      const int* __restrict__ cidx) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int NS = nsym(DIM);
  constexpr int NR = NPT * DIM;
  __shared__ double S[MAXN][MAXN], D[MAXN][MAXN], Sd[MAXN][MAXN], W[NPT];
  __shared__ double u0[DIM][NPT], u1[DIM][NPT];
  __shared__ double x0[DIM][NPT], x1[DIM][NPT];  // nodal coordinates of a curved geometry
  const bool curved = a.X64 != nullptr;
  __shared__ double Mq[DIM * DIM][NPT], tq[NS][NPT], c1q[NPT], c2q[NPT];
  __shared__ long long gdof[NR];
  __shared__ unsigned char cons[NR];
  extern __shared__ double Gq[];  // [NPT or CH][NPT][DIM]
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
      x0[c][t] = curved ? a.X64[node * DIM + c] : 0.0;
      gdof[t * DIM + c] = node * DIM + c;
      cons[t * DIM + c] = (cm >> c) & 1u;
    }
  }
  __syncthreads();
  // forward sweeps of the displacement to the Gauss points (threads t < NPT compute)
  double (*src)[NPT] = u0;
  double (*dst)[NPT] = u1;
  double (*xs)[NPT] = x0;
  double (*xd)[NPT] = x1;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    if (t < NPT) {
      const int stride = ax == 0 ? 1 : (ax == 1 ? N : N * N);
      const int base = t - pc[ax] * stride;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double v = 0.0, w = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          v = fma(S[pc[ax]][j], src[c][base + j * stride], v);
          if (curved) w = fma(S[pc[ax]][j], xs[c][base + j * stride], w);
        }
        dst[c][t] = v;
        xd[c][t] = w;
      }
    }
    __syncthreads();
    double (*tmp)[NPT] = src;
    src = dst;
    dst = tmp;
    tmp = xs;
    xs = xd;
    xd = tmp;
  }
  if (t < NPT) {
    double F[DIM][DIM], Gu[DIM][DIM], GX[DIM][DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int J = 0; J < DIM; ++J) {
        const int stride = J == 0 ? 1 : (J == 1 ? N : N * N);
        const int base = t - pc[J] * stride;
        double v = 0.0, w = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          v = fma(D[pc[J]][j], src[c][base + j * stride], v);
          if (curved) w = fma(D[pc[J]][j], xs[c][base + j * stride], w);
        }
        Gu[c][J] = v;
        GX[c][J] = w;
        F[c][J] = (c == J ? 1.0 : 0.0) + v * a.g.inv_h;
      }
    double invJ[DIM][DIM], Wq = W[t];
    if (curved) {  // isoparametric map: invJ = (dX/dxi)^{-1}, weight w_q det(dX/dxi)
      double det;
      if (DIM == 3) {
        invJ[0][0] = GX[1][1] * GX[2][2] - GX[1][2] * GX[2][1];
        invJ[0][1] = GX[0][2] * GX[2][1] - GX[0][1] * GX[2][2];
        invJ[0][2] = GX[0][1] * GX[1][2] - GX[0][2] * GX[1][1];
        invJ[1][0] = GX[1][2] * GX[2][0] - GX[1][0] * GX[2][2];
        invJ[1][1] = GX[0][0] * GX[2][2] - GX[0][2] * GX[2][0];
        invJ[1][2] = GX[0][2] * GX[1][0] - GX[0][0] * GX[1][2];
        invJ[2][0] = GX[1][0] * GX[2][1] - GX[1][1] * GX[2][0];
        invJ[2][1] = GX[0][1] * GX[2][0] - GX[0][0] * GX[2][1];
        invJ[2][2] = GX[0][0] * GX[1][1] - GX[0][1] * GX[1][0];
        det = GX[0][0] * invJ[0][0] + GX[0][1] * invJ[1][0] + GX[0][2] * invJ[2][0];
      } else {
        invJ[0][0] = GX[1][1];
        invJ[0][1] = -GX[0][1];
        invJ[1][0] = -GX[1][0];
        invJ[1][1] = GX[0][0];
        det = GX[0][0] * GX[1][1] - GX[0][1] * GX[1][0];
      }
      if (!(det > 0.0)) atomicOr(a.err, ERRBIT_JNEG);
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) invJ[i][j] /= det;
      double w = a.b.w[pc[0]] * a.b.w[pc[1]];
      if (DIM == 3) w *= a.b.w[pc[2]];
      Wq = w * det;
      deformation_curved<DIM>(Gu, invJ, F);
    }
    double M[DIM][DIM], tau[NS], c1, c2;
    const double J = neo_hooke_state<DIM>(F, mu_s, lam_s, a.mt.law, Wq, curved ? 1.0 : a.g.inv_h, false, 0.0, M, tau,
                                          c1, c2);
    if (curved) premultiply<DIM>(invJ, M);
    if (!(J > 0.0)) atomicOr(a.err, J != J ? ERRBIT_NAN : ERRBIT_JNEG);
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) Mq[i][t] = M[i / DIM][i % DIM];
#pragma unroll
    for (int i = 0; i < NS; ++i) tq[i][t] = tau[i];
    c1q[t] = c1;
    c2q[t] = c2;
  }
  __syncthreads();
  // g_a(q) = F^{-T} Grad N_a at every (node, point) pair of the cell (of the chunk), once, in shared memory
  constexpr int NA = CH > 0 ? CH : NPT;  // nodes a in the table
  const int a0 = CH > 0 ? (int)blockIdx.y * CH : 0;
  for (int item = t; item < NA * NPT; item += blockDim.x) {
    const int al = item / NPT, q = item % NPT;
    const int an = a0 + al;
    if (an >= NPT) continue;
    const int apc[3] = {an % N, (an / N) % N, DIM == 3 ? an / (N * N) : 0};
    const int qc[3] = {q % N, (q / N) % N, DIM == 3 ? q / (N * N) : 0};
    double gr[DIM];
#pragma unroll
    for (int J = 0; J < DIM; ++J) {
      double v = 1.0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) v *= (i == J ? Sd : S)[qc[i]][apc[i]];
      gr[J] = v;
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      double sa = 0.0;
#pragma unroll
      for (int J = 0; J < DIM; ++J) sa = fma(gr[J], Mq[J * DIM + j][q], sa);
      Gq[(al * NPT + q) * DIM + j] = sa;
    }
  }
  __syncthreads();
  if constexpr (CH == 0) {
    // one node pair (a, b) per work item: its DIM x DIM block of the element matrix,
    //   A_{ac,be} = sum_q [ d_ce g_b.(tau + c1/2 I).g_a + c1/2 g_{a,e} g_{b,c} + c2 g_{a,c} g_{b,e} ].
    // Only the upper triangle of the free-dof matrix is assembled (the Gauss-Jordan passes read nothing else):
    // the lattice numbers a cell's nodes in the order of its local nodes, so the pairs with a > b lie below
    // the diagonal and are skipped, and those with a = b keep c <= e.
    for (int item = t; item < NPT * NPT; item += blockDim.x) {
      const int an = item / NPT, bn = item % NPT;
      if (an > bn) continue;
      double acc[DIM][DIM];
  #pragma unroll
      for (int c = 0; c < DIM; ++c)
  #pragma unroll
        for (int e = 0; e < DIM; ++e) acc[c][e] = 0.0;
      for (int q = 0; q < NPT; ++q) {
        double ga[DIM], gb[DIM];
  #pragma unroll
        for (int j = 0; j < DIM; ++j) {
          ga[j] = Gq[(an * NPT + q) * DIM + j];
          gb[j] = Gq[(bn * NPT + q) * DIM + j];
        }
        const double hc1 = 0.5 * c1q[q], c2 = c2q[q];
        double geo = 0.0, dotab = 0.0;
  #pragma unroll
        for (int al = 0; al < NS; ++al) {
          const int i = vi<DIM>(al), j = vj<DIM>(al);
          geo = fma(tq[al][q], (i == j) ? ga[i] * gb[i] : ga[i] * gb[j] + ga[j] * gb[i], geo);
        }
  #pragma unroll
        for (int j = 0; j < DIM; ++j) dotab = fma(ga[j], gb[j], dotab);
        const double sdiag = fma(hc1, dotab, geo);
  #pragma unroll
        for (int c = 0; c < DIM; ++c)
  #pragma unroll
          for (int e = 0; e < DIM; ++e) {
            double v = fma(hc1, ga[e] * gb[c], c == e ? sdiag : 0.0);
            acc[c][e] += fma(c2, ga[c] * gb[e], v);
          }
      }
  #pragma unroll
      for (int c = 0; c < DIM; ++c)
  #pragma unroll
        for (int e = 0; e < DIM; ++e) {
          const int row = an * DIM + c, col = bn * DIM + e;
          if (cons[row] || cons[col] || (an == bn && c > e)) continue;
          atomicAdd(&Aout[(long long)cidx[gdof[row]] * nfree + cidx[gdof[col]]], acc[c][e]);
        }
    }
  } else {
    // thread b: g_b(q) from the tables and M, then the pairs (a, b), a of the chunk, a <= b
    const int bn = t;
    if (bn < NPT) {
      const int bpc[3] = {bn % N, (bn / N) % N, DIM == 3 ? bn / (N * N) : 0};
      double acc[CH][DIM][DIM];
#pragma unroll
      for (int al = 0; al < CH; ++al)
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int e = 0; e < DIM; ++e) acc[al][c][e] = 0.0;
      for (int q = 0; q < NPT; ++q) {
        const int qc[3] = {q % N, (q / N) % N, DIM == 3 ? q / (N * N) : 0};
        double gr[DIM], gb[DIM];
#pragma unroll
        for (int J = 0; J < DIM; ++J) {
          double v = 1.0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) v *= (i == J ? Sd : S)[qc[i]][bpc[i]];
          gr[J] = v;
        }
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          double sb = 0.0;
#pragma unroll
          for (int J = 0; J < DIM; ++J) sb = fma(gr[J], Mq[J * DIM + j][q], sb);
          gb[j] = sb;
        }
        const double hc1 = 0.5 * c1q[q], c2 = c2q[q];
#pragma unroll
        for (int al = 0; al < CH; ++al) {
          if (a0 + al > bn) continue;  // below the diagonal (or past the last node)
          double ga[DIM];
#pragma unroll
          for (int j = 0; j < DIM; ++j) ga[j] = Gq[(al * NPT + q) * DIM + j];
          double geo = 0.0, dotab = 0.0;
#pragma unroll
          for (int be = 0; be < NS; ++be) {
            const int i = vi<DIM>(be), j = vj<DIM>(be);
            geo = fma(tq[be][q], (i == j) ? ga[i] * gb[i] : ga[i] * gb[j] + ga[j] * gb[i], geo);
          }
#pragma unroll
          for (int j = 0; j < DIM; ++j) dotab = fma(ga[j], gb[j], dotab);
          const double sdiag = fma(hc1, dotab, geo);
#pragma unroll
          for (int c = 0; c < DIM; ++c)
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
              double v = fma(hc1, ga[e] * gb[c], c == e ? sdiag : 0.0);
              acc[al][c][e] += fma(c2, ga[c] * gb[e], v);
            }
        }
      }
#pragma unroll
      for (int al = 0; al < CH; ++al) {
        const int an = a0 + al;
        if (an > bn) continue;
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int e = 0; e < DIM; ++e) {
            const int row = an * DIM + c, col = bn * DIM + e;
            if (cons[row] || cons[col] || (an == bn && c > e)) continue;
            atomicAdd(&Aout[(long long)cidx[gdof[row]] * nfree + cidx[gdof[col]]], acc[al][c][e]);
          }
      }
    }
  }
}

template <int DIM, int N>
void launch_assemble(const CellArgs<double>& a, double* A, long long nfree, const int* cidx, cudaStream_t st) {
  constexpr int NPT = ipow(N, DIM);
  constexpr size_t full = sizeof(double) * NPT * NPT * DIM;  // the whole table: 375 KB for Q4 3D
  if constexpr (full <= 160 * 1024) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(assemble_dense_kernel<DIM, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)full);
      attr = true;
    }
    const int threads = NPT * DIM < 256 ? 256 : ((NPT * DIM + 31) / 32) * 32;
    assemble_dense_kernel<DIM, N, 0><<<a.g.ncells, threads, full, st>>>(a, A, nfree, cidx);
  } else {
    constexpr int CH = 5;
    constexpr size_t dyn = sizeof(double) * CH * NPT * DIM;
    const dim3 grid((unsigned)a.g.ncells, (unsigned)((NPT + CH - 1) / CH));
    assemble_dense_kernel<DIM, N, CH><<<grid, ((NPT + 31) / 32) * 32, dyn, st>>>(a, A, nfree, cidx);
  }
}

// x = A b on the free dofs (one warp per row, fixed summation order); b and x are full level vectors
// indexed through free_idx, whose constrained entries stay zero.
__global__ void dense_gemv(const double* __restrict__ A, const double* __restrict__ b, double* __restrict__ x,
                           long long n, const int* __restrict__ free_idx) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (warp >= n) return;
  const double* row = A + warp * n;
  double s = 0.0;
  for (long long j = lane; j < n; j += 32) s = fma(row[j], b[free_idx[j]], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[free_idx[warp]] = s;
}

}  // namespace

void launch_assemble_dense(int dim, int n, const CellArgs<double>& a, double* A, long long nfree, const int* cidx,
                           cudaStream_t st) {
  using Fn = void (*)(const CellArgs<double>&, double*, long long, const int*, cudaStream_t);
  static const Fn t2[4] = {launch_assemble<2, 2>, launch_assemble<2, 3>, launch_assemble<2, 4>, launch_assemble<2, 5>};
  static const Fn t3[4] = {launch_assemble<3, 2>, launch_assemble<3, 3>, launch_assemble<3, 4>, launch_assemble<3, 5>};
  (dim == 2 ? t2 : t3)[n - 2](a, A, nfree, cidx, st);
}

// ---- blocked Gauss-Jordan: GJB pivots per pass ------------------------------------------------------
// For the pivot block K = [k0, k0 + b) of A (old) the pass writes B (new):
//   B_KK = W = A_KK^{-1},  B_Kj = (W A_K:)_j = Y_j,  B_iK = -(A_iK W) = -X_i,  B_ij = A_ij - A_iK Y_j,
// the block form of b consecutive single-pivot steps; every element of A is read and written once per b
// pivots instead of once per pivot. The element type E is double, or double-float (ff: the same passes on
// the FP32 pipe, about 48 significant bits, the reciprocal of each pivot taken in FP64).
// Symmetry: A is SPD, and after any number of passes an entry (i, j) equals (j, i) when i and j are both
// eliminated (i, j < k0) or both not, and -(j, i) when exactly one is (the eliminated block holds the
// inverse of the leading block, the rest its Schur complement, the cross blocks are negatives of each
// other's transposes). So every pass reads and writes the upper triangle only, which halves the update, and
// the final inverse (all eliminated: symmetric) is mirrored once.
namespace {
constexpr int GJB = 32;

// Entry (p, q) of the current matrix from its upper triangle (before the pass over [k0, k0 + b)).
template <typename E>
__device__ __forceinline__ E sym_get(const E* __restrict__ A, int n, int k0, int p, int q) {
  if (p <= q) return A[(long long)p * n + q];
  const E v = A[(long long)q * n + p];
  return ((p < k0) != (q < k0)) ? -v : v;
}

__device__ __forceinline__ double gj_recip(double p) { return 1.0 / p; }
__device__ __forceinline__ ff gj_recip(ff p) { return rcp_rn(p); }
__device__ __forceinline__ bool gj_positive(double p) { return p > 0.0; }
__device__ __forceinline__ bool gj_positive(ff p) { return p.hi > 0.f; }

// W = A_KK^{-1} by single-pivot Gauss-Jordan on the b x b block in shared memory (one block of 256
// threads); flags a pivot <= 0. The pivot's reciprocal (an FP64 operation, on a pipe of 2 lanes per clock
// per SM) is taken by the first warp alone, which also forms the pivot row and column; then every thread
// updates the four entries (i, j), i = t / 32 + 8 r, j = t mod 32, of the GJB x GJB index space (no integer
// division: this loop is the sequential chain of the whole inversion).
template <typename E>
__global__ void __launch_bounds__(256) gjb_diag(const E* __restrict__ A, int n, int k0, int b, E* __restrict__ W,
                                                unsigned* err) {
  __shared__ E w[GJB][GJB + 1];
  __shared__ E rk[GJB], ck[GJB];
  static_assert(GJB == 32, "one warp forms a pivot row; a thread's column is its lane");
  const int t = threadIdx.x;
  const int j = t & 31, i0 = t >> 5;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + 8 * r;
    if (i < b && j < b) w[i][j] = sym_get(A, n, k0, k0 + i, k0 + j);
  }
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    if (t < 32) {
      const E p = w[k][k];
      if (t == 0 && !gj_positive(p)) atomicOr(err, ERRBIT_NONSPD);
      const E ip = gj_recip(p);
      if (t < b) {
        rk[t] = (t == k ? E(1) : w[k][t]) * ip;
        ck[t] = w[t][k];
      }
    }
    __syncthreads();
    if (j < b) {
      const E rkj = rk[j];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + 8 * r;
        if (i < b) w[i][j] = (i == k) ? rkj : (j == k ? E(0) : w[i][j]) - ck[i] * rkj;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + 8 * r;
    if (i < b && j < b) W[i * b + j] = w[i][j];
  }
}

// Y = W A_K: (b x n) and X = A_:K W (n x b). Thread (r, jy) of a 32 x 8 block computes Y_rj and X_jr for
// the column / row j = 8 blockIdx.x + jy; the block's 8 columns of A_K: and rows of A_:K are staged first.
template <typename E>
__global__ void __launch_bounds__(256) gjb_panels(const E* __restrict__ A, int n, int k0, int b,
                                                  const E* __restrict__ W, E* __restrict__ Y, E* __restrict__ X) {
  __shared__ E w[GJB][GJB + 1];
  __shared__ E colv[8][GJB + 1], rowv[8][GJB + 1];
  const int r = threadIdx.x, jy = threadIdx.y, t = jy * GJB + r;
  for (int idx = t; idx < b * b; idx += 256) w[idx / b][idx % b] = W[idx];
  const int j = blockIdx.x * 8 + jy;
  const bool inb = j < n && r < b;
  colv[jy][r] = inb ? sym_get(A, n, k0, k0 + r, j) : E(0);  // A_Kj
  rowv[jy][r] = inb ? sym_get(A, n, k0, j, k0 + r) : E(0);  // A_jK
  __syncthreads();
  if (!inb) return;
  E y = E(0), x = E(0);
  for (int m = 0; m < b; ++m) {
    y = fma(w[r][m], colv[jy][m], y);
    x = fma(rowv[jy][m], w[m][r], x);
  }
  Y[(long long)r * n + j] = y;
  X[(long long)j * b + r] = x;
}

// Accumulator of the update's dot products. FP64: a fused multiply-add chain. Double-float: the dot product
// of Ogita, Rump and Oishi ("Accurate sum and dot product", 2005, Dot2) with double-word operands -- the
// leading product split exactly by FMA, the leading sums by TwoSum, all error terms (and the cross products
// of the low words) gathered in one float -- normalised once at the end: 12 FP32 operations per term instead
// of the 15 of a double-float multiply-add, the same order of accuracy for the 32 terms of a pass.
template <typename E> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<ff> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(ff x, ff y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ ff value() const { return two_sum(hi, lo); }  // |lo| may exceed |hi| after cancellation
};

// B_ij = A_ij - sum_m A_im Y_mj (i, j outside K); rows K take Y (W on the diagonal block), columns K
// take -X. 64 x 64 output tile per block, 4 x 4 per thread, the A_:K and Y panels staged in shared memory.
template <typename E>
__global__ void __launch_bounds__(256) gjb_update(const E* __restrict__ A, E* __restrict__ B, int n, int k0, int b,
                                                  const E* __restrict__ W, const E* __restrict__ Y,
                                                  const E* __restrict__ X) {
  __shared__ E sA[64][GJB + 1];
  __shared__ E sY[GJB][64 + 1];
  if (blockIdx.x < blockIdx.y) return;  // upper triangle of tiles only
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int t = threadIdx.x;
  // A_iK of the tile's rows: stored in row i where i < k0 (consecutive threads take consecutive m), and as
  // row K's entries (A_Ki, the same or the negated value) where i >= k0 (consecutive threads take consecutive i)
  const bool rows_eliminated = i0 + 64 <= k0;
  for (int idx = t; idx < 64 * GJB; idx += 256) {
    const int r = rows_eliminated ? idx / GJB : idx % 64, m = rows_eliminated ? idx % GJB : idx / 64;
    const int i = i0 + r;
    sA[r][m] = (i < n && m < b) ? sym_get(A, n, k0, i, k0 + m) : E(0);
  }
  for (int idx = t; idx < 64 * GJB; idx += 256) {
    const int mm = idx / 64, c = idx % 64;
    const int j = j0 + c;
    sY[mm][c] = (j < n && mm < b) ? Y[(long long)mm * n + j] : E(0);
  }
  __syncthreads();
  const int tr = (t / 16) * 4, tc = (t % 16) * 4;
  DotAcc<E> acc[4][4];
  for (int m = 0; m < b; ++m) {
    E av[4], yv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = sA[tr + a][m];
#pragma unroll
    for (int c = 0; c < 4; ++c) yv[c] = sY[m][tc + c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c].add(av[a], yv[c]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + tr + a;
    if (i >= n) continue;
    const bool iK = i >= k0 && i < k0 + b;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tc + c;
      if (j >= n || j < i) continue;  // the upper triangle
      const bool jK = j >= k0 && j < k0 + b;
      E v;
      if (iK) v = jK ? W[(i - k0) * b + (j - k0)] : Y[(long long)(i - k0) * n + j];
      else v = jK ? -X[(long long)i * b + (j - k0)] : A[(long long)i * n + j] - acc[a][c].value();
      B[(long long)i * n + j] = v;
    }
  }
}

// lower triangle <- upper triangle (the symmetric inverse after the last pass)
template <typename E>
__global__ void mirror_lower(E* A, int n) {
  const long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (i > j) A[idx] = A[(long long)j * n + i];
  }
}

template <typename E>
E* gj_passes(E* A, E* B, long long n, E* work, unsigned* err, cudaStream_t st) {
  E* W = work;
  E* Y = W + GJB * GJB;
  E* X = Y + (size_t)GJB * n;
  const dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64));
  for (long long k0 = 0; k0 < n; k0 += GJB) {
    const int b = (int)std::min<long long>(GJB, n - k0);
    gjb_diag<E><<<1, 256, 0, st>>>(A, (int)n, (int)k0, b, W, err);
    gjb_panels<E><<<(unsigned)((n + 7) / 8), dim3(GJB, 8), 0, st>>>(A, (int)n, (int)k0, b, W, Y, X);
    gjb_update<E><<<grid, 256, 0, st>>>(A, B, (int)n, (int)k0, b, W, Y, X);
    std::swap(A, B);
  }
  mirror_lower<E><<<(int)std::min<long long>((n * n + 255) / 256, 152LL * 16), 256, 0, st>>>(A, (int)n);
  return A;
}

// in place: the n2 doubles of a become double-float pairs, or back
__global__ void split_to_ff(double* a, long long n2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    reinterpret_cast<ff*>(a)[i] = ff_from(a[i]);
}
__global__ void join_from_ff(double* a, long long n2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    a[i] = vec_out(reinterpret_cast<const ff*>(a)[i]);
}

}  // namespace

// Gauss-Jordan inverse of the SPD n x n matrix in A, ping-ponging with B; returns the buffer that holds
// the inverse (FP64). work: GJB^2 + 2 n GJB doubles. ff: the passes run in double-float arithmetic on
// the same buffers (8-byte elements), A converted on entry and the inverse converted back.
double* launch_gj_invert(double* A, double* B, long long n, double* work, unsigned* err, bool ff_arith,
                         cudaStream_t st) {
  if (!ff_arith) return gj_passes<double>(A, B, n, work, err, st);
  const long long n2 = n * n;
  const int grid = (int)std::min<long long>((n2 + 255) / 256, 152LL * 16);
  split_to_ff<<<grid, 256, 0, st>>>(A, n2);
  ff* r = gj_passes<ff>(reinterpret_cast<ff*>(A), reinterpret_cast<ff*>(B), n, reinterpret_cast<ff*>(work), err, st);
  double* out = reinterpret_cast<double*>(r);
  join_from_ff<<<grid, 256, 0, st>>>(out, n2);
  return out;
}

void launch_dense_gemv(const double* A, const double* b, double* x, long long n, const int* free_idx, cudaStream_t st) {
  const long long threads = n * 32;
  dense_gemv<<<(int)((threads + 255) / 256), 256, 0, st>>>(A, b, x, n, free_idx);
}

}  // namespace hy
