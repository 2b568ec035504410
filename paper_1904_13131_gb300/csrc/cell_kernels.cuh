// Cell kernels of the tangent action (Eq. mf_vmult with Eq. algebraic_tangent) and the device functions they
// share with the setup kernels (setup_kernels.cuh: Gauss-point state build, residual, diagonal), all with sum
// factorisation (Sec. 5).
//
// Work decomposition: one thread block per batch of CB cells, one thread per (cell, Gauss point) --
// the Gauss points and the nodes of a cell are both (k+1)^dim, so the same thread owns node p during
// gather/scatter and Gauss point p during the quadrature work. Each 1D contraction of the sum
// factorisation is a length-(k+1) dot product along one lattice line of the cell, read from shared
// memory; components are processed together so each stage needs one barrier.
//
// Integration is in the reference configuration: the paper integrates over the spatial configuration
// and divides by J (Sec. 5), which is the same integral. With G = d x / d xi (unit-cell derivative),
// M = F^{-1} / h and W = w_q h^dim, the quantity contracted with the unit-cell shape gradients is
//   P~ = Q~ M^T,   Q~ = g tau~ + JC~ : sym(g),   g = G M,   tau~ = W tau,   JC~ = W JC,
// so y_{a,c} = sum_q sum_J P~_{cJ} d N_a / d xi_J, i.e. sum_q W [g tau + JC:grad^s x] : grad(N_a e_c).
#pragma once
#include <type_traits>

#include "hy_internal.cuh"

namespace hy {

template <typename T>
struct CellArgs {
  const vec_t<T>* x;      // apply: source vector (level precision; FP64 for double-float)
  vec_t<T>* y;            // apply / residual / diag: destination, accumulated with atomics
  const vec_t<T>* ubar;   // level displacement (variants that recompute F)
  const double* u64;      // level displacement in FP64 (state build, residual, diagonal)
  const T* cache;         // per-Gauss-point cache in the blocked layout of layout_row<T>()
  T* cache_out;           // state build output
  const uint8_t* mat;     // material id per cell
  unsigned* err;          // device error word (J <= 0, NaN)
  unsigned long long* jmin_bits;  // min J over Gauss points, as ordered bits of a positive double
  Mat<T> mt;
  Geom g;
  Basis1D<T> b;
  long long nqp;          // ncells * NPT
  int pf;                 // apply: L2 prefetch distance in cell blocks (0: none)
  const double* X64;      // nodal coordinates of a curved reference geometry (null: the uniform lattice)
};

// --- asynchronous bulk copy (TMA engine) of a block's cache chunk into shared memory ------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One thread: announce `bytes` of transactions on the barrier and copy them global -> shared in pieces.
// dst, src and bytes are multiples of 16 bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  constexpr unsigned PIECE = 32768;
  for (unsigned off = 0; off < bytes; off += PIECE) {
    const unsigned sz = bytes - off < PIECE ? bytes - off : PIECE;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(static_cast<char*>(dst) + off)),
        "l"(static_cast<const char*>(src) + off), "r"(sz), "r"(smem_u32(bar))
        : "memory");
  }
}
// Order this thread's earlier generic-proxy accesses to shared memory before later async-proxy ones (a bulk
// copy refilling a buffer that threads have read).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Hint the TMA engine to pull `bytes` (multiple of 16, 16-byte aligned src) from global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void* src, unsigned bytes) {
  constexpr unsigned PIECE = 32768;
  for (unsigned off = 0; off < bytes; off += PIECE) {
    const unsigned sz = bytes - off < PIECE ? bytes - off : PIECE;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char*>(src) + off), "r"(sz)
                 : "memory");
  }
}
// Cache chunk `blk + pf` of this problem into L2, if it exists: the block that will read it, a few waves
// later, then finds it there instead of in HBM.
template <int NV, int BS, int CB, typename T>
__device__ __forceinline__ void prefetch_chunk(const CellArgs<T>& a, int blk) {
  if (a.pf <= 0) return;
  const long long nb = (a.g.ncells + CB - 1) / CB;
  const long long pb = (long long)blk + a.pf;
  if (pb < nb) prefetch_l2(a.cache + (size_t)pb * NV * BS, (unsigned)(NV * BS * sizeof(T)));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier; false if it did not complete within limit_ns of GPU wall time
// (checked every 64 polls) or MBAR_POLL_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned long long limit_ns = MBAR_WAIT_NS) {
  const unsigned a = smem_u32(bar);
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < MBAR_POLL_LIMIT; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// --- small helpers ------------------------------------------------------------------------------
template <int N, int STRIDE, bool TR, typename T>
__device__ __forceinline__ T contract(const T* __restrict__ line, int pax, const T (*M)[MAXN]) {
  // line points at the first entry of this thread's lattice line; M[r][j] (TR: M[j][r])
  T s = (TR ? M[0][pax] : M[pax][0]) * line[0];
#pragma unroll
  for (int j = 1; j < N; ++j) s = fma(TR ? M[j][pax] : M[pax][j], line[j * STRIDE], s);
  return s;
}

// Continues an accumulation: acc + sum_j M[r][j] line[j] (TR: M[j][r]).
template <int N, int STRIDE, bool TR, typename T>
__device__ __forceinline__ T contract_acc(const T* __restrict__ line, int pax, const T (*M)[MAXN], T acc) {
#pragma unroll
  for (int j = 0; j < N; ++j) acc = fma(TR ? M[j][pax] : M[pax][j], line[j * STRIDE], acc);
  return acc;
}

template <int DIM, int N>
struct Pt {
  int p, pc[3], stride[3];
  __device__ __forceinline__ explicit Pt(int p_) : p(p_) {
    pc[0] = p_ % N;
    pc[1] = (p_ / N) % N;
    pc[2] = DIM == 3 ? p_ / (N * N) : 0;
    stride[0] = 1;
    stride[1] = N;
    stride[2] = N * N;
  }
  __device__ __forceinline__ int base(int ax) const { return p - pc[ax] * stride[ax]; }
};

// This thread's row (or column) of a 1D table along every axis, read from shared memory before the
// stage that uses it. (Keeping them in registers for the whole kernel was measured on the FP32 action:
// no gain, more registers.)
template <int DIM, int N, typename T>
struct LineCoef {
  T c[DIM][N];
  __device__ __forceinline__ void rows(const T (*M)[MAXN], const Pt<DIM, N>& pt) {
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax)
#pragma unroll
      for (int j = 0; j < N; ++j) c[ax][j] = M[pt.pc[ax]][j];
  }
  __device__ __forceinline__ void cols(const T (*M)[MAXN], const Pt<DIM, N>& pt) {
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax)
#pragma unroll
      for (int j = 0; j < N; ++j) c[ax][j] = M[j][pt.pc[ax]];
  }
};

template <int N, int STRIDE, typename T>
__device__ __forceinline__ T dotline(const T* __restrict__ line, const T (&c)[N], T acc, bool first) {
#pragma unroll
  for (int j = 0; j < N; ++j) acc = (first && j == 0) ? c[0] * line[0] : fma(c[j], line[j * STRIDE], acc);
  return acc;
}

template <int DIM, int N, typename T>
__device__ __forceinline__ T line_ax(const T* line, int ax, const LineCoef<DIM, N, T>& k, T acc, bool first) {
  if (ax == 0) return dotline<N, 1>(line, k.c[0], acc, first);
  if (ax == 1) return dotline<N, N>(line, k.c[DIM > 1 ? 1 : 0], acc, first);
  return dotline<N, N * N>(line, k.c[DIM - 1], acc, first);
}

// Forward sweeps of NCOMP fields (pairs of buffers), coefficients in registers.
template <int DIM, int N, int NF, typename T>
__device__ __forceinline__ void sweeps_forward_coef(T* (&src)[NF], T* (&dst)[NF], const Pt<DIM, N>& pt,
                                                    const LineCoef<DIM, N, T>& kS) {
  constexpr int NPT = ipow(N, DIM);
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const int base = pt.base(ax);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int c = 0; c < DIM; ++c) dst[f][c * NPT + pt.p] = line_ax<DIM, N>(src[f] + c * NPT + base, ax, kS, T(0), true);
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T* t = src[f];
      src[f] = dst[f];
      dst[f] = t;
    }
  }
}

template <int DIM, int N, typename T>
__device__ __forceinline__ void grad_coef(const T* V, const Pt<DIM, N>& pt, const LineCoef<DIM, N, T>& kD, T G[DIM][DIM]) {
  constexpr int NPT = ipow(N, DIM);
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int J = 0; J < DIM; ++J) G[c][J] = line_ax<DIM, N>(V + c * NPT + pt.base(J), J, kD, T(0), true);
}

template <int DIM, int N, typename T>
__device__ __forceinline__ T* backward_coef(const T* bp, T* b0, T* b1, const Pt<DIM, N>& pt,
                                            const LineCoef<DIM, N, T>& kSt, const LineCoef<DIM, N, T>& kDt) {
  constexpr int NPT = ipow(N, DIM);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    T s = T(0);
#pragma unroll
    for (int J = 0; J < DIM; ++J) s = line_ax<DIM, N>(bp + (c * DIM + J) * NPT + pt.base(J), J, kDt, s, J == 0);
    b0[c * NPT + pt.p] = s;
  }
  __syncthreads();
  T* src = b0;
  T* dst = b1;
#pragma unroll
  for (int ax = DIM - 1; ax >= 0; --ax) {
    const int base = pt.base(ax);
#pragma unroll
    for (int c = 0; c < DIM; ++c) dst[c * NPT + pt.p] = line_ax<DIM, N>(src + c * NPT + base, ax, kSt, T(0), true);
    __syncthreads();
    T* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// Forward sum factorisation for NC components stored [c][NPT] at b0: interpolate to the Gauss
// points along every axis (S), ping-ponging through b1. Returns the buffer holding the values.
template <int DIM, int N, int NC, typename T>
__device__ __forceinline__ T* interp_forward(T* b0, T* b1, const Pt<DIM, N>& pt, const T (*S)[MAXN]) {
  constexpr int NPT = ipow(N, DIM);
  T* src = b0;
  T* dst = b1;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const int base = pt.base(ax);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T* line = src + c * NPT + base;
      T v;
      if (ax == 0) v = contract<N, 1, false>(line, pt.pc[0], S);
      else if (ax == 1) v = contract<N, N, false>(line, pt.pc[1], S);
      else v = contract<N, N * N, false>(line, pt.pc[2], S);
      dst[c * NPT + pt.p] = v;
    }
    __syncthreads();
    T* t = src; src = dst; dst = t;
  }
  return src;
}

// Collocation derivatives at the Gauss points: G[c][J] = sum_j D[q_J][j] V_c(q with q_J = j).
template <int DIM, int N, typename T>
__device__ __forceinline__ void colloc_grad(const T* V, const Pt<DIM, N>& pt, const T (*D)[MAXN], T G[DIM][DIM]) {
  constexpr int NPT = ipow(N, DIM);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    G[c][0] = contract<N, 1, false>(V + c * NPT + pt.base(0), pt.pc[0], D);
    G[c][1] = contract<N, N, false>(V + c * NPT + pt.base(1), pt.pc[1], D);
    if (DIM == 3) G[c][DIM - 1] = contract<N, N * N, false>(V + c * NPT + pt.base(2), pt.pc[2], D);
  }
}

// Transposed sum factorisation: from P~[c*DIM+J][NPT] at bp, apply D^T along J and sum over J, then
// S^T along every axis; ping-pongs through b0/b1 and returns the buffer holding nodal values.
template <int DIM, int N, typename T>
__device__ __forceinline__ T* integrate_backward(const T* bp, T* b0, T* b1, const Pt<DIM, N>& pt,
                                                 const T (*S)[MAXN], const T (*D)[MAXN]) {
  constexpr int NPT = ipow(N, DIM);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const T* P0 = bp + (c * DIM + 0) * NPT;
    const T* P1 = bp + (c * DIM + 1) * NPT;
    T s = contract<N, 1, true>(P0 + pt.base(0), pt.pc[0], D);
    s = contract_acc<N, N, true>(P1 + pt.base(1), pt.pc[1], D, s);
    if (DIM == 3) s = contract_acc<N, N * N, true>(bp + (c * DIM + DIM - 1) * NPT + pt.base(2), pt.pc[2], D, s);
    b0[c * NPT + pt.p] = s;
  }
  __syncthreads();
  T* src = b0;
  T* dst = b1;
#pragma unroll
  for (int ax = DIM - 1; ax >= 0; --ax) {
    const int base = pt.base(ax);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const T* line = src + c * NPT + base;
      T v;
      if (ax == 0) v = contract<N, 1, true>(line, pt.pc[0], S);
      else if (ax == 1) v = contract<N, N, true>(line, pt.pc[1], S);
      else v = contract<N, N * N, true>(line, pt.pc[2], S);
      dst[c * NPT + pt.p] = v;
    }
    __syncthreads();
    T* t = src; src = dst; dst = t;
  }
  return src;
}

// Voigt pairs: 3D (00,11,22,01,02,12), 2D (00,11,01).
template <int DIM> __device__ __forceinline__ constexpr int vi(int a) {
  return DIM == 3 ? (a < 3 ? a : (a == 5 ? 1 : 0)) : (a < 2 ? a : 0);
}
template <int DIM> __device__ __forceinline__ constexpr int vj(int a) {
  return DIM == 3 ? (a < 3 ? a : (a == 3 ? 1 : 2)) : (a < 2 ? a : 1);
}

// P~ = Q M^T with Q = g tau + S (S symmetric, Voigt), g = G M.
template <int DIM, typename T>
__device__ __forceinline__ void finish_flux(const T g[DIM][DIM], const T tau[nsym(DIM)], const T Sv[nsym(DIM)],
                                            const T M[DIM][DIM], T P[DIM][DIM]) {
  constexpr int NS = nsym(DIM);
  T tf[DIM][DIM];
#pragma unroll
  for (int a = 0; a < NS; ++a) {
    tf[vi<DIM>(a)][vj<DIM>(a)] = tau[a];
    tf[vj<DIM>(a)][vi<DIM>(a)] = tau[a];
  }
  T Sf[DIM][DIM];
#pragma unroll
  for (int a = 0; a < NS; ++a) {
    Sf[vi<DIM>(a)][vj<DIM>(a)] = Sv[a];
    Sf[vj<DIM>(a)][vi<DIM>(a)] = Sv[a];
  }
  T Q[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      T s = Sf[i][j];
#pragma unroll
      for (int k = 0; k < DIM; ++k) s = fma(g[i][k], tf[k][j], s);
      Q[i][j] = s;
    }
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int J = 0; J < DIM; ++J) {
      T s = Q[c][0] * M[J][0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) s = fma(Q[c][j], M[J][j], s);
      P[c][J] = s;
    }
}

template <int DIM, typename T>
__device__ __forceinline__ void matmul(const T A[DIM][DIM], const T B[DIM][DIM], T C[DIM][DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      T s = A[i][0] * B[0][j];
#pragma unroll
      for (int k = 1; k < DIM; ++k) s = fma(A[i][k], B[k][j], s);
      C[i][j] = s;
    }
}

// Volumetric part of the law: p = J U'(J) and J p'(J). Law 0 is the paper's U = lambda ln^2 J (Sec. 2.3):
// p = 2 lambda ln J, J p' = 2 lambda. Law 1 is U = lambda/4 (J^2 - 1 - 2 ln J): p = lambda/2 (J^2 - 1),
// J p' = lambda J^2. Then tau = mu b - (mu - p) I and J*C = 2 (mu - p) S + J p' I (x) I.
template <typename T>
__device__ __forceinline__ void volumetric(T J, T lam, int law, T& p, T& jdp) {
  if (law == 1) {
    const T J2 = J * J;
    p = T(0.5) * lam * (J2 - T(1));
    jdp = lam * J2;
  } else {
    p = T(2) * lam * log(J);
    jdp = T(2) * lam;
  }
}

// Neo-Hooke state at a Gauss point from F (Sec. 2.3), in the scaled form used by the kernels:
// M = F^{-1}/h, tau~ = W (mu b - (mu - 2 lambda ln J) I), c1~ = 2 W (mu - 2 lambda ln J), c2~ = 2 W lambda.
// If c1 is given (>= 0 flag), it replaces mu - 2 lambda ln J (Algorithm 1 caches it).
template <int DIM, typename T>
__device__ __forceinline__ T neo_hooke_state(const T F[DIM][DIM], T mu, T lam, int law, T W, T inv_h, bool have_c,
                                             T c_in, T M[DIM][DIM], T tau[nsym(DIM)], T& c1, T& c2) {
  T J;
  if (DIM == 3) {
    const T a00 = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    const T a01 = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    const T a02 = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    const T a10 = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    const T a11 = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    const T a12 = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    const T a20 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    const T a21 = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    const T a22 = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    J = F[0][0] * a00 + F[0][1] * a10 + F[0][2] * a20;
    const T s = inv_h / J;
    M[0][0] = a00 * s; M[0][1] = a01 * s; M[0][2] = a02 * s;
    M[1][0] = a10 * s; M[1][1] = a11 * s; M[1][2] = a12 * s;
    M[2][0] = a20 * s; M[2][1] = a21 * s; M[2][2] = a22 * s;
  } else {
    J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    const T s = inv_h / J;
    M[0][0] = F[1][1] * s; M[0][1] = -F[0][1] * s;
    M[1][0] = -F[1][0] * s; M[1][1] = F[0][0] * s;
  }
  T pv, jdp;
  volumetric(J, lam, law, pv, jdp);
  const T c = have_c ? c_in : mu - pv;
  const T Wmu = W * mu;
#pragma unroll
  for (int a = 0; a < nsym(DIM); ++a) {
    const int i = vi<DIM>(a), j = vj<DIM>(a);
    T bij = F[i][0] * F[j][0];
#pragma unroll
    for (int k = 1; k < DIM; ++k) bij = fma(F[i][k], F[j][k], bij);
    tau[a] = Wmu * bij - (i == j ? W * c : T(0));
  }
  c1 = T(2) * W * c;
  c2 = W * jdp;
  return J;
}

// Neo-Hooke state for the variants that recompute it in every application (the paper's law: a second law
// goes through the caching variants, whose state kernel evaluates it), scaled so that no
// F^{-1} is formed: with adj = J F^{-1}, rho = 1/J and kappa = (W/h) rho^2, the flux contracted with
// the unit-cell shape gradients is P~ = Q' adj^T, Q' = g' tau' + c1' sym(g') + c2' tr(g') I, where
// g' = Grad x adj, tau' = kappa tau, c1' = 2 kappa (mu - 2 lambda ln J), c2' = 2 kappa lambda -- the same
// quantity as W/h (g tau + JC : sym g) F^{-T} with g = Grad x F^{-1}.
// LAW: the volumetric function is the material's (law 0 or 1, chosen at run time) instead of the paper's.
template <int DIM, typename T, bool LAW = false>
__device__ __forceinline__ void neo_hooke_adj(const T F[DIM][DIM], T mu, T lam, T Wh, bool have_c, T c_in,
                                              T adj[DIM][DIM], T tau[nsym(DIM)], T& c1, T& c2, int law = 0) {
  T J;
  if (DIM == 3) {
    adj[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    adj[0][1] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    adj[0][2] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    adj[1][0] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    adj[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    adj[1][2] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    adj[2][0] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    adj[2][1] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    adj[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    J = F[0][0] * adj[0][0] + F[0][1] * adj[1][0] + F[0][2] * adj[2][0];
  } else {
    adj[0][0] = F[1][1];
    adj[0][1] = -F[0][1];
    adj[1][0] = -F[1][0];
    adj[1][1] = F[0][0];
    J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  }
  T rho;
  rho = rcp_rn(J);
  const T kappa = Wh * rho * rho;
  T c, jdp;
  if (LAW) {
    T pv;
    volumetric(J, lam, law, pv, jdp);
    c = have_c ? c_in : mu - pv;
  } else {
    c = have_c ? c_in : mu - T(2) * lam * log(J);
    jdp = T(2) * lam;
  }
  const T kmu = kappa * mu, kc = kappa * c;
#pragma unroll
  for (int a = 0; a < nsym(DIM); ++a) {
    const int i = vi<DIM>(a), j = vj<DIM>(a);
    T bij = F[i][0] * F[j][0];
#pragma unroll
    for (int k = 1; k < DIM; ++k) bij = fma(F[i][k], F[j][k], bij);
    tau[a] = (i == j) ? fma(kmu, bij, -kc) : kmu * bij;
  }
  c1 = T(2) * kc;
  c2 = kappa * jdp;
}

// Material part for the neo-Hooke action (Eq. simplified_action): S = c1 sym(g) + c2 tr(g) I.
template <int DIM, typename T>
__device__ __forceinline__ void nh_action(const T g[DIM][DIM], T c1, T c2, T Sv[nsym(DIM)]) {
  T tr = g[0][0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) tr += g[i][i];
  const T ct = c2 * tr;
  const T hc = T(0.5) * c1;
#pragma unroll
  for (int a = 0; a < nsym(DIM); ++a) {
    const int i = vi<DIM>(a), j = vj<DIM>(a);
    Sv[a] = (i == j) ? fma(c1, g[i][i], ct) : hc * (g[i][j] + g[j][i]);
  }
}

// Shared-memory layout of one block.
template <int DIM, int N, typename T, int CB_ = cells_per_block(DIM, N)>
struct Smem {
  static constexpr int NPT = ipow(N, DIM);
  static constexpr int CB = CB_;
  T S[MAXN][MAXN], D[MAXN][MAXN], Dh[MAXN][MAXN], W[NPT], Wh[NPT];
  T mu[MAXMAT], lam[MAXMAT];
  T bp[CB][DIM * DIM][NPT];  // fluxes; also the ping-pong pair for the displacement
  T b0[CB][DIM][NPT];
  T b1[CB][DIM][NPT];
};

template <int DIM, int N, typename T, int CB>
__device__ __forceinline__ void load_tables(Smem<DIM, N, T, CB>& s, const CellArgs<T>& a) {
  constexpr int NPT = ipow(N, DIM);
  const int t = threadIdx.x;
  if (t < MAXN * MAXN) {
    s.S[t / MAXN][t % MAXN] = a.b.S[t / MAXN][t % MAXN];
    s.D[t / MAXN][t % MAXN] = a.b.D[t / MAXN][t % MAXN];
    s.Dh[t / MAXN][t % MAXN] = a.b.D[t / MAXN][t % MAXN] * T(a.g.inv_h);  // derivative in physical units
  }
  if (t < NPT) {
    const int q0 = t % N, q1 = (t / N) % N, q2 = DIM == 3 ? t / (N * N) : 0;
    T w = a.b.w[q0] * a.b.w[q1];
    if (DIM == 3) w *= a.b.w[q2];
    T hd = T(a.g.h) * T(a.g.h);
    if (DIM == 3) hd *= T(a.g.h);
    s.W[t] = w * hd;
    s.Wh[t] = w * hd * T(a.g.inv_h);
  }
  if (t < MAXMAT) {
    s.mu[t] = a.mt.mu[t];
    s.lam[t] = a.mt.lam[t];
  }
}

// Lattice location of (cell, local node p).
template <int DIM, int N>
struct CellLoc {
  int node;
  uint32_t cmask;
  __device__ __forceinline__ CellLoc(const Geom& g, int cell, const Pt<DIM, N>& pt) {
    constexpr int K = N - 1;
    const int m = g.m;
    const int c0 = cell % m;
    const int c1 = (cell / m) % m;
    const int c2 = DIM == 3 ? cell / (m * m) : 0;
    const int i0 = K * c0 + pt.pc[0], i1 = K * c1 + pt.pc[1], i2 = K * c2 + pt.pc[2];
    node = i0 + g.L * (i1 + (DIM == 3 ? g.L * i2 : 0));
    cmask = node_cmask<DIM>(g, i0, i1, i2);
  }
};

// ------------------------------------------------------------------------------------------------
// Flux P~ at one Gauss point from the gradient G of x (and Gu of the displacement for SC/NC), the point's
// cache entries (row stride st, entry qg of the shared-memory chunk cs) and the material, per variant:
//   T4: P~ = (g tau~ + JC~ : sym g) M^T, g = G M with M = F^{-1}/h, tau~, JC~ cached   (Algorithm 3)
//   T2: the same with JC~ : s = c1~ s + c2~ tr(s) I                                     (Algorithm 2)
//   FC/SC/NC: the state recomputed from F (cached, or I + Grad u), with g' = Grad x adj F (Algorithm 1 for SC).
//   FCG/SCG/NCG (curved cells, either law): G and Gu are unit-cell derivatives, mapped by the cached
//   inverse Jacobian invJ; the cached weight W replaces W/h, and the flux is mapped back, P~ = P invJ^T.
template <int DIM, int VAR, typename T>
__device__ __forceinline__ void qp_flux(const T G[DIM][DIM], const T Gu[DIM][DIM], const T* __restrict__ cs, int st,
                                        int qg, bool active, int id, const T* mu, const T* lam, T Wh, T P[DIM][DIM],
                                        int law = 0) {
  constexpr int NS = nsym(DIM);
  constexpr int BV = base_variant(VAR);
  constexpr bool GEN = is_general(VAR);
  T M[DIM][DIM], tau[NS], Sv[NS], g[DIM][DIM];
  if (VAR == VAR_T4 || VAR == VAR_T2) {
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) M[i / DIM][i % DIM] = active ? cs[i * st + qg] : T(0);
#pragma unroll
    for (int i = 0; i < NS; ++i) tau[i] = active ? cs[(DIM * DIM + i) * st + qg] : T(0);
    matmul<DIM>(G, M, g);
    if (VAR == VAR_T4) {
      constexpr int OFF = DIM * DIM + NS;
      T v[NS];
#pragma unroll
      for (int al = 0; al < NS; ++al) {
        const int i = vi<DIM>(al), j = vj<DIM>(al);
        v[al] = (i == j) ? g[i][i] : g[i][j] + g[j][i];
      }
#pragma unroll
      for (int al = 0; al < NS; ++al) {
        T acc = T(0);
#pragma unroll
        for (int be = 0; be < NS; ++be) {
          const int lo = al < be ? al : be, hi = al < be ? be : al;
          const int idx = lo * NS - lo * (lo - 1) / 2 + (hi - lo);  // upper triangle, row major
          const T cv = active ? cs[(OFF + idx) * st + qg] : T(0);
          acc = (be == 0) ? cv * v[be] : fma(cv, v[be], acc);
        }
        Sv[al] = acc;
      }
    } else {
      const T c1 = active ? cs[(DIM * DIM + NS) * st + qg] : T(0);
      const T c2 = active ? cs[(DIM * DIM + NS + 1) * st + qg] : T(0);
      nh_action<DIM>(g, c1, c2, Sv);
    }
  } else {
    // the reference map of this point (general build): invJ rows after the variant's own, then W
    constexpr int GOFF = cache_values(BV, DIM);
    T Ji[DIM][DIM], Gx[DIM][DIM], W = Wh;
    if (GEN) {
#pragma unroll
      for (int i = 0; i < DIM * DIM; ++i)
        Ji[i / DIM][i % DIM] = active ? cs[(GOFF + i) * st + qg] : (i % (DIM + 1) == 0 ? T(1) : T(0));
      W = active ? cs[(GOFF + DIM * DIM) * st + qg] : T(0);
      matmul<DIM>(G, Ji, Gx);
    }
    T F[DIM][DIM];
    if (BV == VAR_FC) {
#pragma unroll
      for (int i = 0; i < DIM * DIM; ++i)
        F[i / DIM][i % DIM] = active ? cs[i * st + qg] : (i % (DIM + 1) == 0 ? T(1) : T(0));
    } else {
      T Gp[DIM][DIM];
      if (GEN) {
        matmul<DIM>(Gu, Ji, Gp);
      } else {
#pragma unroll
        for (int i = 0; i < DIM * DIM; ++i) Gp[i / DIM][i % DIM] = Gu[i / DIM][i % DIM];
      }
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int J = 0; J < DIM; ++J) F[i][J] = (i == J) ? T(1) + Gp[i][J] : Gp[i][J];
    }
    const T cin = (BV == VAR_SC && active) ? cs[qg] : T(0);
    T c1, c2;
    neo_hooke_adj<DIM, T, GEN>(F, mu[id], lam[id], W, BV == VAR_SC, cin, M, tau, c1, c2, law);  // M = adj
    if (GEN) {
      matmul<DIM>(Gx, M, g);
    } else {
      matmul<DIM>(G, M, g);
    }
    nh_action<DIM>(g, c1, c2, Sv);
    if (GEN) {
      T Pp[DIM][DIM];
      finish_flux<DIM>(g, tau, Sv, M, Pp);
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int J = 0; J < DIM; ++J) {
          T v = Pp[c][0] * Ji[J][0];
#pragma unroll
          for (int K = 1; K < DIM; ++K) v = fma(Pp[c][K], Ji[J][K], v);
          P[c][J] = v;
        }
      return;
    }
  }
  finish_flux<DIM>(g, tau, Sv, M, P);
}

// ------------------------------------------------------------------------------------------------
// Tangent action y += A(u) x on the cells of this block (Eq. mf_vmult), variants:
//   T4: cache M, tau~, JC~ (Algorithm 3)            T2: cache M, tau~, c1~, c2~ (Algorithm 2)
//   FC: cache F, recompute the neo-Hooke state      SC: cache mu - 2 lambda ln J, recompute F (Algorithm 1)
//   NC: nothing cached, recompute F and the state from the gathered displacement.
// Constrained dofs: x is read as zero there and nothing is added to y there.
// blk is the index of the block of cells (and of the cache chunk) that this thread block processes.
template <int DIM, int N, int VAR, typename T>
__device__ __forceinline__ void apply_point_body(const CellArgs<T>& a, const int blk) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int CB = layout_cells<T>(DIM, N);
  constexpr int NS = nsym(DIM);
  constexpr int BV = base_variant(VAR);
  constexpr bool NEED_U = (BV == VAR_NC || BV == VAR_SC);
  constexpr int NV = cache_values(VAR, DIM);
  constexpr int BS = layout_row<T>(DIM, N);
  __shared__ Smem<DIM, N, T, CB> s;
  __shared__ __align__(8) unsigned long long bar;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  // This block's cache chunk [NV][BS]: staged in shared memory by a bulk copy, except in double-float,
  // whose FP32-pipe-bound work gains more from the occupancy that a 70 KB chunk would cost; there the
  // Gauss-point work reads it from global memory, coalesced (thread i reads entry i of every row).
  constexpr bool STAGE = !std::is_same<T, ff>::value;
  const T* cs = STAGE ? reinterpret_cast<const T*>(dyn_smem) : a.cache + (size_t)blk * NV * BS;
  if (STAGE && NV > 0 && threadIdx.x == 0) {
    // the chunk streams in (TMA bulk copy) while the block gathers x and runs the forward sweeps
    mbar_init(&bar, 1);
    bulk_load(dyn_smem, a.cache + (size_t)blk * NV * BS, (unsigned)(NV * BS * sizeof(T)), &bar);
    prefetch_chunk<NV, BS, CB>(a, blk);
  }
  load_tables<DIM, N>(s, a);
  const int cl = threadIdx.x / NPT;
  const Pt<DIM, N> pt(threadIdx.x % NPT);
  const int cell = blk * CB + cl;
  const bool active = cell < a.g.ncells;
  const CellLoc<DIM, N> loc(a.g, active ? cell : 0, pt);
  T* b0 = &s.b0[cl][0][0];
  T* b1 = &s.b1[cl][0][0];
  T* bp = &s.bp[cl][0][0];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    T v = T(0), w = T(0);
    if (active) {
      v = ((loc.cmask >> c) & 1u) ? T(0) : vec_in<T>(a.x[(long long)loc.node * DIM + c]);
      if (NEED_U) w = vec_in<T>(a.ubar[(long long)loc.node * DIM + c]);
    }
    b0[c * NPT + pt.p] = v;
    if (NEED_U) bp[c * NPT + pt.p] = w;
  }
  __syncthreads();
  // coefficient rows of this thread's lines: loaded once (FP32) or before each stage (FP64)
  constexpr bool HOIST = false;
  // derivatives in physical units (D / h) on the lattice; the general build maps unit-cell ones itself
  constexpr bool PHYS = (BV == VAR_FC || NEED_U) && !is_general(VAR);
  LineCoef<DIM, N, T> kS, kD, kSt, kDt;
  if (HOIST) {
    kS.rows(s.S, pt);
    kD.rows(PHYS ? s.Dh : s.D, pt);
    kSt.cols(s.S, pt);
    kDt.cols(s.D, pt);
  }
  // forward: x (and u) to the Gauss points, then collocation derivatives
  T G[DIM][DIM], Gu[DIM][DIM];
  if (!HOIST) kS.rows(s.S, pt);
  if (NEED_U) {
    T* src[2] = {b0, bp};
    T* dst[2] = {b1, bp + DIM * NPT};
    sweeps_forward_coef<DIM, N, 2>(src, dst, pt, kS);  // both fields in the same stages
    if (!HOIST) kD.rows(PHYS ? s.Dh : s.D, pt);
    grad_coef<DIM, N>(src[0], pt, kD, G);   // physical gradients: Grad x, Grad u
    grad_coef<DIM, N>(src[1], pt, kD, Gu);
    __syncthreads();  // bp is overwritten with the fluxes below
  } else {
    T* src[1] = {b0};
    T* dst[1] = {b1};
    sweeps_forward_coef<DIM, N, 1>(src, dst, pt, kS);
    if (!HOIST) kD.rows(PHYS ? s.Dh : s.D, pt);
    grad_coef<DIM, N>(src[0], pt, kD, G);  // Grad x (FC) or d x / d xi (T4, T2: M holds F^{-1}/h)
  }
  if (STAGE && NV > 0) {
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // the copy never completed: flag it, give it one more bounded wait, leave
      if (threadIdx.x == 0) atomicOr(a.err, ERRBIT_TIMEOUT);
      mbar_wait(&bar, 0);
      return;
    }
  }
  // quadrature-point work
  T P[DIM][DIM];
  qp_flux<DIM, VAR>(G, Gu, cs, BS, threadIdx.x, active, active ? a.mat[cell] : 0, s.mu, s.lam, s.Wh[pt.p], P,
                    a.mt.law);
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int J = 0; J < DIM; ++J) bp[(c * DIM + J) * NPT + pt.p] = P[c][J];
  __syncthreads();
  if (!HOIST) {
    kSt.cols(s.S, pt);
    kDt.cols(s.D, pt);
  }
  const T* Y = backward_coef<DIM, N>(bp, b0, b1, pt, kSt, kDt);
  if (active) {
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (!((loc.cmask >> c) & 1u)) atomicAdd(&a.y[(long long)loc.node * DIM + c], vec_out(Y[c * NPT + pt.p]));
  }
}

// ------------------------------------------------------------------------------------------------
// Tangent action, one thread per x-line of a cell (the FP32 form). The thread holds the (k+1) nodes of its
// line, and later its (k+1) Gauss points, in registers: sweeps and derivatives along x need no shared
// memory, and gather and scatter touch one contiguous run of (k+1)*dim values. The y and z sweeps exchange
// values through shared memory, the thread playing the line (q0 varies; q1 = l1, q2 = l2) of each stage.
// Same arithmetic, variants and Dirichlet treatment as apply_kernel.
// PERSIST: the thread block loops over the cell blocks blk0, blk0 + step, ... with one shared-memory
// stage of the cache: the bulk copy of the next chunk is issued as soon as the Gauss-point work has read
// the current one, so it runs under the transposed sweeps, the scatter, the next gather and the forward
// sweeps (tables are loaded once per thread block). Otherwise the thread block processes the one cell
// block blk0.
template <int DIM, int N, int VAR, typename T, bool PERSIST = false>
__device__ __forceinline__ void apply_line_body(const CellArgs<T>& a, const int blk0, const int step) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int NLC = ipow(N, DIM - 1);
  constexpr int CB = layout_cells<T>(DIM, N);
  constexpr int TL = CB * NLC;  // line threads of the block
  constexpr int K = N - 1;
  constexpr int BV = base_variant(VAR);
  constexpr bool NEED_U = (BV == VAR_NC || BV == VAR_SC);
  constexpr bool PHYS = (BV == VAR_FC || NEED_U) && !is_general(VAR);
  constexpr int NV = cache_values(VAR, DIM);
  constexpr int BS = layout_row<T>(DIM, N);
  // Line buffers, component- and Gauss-index-major: entry (c, q, line i of the block) at (c N + q) TL + i,
  // so that the stores of a stage (thread i writes its own line) fall in consecutive banks.
  constexpr int NB = DIM * N * TL;
  constexpr int NBU = NEED_U ? NB : 1;
  __shared__ T tS[MAXN][MAXN], tD[MAXN][MAXN], tDh[MAXN][MAXN], tWh[NPT], tmu[MAXMAT], tlam[MAXMAT];
  __shared__ T buf0[NB], buf1[NB];
  __shared__ T ubuf0[NBU], ubuf1[NBU];
  __shared__ T flux[DIM * (DIM - 1) * N * TL];  // (c, J - 1, q, i) at ((c (DIM-1) + J - 1) N + q) TL + i
  __shared__ __align__(8) unsigned long long bar;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  T* const cs = reinterpret_cast<T*>(dyn_smem);
  const int t = threadIdx.x;
  // The block's cache chunk streams into shared memory with one bulk copy (measured faster for T4 than
  // reading the cache straight from global memory at the Gauss points, with or without an L2 prefetch of
  // the chunks ahead of use).
  constexpr unsigned CHUNK = (unsigned)(NV * BS * sizeof(T));
  const int nb = PERSIST ? (a.g.ncells + CB - 1) / CB : blk0 + 1;
  if (NV > 0 && t == 0) {
    mbar_init(&bar, 1);
    if (blk0 < nb) {
      bulk_load(cs, a.cache + (size_t)blk0 * NV * BS, CHUNK, &bar);
      if (!PERSIST) prefetch_chunk<NV, BS, CB>(a, blk0);
    }
  }
  // tables (strided loops: a block may have fewer threads than entries). The rows a thread indexes by
  // its own line (l1, l2) are read from shared memory; entries with compile-time indices (the x
  // direction) come straight from the kernel arguments.
  for (int i = t; i < MAXN * MAXN; i += blockDim.x) {
    tS[i / MAXN][i % MAXN] = a.b.S[i / MAXN][i % MAXN];
    tD[i / MAXN][i % MAXN] = a.b.D[i / MAXN][i % MAXN];
    tDh[i / MAXN][i % MAXN] = a.b.D[i / MAXN][i % MAXN] * T(a.g.inv_h);
  }
  for (int i = t; i < NPT; i += blockDim.x) {
    const int q0 = i % N, q1 = (i / N) % N, q2 = DIM == 3 ? i / (N * N) : 0;
    T w = a.b.w[q0] * a.b.w[q1];
    T hd = T(a.g.h) * T(a.g.h);
    if (DIM == 3) {
      w *= a.b.w[q2];
      hd *= T(a.g.h);
    }
    tWh[i] = w * hd * T(a.g.inv_h);
  }
  for (int i = t; i < MAXMAT; i += blockDim.x) {
    tmu[i] = a.mt.mu[i];
    tlam[i] = a.mt.lam[i];
  }
  const T xh = PHYS ? T(a.g.inv_h) : T(1);  // x derivatives: D from the arguments, scaled once
  const int cl = t / NLC, l = t % NLC;
  const int l1 = l % N, l2 = DIM == 3 ? l / N : 0;
  const int ly = cl * NLC + N * l2;  // line of this cell with y index 0 and this thread's z index
  const int lz = cl * NLC + l1;      // line of this cell with this thread's y index and z index 0
  auto B = [](int c, int q, int i) { return (c * N + q) * TL + i; };
  auto FX = [](int c, int J, int q, int i) { return ((c * (DIM - 1) + J) * N + q) * TL + i; };
  int it = 0;
  for (int blk = blk0; blk < nb; blk += step, ++it) {
    const int cell = blk * CB + cl;
    const bool active = cell < a.g.ncells;
    const int m = a.g.m;
    const int cc = active ? cell : 0;
    const int c0 = cc % m, c1 = (cc / m) % m, c2 = DIM == 3 ? cc / (m * m) : 0;
    const int i1 = K * c1 + l1, i2 = K * c2 + l2;
    const long long node0 = K * c0 + (long long)a.g.L * (i1 + (DIM == 3 ? (long long)a.g.L * i2 : 0));
    uint32_t cms[N];
    T v[N][DIM], vu[N][DIM];
#pragma unroll
    for (int a0 = 0; a0 < N; ++a0) {
      cms[a0] = node_cmask<DIM>(a.g, K * c0 + a0, i1, i2);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const long long dof = (node0 + a0) * DIM + c;
        v[a0][c] = (active && !((cms[a0] >> c) & 1u)) ? vec_in<T>(a.x[dof]) : T(0);
        vu[a0][c] = (NEED_U && active) ? vec_in<T>(a.ubar[dof]) : T(0);
      }
    }
    __syncthreads();
    // x: interpolation to the Gauss points of the line, in registers
    T X[N][DIM], XU[N][DIM];
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T sx = T(0), su = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          sx = fma(a.b.S[q][j], v[j][c], sx);
          if (NEED_U) su = fma(a.b.S[q][j], vu[j][c], su);
        }
        X[q][c] = sx;
        XU[q][c] = su;
      }
    // y (and z): through shared memory
    T V[N][DIM], VU[N][DIM];
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        buf0[B(c, q, t)] = X[q][c];
        if (NEED_U) ubuf0[NEED_U ? B(c, q, t) : 0] = XU[q][c];
      }
    __syncthreads();
    if (DIM == 3) {
      // y: this thread plays (q1 = l1, a2 = l2)
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          T sx = T(0), su = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            sx = fma(tS[l1][j], buf0[B(c, q, ly + j)], sx);
            if (NEED_U) su = fma(tS[l1][j], ubuf0[NEED_U ? B(c, q, ly + j) : 0], su);
          }
          buf1[B(c, q, t)] = sx;
          if (NEED_U) ubuf1[NEED_U ? B(c, q, t) : 0] = su;
        }
      __syncthreads();
      // z: (q1 = l1, q2 = l2)
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          T sx = T(0), su = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            sx = fma(tS[l2][j], buf1[B(c, q, lz + N * j)], sx);
            if (NEED_U) su = fma(tS[l2][j], ubuf1[NEED_U ? B(c, q, lz + N * j) : 0], su);
          }
          V[q][c] = sx;
          VU[q][c] = su;
        }
    } else {
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          T sx = T(0), su = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            sx = fma(tS[l1][j], buf0[B(c, q, ly + j)], sx);
            if (NEED_U) su = fma(tS[l1][j], ubuf0[NEED_U ? B(c, q, ly + j) : 0], su);
          }
          V[q][c] = sx;
          VU[q][c] = su;
        }
    }
    // values at the Gauss points of the line go to shared memory for the y/z derivatives of the others
    // (3D: buf0 was last read before the previous barrier; 2D: buf1 is unused so far)
    T* const vb = DIM == 3 ? buf0 : buf1;
    T* const vub = DIM == 3 ? ubuf0 : ubuf1;
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        vb[B(c, q, t)] = V[q][c];
        if (NEED_U) vub[NEED_U ? B(c, q, t) : 0] = VU[q][c];
      }
    __syncthreads();
    if (NV > 0) {
      const unsigned parity = it & 1;  // the it-th copy completes phase it of the barrier
      const bool ok = mbar_wait(&bar, parity);
      if (__syncthreads_or(!ok)) {  // the copy never completed: flag it, give it one more bounded wait, leave
        if (t == 0) atomicOr(a.err, ERRBIT_TIMEOUT);
        mbar_wait(&bar, parity);
        return;
      }
    }
    const T* cq = cs;
    const T (*Dd)[MAXN] = PHYS ? tDh : tD;
    const int id = active ? a.mat[cell] : 0;
    T Px[N][DIM];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const int p = q + N * l;
      T G[DIM][DIM], Gu[DIM][DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T g0 = T(0), u0 = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          g0 = fma(a.b.D[q][j], V[j][c], g0);
          if (NEED_U) u0 = fma(a.b.D[q][j], VU[j][c], u0);
        }
        G[c][0] = PHYS ? g0 * xh : g0;
        Gu[c][0] = PHYS ? u0 * xh : u0;
        T g1 = T(0), u1 = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          g1 = fma(Dd[l1][j], vb[B(c, q, ly + j)], g1);
          if (NEED_U) u1 = fma(Dd[l1][j], vub[NEED_U ? B(c, q, ly + j) : 0], u1);
        }
        G[c][1] = g1;
        Gu[c][1] = u1;
        if (DIM == 3) {
          T g2 = T(0), u2 = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            g2 = fma(Dd[l2][j], vb[B(c, q, lz + N * j)], g2);
            if (NEED_U) u2 = fma(Dd[l2][j], vub[NEED_U ? B(c, q, lz + N * j) : 0], u2);
          }
          G[c][DIM - 1] = g2;
          Gu[c][DIM - 1] = u2;
        }
      }
      T P[DIM][DIM];
      qp_flux<DIM, VAR>(G, Gu, cq, BS, cl * NPT + p, active, id, tmu, tlam, tWh[p], P, a.mt.law);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        Px[q][c] = P[c][0];
#pragma unroll
        for (int J = 1; J < DIM; ++J) flux[FX(c, J - 1, q, t)] = P[c][J];
      }
    }
    __syncthreads();
    if (PERSIST && NV > 0 && t == 0 && blk + step < nb) {
      // every thread has read this chunk (barrier above): refill the stage with the next one
      fence_proxy_async();
      bulk_load(cs, a.cache + (size_t)(blk + step) * NV * BS, CHUNK, &bar);
    }
    // transposed derivatives summed over the directions: x from registers, y/z from shared memory
    T Wq[N][DIM];
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(a.b.D[j][q], Px[j][c], s);
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(tD[j][l1], flux[FX(c, 0, q, ly + j)], s);
        if (DIM == 3) {
#pragma unroll
          for (int j = 0; j < N; ++j) s = fma(tD[j][l2], flux[FX(c, DIM - 2, q, lz + N * j)], s);
        }
        Wq[q][c] = s;
      }
    // transposed interpolation: z, y through shared memory (buffers free since the flux barrier), x in registers
    T Yb[N][DIM];
    if (DIM == 3) {
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) buf1[B(c, q, t)] = Wq[q][c];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {  // z: (q1 = l1, a2 = l2)
          T sz = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) sz = fma(tS[j][l2], buf1[B(c, q, lz + N * j)], sz);
          buf0[B(c, q, t)] = sz;
        }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {  // y: (a1 = l1, a2 = l2)
          T sy = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) sy = fma(tS[j][l1], buf0[B(c, q, ly + j)], sy);
          Yb[q][c] = sy;
        }
    } else {
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) buf0[B(c, q, t)] = Wq[q][c];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < N; ++q)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          T sy = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) sy = fma(tS[j][l1], buf0[B(c, q, ly + j)], sy);
          Yb[q][c] = sy;
        }
    }
    if (active) {
#pragma unroll
      for (int a0 = 0; a0 < N; ++a0)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          if ((cms[a0] >> c) & 1u) continue;
          T s = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) s = fma(a.b.S[j][a0], Yb[j][c], s);
          atomicAdd(&a.y[(node0 + a0) * DIM + c], vec_out(s));
        }
    }
    if (PERSIST) __syncthreads();  // the next cell block reuses the buffers and refills this cache stage
  }
}

// ------------------------------------------------------------------------------------------------
// Tangent action, one thread per z-plane of a cell (3D, FP32). The thread holds the (k+1)^2 nodes of its
// node plane a2 = l2, then the (k+1)^2 Gauss points of Gauss plane q2 = l2, in registers: interpolation,
// derivatives and their transposes along x and y need no shared memory, and only the z direction exchanges
// values between the k+1 threads of a cell through shared memory -- four exchanges of (k+1)^2 d values per
// thread (the z sweep, the z derivative, the z part of the flux, the transposed z sweep), about 60 % of the
// shared-memory traffic of the line form. Same arithmetic, variants, cache layout and Dirichlet treatment as
// apply_kernel. The transposed x and y derivatives are accumulated Gauss point by Gauss point.
// Built for degrees 1-2 (n <= PLANE_MAX_N): at higher degrees a plane is 16-25 nodes per component, too many
// registers; the line form serves those.
constexpr int PLANE_MAX_N = 3;
template <int N, int VAR, typename T>
__device__ __forceinline__ void apply_plane_body(const CellArgs<T>& a, const int blk) {
  constexpr int DIM = 3;
  constexpr int NPT = N * N * N;
  constexpr int NP = N * N;  // nodes or Gauss points of a plane
  constexpr int CB = layout_cells<T>(DIM, N);
  constexpr int TP = CB * N;  // plane threads of the block
  constexpr int K = N - 1;
  constexpr int BV = base_variant(VAR);
  constexpr bool NEED_U = (BV == VAR_NC || BV == VAR_SC);
  constexpr bool PHYS = (BV == VAR_FC || NEED_U) && !is_general(VAR);
  constexpr int NV = cache_values(VAR, DIM);
  constexpr int BS = layout_row<T>(DIM, N);
  // exchange buffers: entry (component c, point r of the plane, plane thread t) at (c NP + r) TP + t
  constexpr int NB = DIM * NP * TP;
  constexpr int NBU = NEED_U ? NB : 1;
  __shared__ T tD[MAXN][MAXN], tS[MAXN][MAXN], tWh[NPT], tmu[MAXMAT], tlam[MAXMAT];
  __shared__ T xb0[NB], xb1[NB];
  __shared__ T ub0[NBU], ub1[NBU];
  __shared__ __align__(8) unsigned long long bar;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  T* const cs = reinterpret_cast<T*>(dyn_smem);
  const int t = threadIdx.x;
  constexpr unsigned CHUNK = (unsigned)(NV * BS * sizeof(T));
  if (NV > 0 && t == 0) {
    // the block's cache chunk streams in (bulk copy) under the gather and the forward sweeps
    mbar_init(&bar, 1);
    bulk_load(cs, a.cache + (size_t)blk * NV * BS, CHUNK, &bar);
  }
  for (int i = t; i < MAXN * MAXN; i += blockDim.x) {
    tS[i / MAXN][i % MAXN] = a.b.S[i / MAXN][i % MAXN];
    tD[i / MAXN][i % MAXN] = a.b.D[i / MAXN][i % MAXN];
  }
  for (int i = t; i < NPT; i += blockDim.x) {
    const int q0 = i % N, q1 = (i / N) % N, q2 = i / NP;
    const T hd = T(a.g.h) * T(a.g.h) * T(a.g.h);
    tWh[i] = a.b.w[q0] * a.b.w[q1] * a.b.w[q2] * hd * T(a.g.inv_h);
  }
  for (int i = t; i < MAXMAT; i += blockDim.x) {
    tmu[i] = a.mt.mu[i];
    tlam[i] = a.mt.lam[i];
  }
  const int cl = t / N, l2 = t % N;  // plane l2 of cell cl: the k+1 threads of a cell are adjacent
  const int zb = cl * N;             // plane thread of this cell with plane index 0
  const int cell = blk * CB + cl;
  const bool active = cell < a.g.ncells;
  const int m = a.g.m;
  const int cc = active ? cell : 0;
  const int c0 = cc % m, c1 = (cc / m) % m, c2 = cc / (m * m);
  const int i2 = K * c2 + l2;
  const T sh = PHYS ? T(a.g.inv_h) : T(1);
  auto XB = [](int c, int r, int i) { return (c * NP + r) * TP + i; };
  // gather the node plane a2 = l2 (x read as zero on constrained dofs)
  uint32_t cms[NP];
  T V[NP][DIM], VU[NEED_U ? NP : 1][DIM];
#pragma unroll
  for (int a1 = 0; a1 < N; ++a1)
#pragma unroll
    for (int a0 = 0; a0 < N; ++a0) {
      const int r = a0 + N * a1;
      const int i0 = K * c0 + a0, i1 = K * c1 + a1;
      cms[r] = node_cmask<DIM>(a.g, i0, i1, i2);
      const long long node = i0 + (long long)a.g.L * (i1 + (long long)a.g.L * i2);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        V[r][c] = (active && !((cms[r] >> c) & 1u)) ? vec_in<T>(a.x[node * DIM + c]) : T(0);
        if (NEED_U) VU[NEED_U ? r : 0][c] = active ? vec_in<T>(a.ubar[node * DIM + c]) : T(0);
      }
    }
  // x, then y interpolation in registers: values at (q0, q1) of node plane l2
  {
    T X[NP][DIM], XU[NEED_U ? NP : 1][DIM];
#pragma unroll
    for (int a1 = 0; a1 < N; ++a1)
#pragma unroll
      for (int q0 = 0; q0 < N; ++q0)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          T sx = T(0), su = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            sx = fma(a.b.S[q0][j], V[j + N * a1][c], sx);
            if (NEED_U) su = fma(a.b.S[q0][j], VU[NEED_U ? j + N * a1 : 0][c], su);
          }
          X[q0 + N * a1][c] = sx;
          if (NEED_U) XU[NEED_U ? q0 + N * a1 : 0][c] = su;
        }
#pragma unroll
    for (int q1 = 0; q1 < N; ++q1)
#pragma unroll
      for (int q0 = 0; q0 < N; ++q0)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          T sx = T(0), su = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            sx = fma(a.b.S[q1][j], X[q0 + N * j][c], sx);
            if (NEED_U) su = fma(a.b.S[q1][j], XU[NEED_U ? q0 + N * j : 0][c], su);
          }
          xb0[XB(c, q0 + N * q1, t)] = sx;
          if (NEED_U) ub0[NEED_U ? XB(c, q0 + N * q1, t) : 0] = su;
        }
  }
  __syncthreads();
  // z interpolation: this thread's Gauss plane q2 = l2 from the k+1 node planes of its cell
#pragma unroll
  for (int r = 0; r < NP; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T sx = T(0), su = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        sx = fma(tS[l2][j], xb0[XB(c, r, zb + j)], sx);
        if (NEED_U) su = fma(tS[l2][j], ub0[NEED_U ? XB(c, r, zb + j) : 0], su);
      }
      V[r][c] = sx;
      if (NEED_U) VU[NEED_U ? r : 0][c] = su;
    }
#pragma unroll
  for (int r = 0; r < NP; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      xb1[XB(c, r, t)] = V[r][c];
      if (NEED_U) ub1[NEED_U ? XB(c, r, t) : 0] = VU[NEED_U ? r : 0][c];
    }
  __syncthreads();
  if (NV > 0) {
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // the copy never completed: flag it, give it one more bounded wait, leave
      if (t == 0) atomicOr(a.err, ERRBIT_TIMEOUT);
      mbar_wait(&bar, 0);
      return;
    }
  }
  // Gauss-point work on plane l2; the transposed x and y derivatives accumulate in W, the z part of the
  // flux goes to shared memory
  const int id = active ? a.mat[cell] : 0;
  T W[NP][DIM];
#pragma unroll
  for (int r = 0; r < NP; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) W[r][c] = T(0);
#pragma unroll
  for (int q1 = 0; q1 < N; ++q1)
#pragma unroll
    for (int q0 = 0; q0 < N; ++q0) {
      const int r = q0 + N * q1;
      const int p = r + NP * l2;
      T G[DIM][DIM], Gu[DIM][DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T gx = T(0), gy = T(0), gz = T(0), ux = T(0), uy = T(0), uz = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          gx = fma(a.b.D[q0][j], V[j + N * q1][c], gx);
          gy = fma(a.b.D[q1][j], V[q0 + N * j][c], gy);
          gz = fma(tD[l2][j], xb1[XB(c, r, zb + j)], gz);
          if (NEED_U) {
            ux = fma(a.b.D[q0][j], VU[NEED_U ? j + N * q1 : 0][c], ux);
            uy = fma(a.b.D[q1][j], VU[NEED_U ? q0 + N * j : 0][c], uy);
            uz = fma(tD[l2][j], ub1[NEED_U ? XB(c, r, zb + j) : 0], uz);
          }
        }
        G[c][0] = gx * sh;
        G[c][1] = gy * sh;
        G[c][2] = gz * sh;
        Gu[c][0] = ux * sh;
        Gu[c][1] = uy * sh;
        Gu[c][2] = uz * sh;
      }
      T P[DIM][DIM];
      qp_flux<DIM, VAR>(G, Gu, cs, BS, cl * NPT + p, active, id, tmu, tlam, tWh[p], P, a.mt.law);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          W[j + N * q1][c] = fma(a.b.D[q0][j], P[c][0], W[j + N * q1][c]);
          W[q0 + N * j][c] = fma(a.b.D[q1][j], P[c][1], W[q0 + N * j][c]);
        }
        xb0[XB(c, r, t)] = P[c][2];
      }
    }
  __syncthreads();
  // the z part of the transposed derivatives: Gauss plane l2 collects from the k+1 planes of its cell
#pragma unroll
  for (int r = 0; r < NP; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T s = W[r][c];
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(tD[j][l2], xb0[XB(c, r, zb + j)], s);
      xb1[XB(c, r, t)] = s;
    }
  __syncthreads();
  // transposed z interpolation (node plane l2), then y and x in registers
#pragma unroll
  for (int r = 0; r < NP; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(tS[j][l2], xb1[XB(c, r, zb + j)], s);
      W[r][c] = s;
    }
  T Y[NP][DIM];
#pragma unroll
  for (int a1 = 0; a1 < N; ++a1)
#pragma unroll
    for (int q0 = 0; q0 < N; ++q0)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(a.b.S[j][a1], W[q0 + N * j][c], s);
        Y[q0 + N * a1][c] = s;
      }
  if (active) {
#pragma unroll
    for (int a1 = 0; a1 < N; ++a1)
#pragma unroll
      for (int a0 = 0; a0 < N; ++a0) {
        const int r = a0 + N * a1;
        const long long node = (K * c0 + a0) + (long long)a.g.L * ((K * c1 + a1) + (long long)a.g.L * i2);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          if ((cms[r] >> c) & 1u) continue;
          T s = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) s = fma(a.b.S[j][a0], Y[j + N * a1][c], s);
          atomicAdd(&a.y[node * DIM + c], vec_out(s));
        }
      }
  }
}

// ---- kernels: one problem (arguments by value), or a work list of problems in one launch ----------
// Work list: problem p owns the thread blocks start[p] .. start[p+1]-1 of the grid (start[count] = grid
// size); each problem's arguments are read from global memory. The problems share dim, degree, variant
// and precision, and may differ in everything else (mesh size, material, cache, vectors).
__device__ __forceinline__ int work_item(const int* __restrict__ start, int count, int b) {
  int lo = 0, hi = count - 1;  // the last p with start[p] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM))
apply_kernel(const CellArgs<T> a) {
  apply_point_body<DIM, N, VAR, T>(a, blockIdx.x);
}

template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM))
apply_list_kernel(const CellArgs<T>* __restrict__ list, const int* __restrict__ start, int count) {
  const int p = work_item(start, count, blockIdx.x);
  apply_point_body<DIM, N, VAR, T>(list[p], blockIdx.x - start[p]);
}

// The point form in double-float stages no cache chunk and asks for three resident blocks per SM (register
// limit 85). The other precisions keep the compiler's default register budget; an explicit minimum of one
// block would let it take up to 152 registers for FP64 NC and fall to one block per SM.
template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM), 3)
apply_kernel_ff(const CellArgs<T> a) {
  apply_point_body<DIM, N, VAR, T>(a, blockIdx.x);
}

template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM), 3)
apply_list_kernel_ff(const CellArgs<T>* __restrict__ list, const int* __restrict__ start, int count) {
  const int p = work_item(start, count, blockIdx.x);
  apply_point_body<DIM, N, VAR, T>(list[p], blockIdx.x - start[p]);
}

template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM - 1))
apply_line_kernel(const CellArgs<T> a) {
  apply_line_body<DIM, N, VAR, T>(a, blockIdx.x, 1);
}

template <int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(3, N) * N)
apply_plane_kernel(const CellArgs<T> a) {
  apply_plane_body<N, VAR, T>(a, blockIdx.x);
}

template <int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(3, N) * N)
apply_plane_list_kernel(const CellArgs<T>* __restrict__ list, const int* __restrict__ start, int count) {
  const int p = work_item(start, count, blockIdx.x);
  apply_plane_body<N, VAR, T>(list[p], blockIdx.x - start[p]);
}

// persistent: gridDim.x thread blocks loop over all cell blocks, the next chunk copied in early
template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM - 1))
apply_line_persist_kernel(const CellArgs<T> a) {
  apply_line_body<DIM, N, VAR, T, true>(a, blockIdx.x, gridDim.x);
}

template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(layout_cells<T>(DIM, N) * ipow(N, DIM - 1))
apply_line_list_kernel(const CellArgs<T>* __restrict__ list, const int* __restrict__ start, int count) {
  const int p = work_item(start, count, blockIdx.x);
  apply_line_body<DIM, N, VAR, T>(list[p], blockIdx.x - start[p], 1);
}

// ------------------------------------------------------------------------------------------------
// Curved cells (an isoparametric Q_k reference map with nodal coordinates a.X64): the kernels that form
// the state from the displacement sweep the cell's coordinates like a displacement, take GX = dX/dxi at
// their Gauss point and use invJ = GX^{-1} (dxi/dX) and the volume weight w_q det GX in place of 1/h and
// w_q h^d. Every thread of the block calls qp_geometry (it synchronises); inactive threads get the
// identity map.
template <int DIM, int N, typename SM>
__device__ __forceinline__ void qp_geometry(const CellArgs<double>& a, const SM& s, const CellLoc<DIM, N>& loc,
                                            const Pt<DIM, N>& pt, bool active, double* b0, double* b1,
                                            double invJ[DIM][DIM], double& wdet) {
  constexpr int NPT = ipow(N, DIM);
  __syncthreads();  // the caller's sweep buffers are free again
#pragma unroll
  for (int c = 0; c < DIM; ++c) b0[c * NPT + pt.p] = active ? a.X64[(long long)loc.node * DIM + c] : 0.0;
  __syncthreads();
  const double* V = interp_forward<DIM, N, DIM>(b0, b1, pt, s.S);
  double GX[DIM][DIM];
  colloc_grad<DIM, N>(V, pt, s.D, GX);
  __syncthreads();
  double w = a.b.w[pt.pc[0]] * a.b.w[pt.pc[1]];
  if (DIM == 3) w *= a.b.w[pt.pc[2]];
  if (!active) {
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) invJ[i][j] = i == j ? 1.0 : 0.0;
    wdet = w;
    return;
  }
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
  const double r = 1.0 / det;
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) invJ[i][j] *= r;
  wdet = w * det;
}

// F = I + Gu invJ (Gu = du/dxi at the point); on the lattice invJ = I/h.
template <int DIM>
__device__ __forceinline__ void deformation_curved(const double Gu[DIM][DIM], const double invJ[DIM][DIM],
                                                   double F[DIM][DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int J = 0; J < DIM; ++J) {
      double v = Gu[i][0] * invJ[0][J];
#pragma unroll
      for (int L = 1; L < DIM; ++L) v = fma(Gu[i][L], invJ[L][J], v);
      F[i][J] = (i == J ? 1.0 : 0.0) + v;
    }
}

// M <- invJ M (M = F^{-1} on entry): the map from unit-cell gradients to the spatial ones.
template <int DIM>
__device__ __forceinline__ void premultiply(const double invJ[DIM][DIM], double M[DIM][DIM]) {
  double R[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      double v = invJ[i][0] * M[0][j];
#pragma unroll
      for (int L = 1; L < DIM; ++L) v = fma(invJ[i][L], M[L][j], v);
      R[i][j] = v;
    }
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) M[i][j] = R[i][j];
}

}  // namespace hy
