// Setup kernels of a linearisation: the Gauss-point state build, the residual (Eq. weak_form) and the
// operator diagonal, with the sum factorisation and Gauss-point device functions of cell_kernels.cuh. They
// live apart from the tangent action so that the action's source (cell_kernels.cuh) changes only when the
// action does.
#pragma once
#include "cell_kernels.cuh"

namespace hy {

// ------------------------------------------------------------------------------------------------
// Gauss-point state from the level displacement (FP64 kinematics F, J, ln J; Sec. 2.1, 2.3), stored
// per variant in T: T4 {M, tau~, JC~ (Voigt upper triangle)}, T2 {M, tau~, c1~, c2~}, FC {F},
// SC {mu - 2 lambda ln J}. Flags J <= 0 / NaN in the error word and tracks min J.
template <int DIM, int N, int VAR, typename T>
__global__ void __launch_bounds__(cells_per_block(DIM, N) * ipow(N, DIM))
qp_state_kernel(const CellArgs<double> a, T* __restrict__ out) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NS = nsym(DIM);
  __shared__ Smem<DIM, N, double> s;
  load_tables<DIM, N>(s, a);
  const int cl = threadIdx.x / NPT;
  const Pt<DIM, N> pt(threadIdx.x % NPT);
  const int cell = blockIdx.x * CB + cl;
  const bool active = cell < a.g.ncells;
  const CellLoc<DIM, N> loc(a.g, active ? cell : 0, pt);
  double* b0 = &s.b0[cl][0][0];
  double* b1 = &s.b1[cl][0][0];
#pragma unroll
  for (int c = 0; c < DIM; ++c) b0[c * NPT + pt.p] = active ? a.u64[(long long)loc.node * DIM + c] : 0.0;
  __syncthreads();
  const double* V = interp_forward<DIM, N, DIM>(b0, b1, pt, s.S);
  double Gu[DIM][DIM];
  colloc_grad<DIM, N>(V, pt, s.D, Gu);
  const bool curved = a.X64 != nullptr;  // the same for every thread of the grid
  double invJ[DIM][DIM], wdet = 0.0;
  if (curved) qp_geometry<DIM, N>(a, s, loc, pt, active, b0, b1, invJ, wdet);
  if (!active) return;
  const double inv_h = a.g.inv_h;
  double F[DIM][DIM];
  if (curved) {
    deformation_curved<DIM>(Gu, invJ, F);
  } else {
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int J = 0; J < DIM; ++J) F[i][J] = (i == J ? 1.0 : 0.0) + Gu[i][J] * inv_h;
  }
  const int id = a.mat[cell];
  const double mu = s.mu[id], lam = s.lam[id];
  double M[DIM][DIM], tau[NS], c1, c2;
  const double J = neo_hooke_state<DIM>(F, mu, lam, a.mt.law, curved ? wdet : s.W[pt.p], curved ? 1.0 : inv_h, false,
                                        0.0, M, tau, c1, c2);
  if (curved) premultiply<DIM>(invJ, M);
  if (!(J > 0.0)) {
    atomicOr(a.err, J != J ? ERRBIT_NAN : ERRBIT_JNEG);
  } else {
    atomicMin(a.jmin_bits, (unsigned long long)__double_as_longlong(J));
  }
  // blocked layout of the reader of this cache (its own cells per block): (block * NV + v) * BS + local
  constexpr int NVO = cache_values(VAR, DIM);
  constexpr int CBL = layout_cells<T>(DIM, N);
  constexpr int BS = layout_row<T>(DIM, N);
  const long long qg = (long long)(cell / CBL) * NVO * BS + (cell % CBL) * NPT + pt.p;
  constexpr long long st = BS;
  if (VAR == VAR_T4 || VAR == VAR_T2) {
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) out[i * st + qg] = T(M[i / DIM][i % DIM]);
#pragma unroll
    for (int i = 0; i < NS; ++i) out[(DIM * DIM + i) * st + qg] = T(tau[i]);
    if (VAR == VAR_T2) {
      out[(DIM * DIM + NS) * st + qg] = T(c1);
      out[(DIM * DIM + NS + 1) * st + qg] = T(c2);
    } else {
      // JC~ = c1~ S + c2~ I (x) I (Sec. 2.3) in Voigt form: K_ab = JC_{i(a) j(a) k(b) l(b)}
      constexpr int OFF = DIM * DIM + NS;
      int idx = 0;
#pragma unroll
      for (int al = 0; al < NS; ++al)
#pragma unroll
        for (int be = al; be < NS; ++be) {
          const int i = vi<DIM>(al), j = vj<DIM>(al), k = vi<DIM>(be), l = vj<DIM>(be);
          const double Sijkl = 0.5 * ((i == k && j == l ? 1.0 : 0.0) + (i == l && j == k ? 1.0 : 0.0));
          const double v = c1 * Sijkl + (i == j && k == l ? c2 : 0.0);
          out[(OFF + idx) * st + qg] = T(v);
          ++idx;
        }
    }
  } else if (base_variant(VAR) == VAR_FC) {
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) out[i * st + qg] = T(F[i / DIM][i % DIM]);
  } else if (base_variant(VAR) == VAR_SC) {
    double pv, jdp;
    volumetric(J, lam, a.mt.law, pv, jdp);
    out[qg] = T(mu - pv);
  }
  if (is_general(VAR)) {  // the reference map of the point: invJ (I/h on the lattice), then w_q det(dX/dxi)
    constexpr int GOFF = cache_values(base_variant(VAR), DIM);
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) {
      const int r = i / DIM, c = i % DIM;
      out[(GOFF + i) * st + qg] = T(curved ? invJ[r][c] : (r == c ? inv_h : 0.0));
    }
    out[(GOFF + DIM * DIM) * st + qg] = T(curved ? wdet : s.W[pt.p]);
  }
}

// ------------------------------------------------------------------------------------------------
// Residual r += R(u) (Eq. weak_form) in FP64: P~ = tau~ M^T integrated against the shape gradients.
// Constrained rows receive nothing (the caller zeroes r first).
template <int DIM, int N>
__global__ void __launch_bounds__(cells_per_block(DIM, N) * ipow(N, DIM))
residual_kernel(const CellArgs<double> a) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NS = nsym(DIM);
  __shared__ Smem<DIM, N, double> s;
  load_tables<DIM, N>(s, a);
  const int cl = threadIdx.x / NPT;
  const Pt<DIM, N> pt(threadIdx.x % NPT);
  const int cell = blockIdx.x * CB + cl;
  const bool active = cell < a.g.ncells;
  const CellLoc<DIM, N> loc(a.g, active ? cell : 0, pt);
  double* b0 = &s.b0[cl][0][0];
  double* b1 = &s.b1[cl][0][0];
  double* bp = &s.bp[cl][0][0];
#pragma unroll
  for (int c = 0; c < DIM; ++c) b0[c * NPT + pt.p] = active ? a.u64[(long long)loc.node * DIM + c] : 0.0;
  __syncthreads();
  const double* V = interp_forward<DIM, N, DIM>(b0, b1, pt, s.S);
  double Gu[DIM][DIM];
  colloc_grad<DIM, N>(V, pt, s.D, Gu);
  const bool curved = a.X64 != nullptr;
  double invJ[DIM][DIM], wdet = 0.0;
  if (curved) qp_geometry<DIM, N>(a, s, loc, pt, active, b0, b1, invJ, wdet);
  const double inv_h = a.g.inv_h;
  double F[DIM][DIM];
  if (curved) {
    deformation_curved<DIM>(Gu, invJ, F);
  } else {
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int J = 0; J < DIM; ++J) F[i][J] = (i == J ? 1.0 : 0.0) + Gu[i][J] * inv_h;
  }
  const int id = active ? a.mat[cell] : 0;
  double M[DIM][DIM], tau[NS], c1, c2;
  const double J = neo_hooke_state<DIM>(F, s.mu[id], s.lam[id], a.mt.law, curved ? wdet : s.W[pt.p],
                                        curved ? 1.0 : inv_h, false, 0.0, M, tau, c1, c2);
  if (curved) premultiply<DIM>(invJ, M);
  if (active && !(J > 0.0)) atomicOr(a.err, J != J ? ERRBIT_NAN : ERRBIT_JNEG);
  double tf[DIM][DIM];
#pragma unroll
  for (int al = 0; al < NS; ++al) {
    tf[vi<DIM>(al)][vj<DIM>(al)] = tau[al];
    tf[vj<DIM>(al)][vi<DIM>(al)] = tau[al];
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int Jx = 0; Jx < DIM; ++Jx) {
      double acc = tf[c][0] * M[Jx][0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) acc = fma(tf[c][j], M[Jx][j], acc);
      bp[(c * DIM + Jx) * NPT + pt.p] = active ? acc : 0.0;
    }
  __syncthreads();
  const double* Y = integrate_backward<DIM, N>(bp, b0, b1, pt, s.S, s.D);
  if (active) {
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (!((loc.cmask >> c) & 1u)) atomicAdd(&a.y[(long long)loc.node * DIM + c], Y[c * NPT + pt.p]);
  }
}

// ------------------------------------------------------------------------------------------------
// Diagonal of the tangent, d += diag A(u). For node a and component c:
//   A_{ac,ac} = sum_q W [ g_a . tau . g_a + c1 (|g_a|^2 + g_{a,c}^2)/2 + c2 g_{a,c}^2 ],  g_a = F^{-T} Grad N_a,
// the geometric and material parts of Eq. algebraic_tangent with the action of Eq. simplified_action.
//   With r = grad_xi N_a(q) the reference gradient and g_a = M^T r (M: the point's map, carrying 1/h or, on
// curved cells, the inverse Jacobian), the entry is a quadratic form in r,
//   A_{ac,ac} = sum_q sum_{J,L} r_J r_L K^c_{JL}(q),   K^c = M (tau + c1/2 I) M^T + (c1/2 + c2) m_c m_c^T,
// m_c the column c of M (weights folded into tau, c1, c2). On the tensor-product element r_J r_L is a
// product of one 1D factor per direction -- S^2, S S' or S'^2 (S the nodal basis at the Gauss points, S' its
// derivative) as the direction occurs 0, 1 or 2 times in (J, L) -- so the sum over q factorises into dim 1D
// contractions per (J, L) pair and component: (k+1)^(dim+1) multiply-adds per field and cell instead of the
// (k+1)^(2 dim) of a sum over (node, point) pairs.
//   One thread per (cell, Gauss point) forms the FP64 state and K^c; per component c the NS fields K^c_{JL}
// (J <= L, the off-diagonal pairs doubled) go to shared memory in E and are contracted along x, y (and z)
// by the same threads, which end as (cell, node) and hold the entry. E is double, or double-float (the
// FP32 pipe, about 48 significant bits).
//   SRC = 0 evaluates the state from the displacement. SRC = 1 (T4) or 2 (T2) reads M, tau~, c1~, c2~ of the
// point from the level's cache of that variant in element type E (the same cell blocks as this kernel): the
// values the state kernel wrote, with c1~ = JC~_0000 - JC~_0011 and c2~ = JC~_0011 for T4.
__device__ __forceinline__ double cached_double(double v) { return v; }
__device__ __forceinline__ double cached_double(ff v) { return (double)v.hi + (double)v.lo; }
template <int DIM, int N, typename E, int SRC = 0>
__global__ void __launch_bounds__(cells_per_block(DIM, N) * ipow(N, DIM))
diag_kernel(const CellArgs<double> a) {
  constexpr int NPT = ipow(N, DIM);
  constexpr int CB = cells_per_block(DIM, N);
  constexpr int NS = nsym(DIM);
  static_assert(sizeof(E) == sizeof(double), "E values reuse double buffers");
  static_assert(NS <= DIM * DIM && NS <= 2 * DIM, "the fields fit the flux and displacement buffers");
  __shared__ Smem<DIM, N, double> s;
  __shared__ E tab[3][MAXN][MAXN];  // tab[k][q][a] = S[q][a]^(2-k) S'[q][a]^k
  load_tables<DIM, N>(s, a);
  if (threadIdx.x < MAXN * MAXN) {
    const int q = threadIdx.x / MAXN, n = threadIdx.x % MAXN;
    const double sv = a.b.S[q][n], dv = a.b.Sd[q][n];
    tab[0][q][n] = E(sv * sv);
    tab[1][q][n] = E(sv * dv);
    tab[2][q][n] = E(dv * dv);
  }
  const int cl = threadIdx.x / NPT;
  const Pt<DIM, N> pt(threadIdx.x % NPT);
  const int cell = blockIdx.x * CB + cl;
  const bool active = cell < a.g.ncells;
  const CellLoc<DIM, N> loc(a.g, active ? cell : 0, pt);
  __syncthreads();
  double M[DIM][DIM], tau[NS], c1, c2;
  if constexpr (SRC == 0) {
    double* b0 = &s.b0[cl][0][0];
    double* b1 = &s.b1[cl][0][0];
#pragma unroll
    for (int c = 0; c < DIM; ++c) b0[c * NPT + pt.p] = active ? a.u64[(long long)loc.node * DIM + c] : 0.0;
    __syncthreads();
    const double* V = interp_forward<DIM, N, DIM>(b0, b1, pt, s.S);
    double Gu[DIM][DIM];
    colloc_grad<DIM, N>(V, pt, s.D, Gu);
    const bool curved = a.X64 != nullptr;
    double invJ[DIM][DIM], wdet = 0.0;
    if (curved) qp_geometry<DIM, N>(a, s, loc, pt, active, b0, b1, invJ, wdet);
    const double inv_h = a.g.inv_h;
    double F[DIM][DIM];
    if (curved) {
      deformation_curved<DIM>(Gu, invJ, F);
    } else {
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int J = 0; J < DIM; ++J) F[i][J] = (i == J ? 1.0 : 0.0) + Gu[i][J] * inv_h;
    }
    const int id = active ? a.mat[cell] : 0;
    neo_hooke_state<DIM>(F, s.mu[id], s.lam[id], a.mt.law, curved ? wdet : s.W[pt.p], curved ? 1.0 : inv_h, false,
                         0.0, M, tau, c1, c2);
    if (curved) premultiply<DIM>(invJ, M);
  } else {
    static_assert(SRC == 1 || SRC == 2, "T4 or T2 cache");
    constexpr int NV = cache_values(SRC == 1 ? VAR_T4 : VAR_T2, DIM);
    constexpr int BS = layout_row<E>(DIM, N);
    constexpr int NM = DIM * DIM + NS;
    static_assert(layout_cells<E>(DIM, N) == CB, "the cache's cell blocks are this kernel's");
    const E* cq = reinterpret_cast<const E*>(a.cache) + (size_t)blockIdx.x * NV * BS + cl * NPT + pt.p;
    auto rd = [&](int v) { return active ? cached_double(cq[(size_t)v * BS]) : 0.0; };
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) M[i / DIM][i % DIM] = rd(i);
#pragma unroll
    for (int al = 0; al < NS; ++al) tau[al] = rd(DIM * DIM + al);
    if (SRC == 1) {
      const double k00 = rd(NM), k01 = rd(NM + 1);
      c2 = k01;
      c1 = k00 - k01;
    } else {
      c1 = rd(NM);
      c2 = rd(NM + 1);
    }
  }
  // G = M (tau + c1/2 I) M^T (upper triangle) and kappa = c1/2 + c2
  double G[NS];
  {
    double T[DIM][DIM];
#pragma unroll
    for (int al = 0; al < NS; ++al) {
      T[vi<DIM>(al)][vj<DIM>(al)] = tau[al];
      T[vj<DIM>(al)][vi<DIM>(al)] = tau[al];
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) T[i][i] += 0.5 * c1;
    double MT[DIM][DIM];
#pragma unroll
    for (int J = 0; J < DIM; ++J)
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        double acc = M[J][0] * T[0][j];
#pragma unroll
        for (int i = 1; i < DIM; ++i) acc = fma(M[J][i], T[i][j], acc);
        MT[J][j] = acc;
      }
#pragma unroll
    for (int al = 0; al < NS; ++al) {
      const int J = vi<DIM>(al), L = vj<DIM>(al);
      double acc = MT[J][0] * M[L][0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) acc = fma(MT[J][j], M[L][j], acc);
      G[al] = acc;
    }
  }
  const double kappa = 0.5 * c1 + c2;
  // field buffers: A = the first NS rows of the cell's flux buffer, B = its two displacement buffers
  E(*A)[DIM * DIM][NPT] = reinterpret_cast<E(*)[DIM * DIM][NPT]>(&s.bp[0][0][0]);
  E(*B0)[DIM][NPT] = reinterpret_cast<E(*)[DIM][NPT]>(&s.b0[0][0][0]);
  E(*B1)[DIM][NPT] = reinterpret_cast<E(*)[DIM][NPT]>(&s.b1[0][0][0]);
  auto Bf = [&](int f, int p) -> E& { return f < DIM ? B0[cl][f][p] : B1[cl][f - DIM][p]; };
  // the 1D factor of pair al along direction d: how often d occurs in (vi, vj)
  auto fac = [](int al, int d) { return (vi<DIM>(al) == d ? 1 : 0) + (vj<DIM>(al) == d ? 1 : 0); };
  E dsum[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    __syncthreads();  // the buffers are free: the state reads (c = 0) or the last sweep (c > 0) are done
#pragma unroll
    for (int al = 0; al < NS; ++al) {
      const int J = vi<DIM>(al), L = vj<DIM>(al);
      const double k = fma(kappa * M[J][c], M[L][c], G[al]);
      A[cl][al][pt.p] = active ? E(J == L ? k : 2.0 * k) : E(0);
    }
    __syncthreads();
    // x: (q0, q1, q2) -> (a0, q1, q2), A -> B
    {
      const int a0 = pt.pc[0], base = pt.base(0);
#pragma unroll
      for (int al = 0; al < NS; ++al) {
        const int f = fac(al, 0);
        E acc = tab[f][0][a0] * A[cl][al][base];
#pragma unroll
        for (int q = 1; q < N; ++q) acc = fma(tab[f][q][a0], A[cl][al][base + q], acc);
        Bf(al, pt.p) = acc;
      }
    }
    __syncthreads();
    // y: (a0, q1, q2) -> (a0, a1, q2), B -> A; in 2D the last sweep, summed over the pairs
    {
      const int a1 = pt.pc[1], base = pt.base(1);
      E tot = E(0);
#pragma unroll
      for (int al = 0; al < NS; ++al) {
        const int f = fac(al, 1);
        E acc = tab[f][0][a1] * Bf(al, base);
#pragma unroll
        for (int q = 1; q < N; ++q) acc = fma(tab[f][q][a1], Bf(al, base + q * N), acc);
        if (DIM == 3) A[cl][al][pt.p] = acc;
        else tot = tot + acc;
      }
      if (DIM == 2) dsum[c] = tot;
    }
    if (DIM == 3) {
      __syncthreads();
      // z: (a0, a1, q2) -> (a0, a1, a2), summed over the pairs
      const int a2 = pt.pc[2], base = pt.base(2);
      E tot = E(0);
#pragma unroll
      for (int al = 0; al < NS; ++al) {
        const int f = fac(al, 2);
        E acc = tab[f][0][a2] * A[cl][al][base];
#pragma unroll
        for (int q = 1; q < N; ++q) acc = fma(tab[f][q][a2], A[cl][al][base + q * N * N], acc);
        tot = tot + acc;
      }
      dsum[c] = tot;
    }
  }
  if (active) {
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (!((loc.cmask >> c) & 1u)) atomicAdd(&a.y[(long long)loc.node * DIM + c], vec_out(dsum[c]));
  }
}

}  // namespace hy
