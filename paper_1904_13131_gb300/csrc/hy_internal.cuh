// Internal definitions shared by the CUDA translation units of libhyperelastic.
//
// Mesh model: uniform m^dim Cartesian cells of side h = 1/m on the unit square/cube, Q_k Lagrange
// elements on Gauss-Lobatto-Legendre nodes, (k+1)^dim Gauss points per cell (Sec. 7, Tables 1-2:
// q = p + 1). Vectors live on the (k m + 1)^dim node lattice, x fastest, the dim displacement
// components of a node interleaved (dof = node * dim + comp). A cell gathers (k+1)^{dim-1} contiguous
// runs of (k+1)*dim values, so no index array is stored.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ff.cuh"

namespace hy {

constexpr int MAXN = 5;      // polynomial degree <= 4
constexpr int MAXMAT = 16;   // materials per level

// Sizes of the per-Gauss-point caches of the tangent variants (Algorithms 1-3 and the two
// cached/recomputed variants), as a function of dim.
//   The variants that form the state inside the action (FC, SC, NC) come in two builds. The plain one
// assumes the uniform lattice (1/h and w_q h^d as constants) and the paper's volumetric function. The
// general one (FCG, SCG, NCG) reads the reference map of its Gauss point from the cache -- the inverse
// Jacobian d xi / d X (dim^2 values) and the volume weight w_q det(dX/dxi), as the paper's matrix-free
// operators keep the mapping data of curved cells per quadrature point -- and evaluates the material's
// volumetric function chosen at run time: curved cells and the second law. (Index 5 is VAR_NONE, the
// state kernel that only checks J.)
enum Variant { VAR_T4 = 0, VAR_T2 = 1, VAR_FC = 2, VAR_SC = 3, VAR_NC = 4, VAR_FCG = 6, VAR_SCG = 7, VAR_NCG = 8 };

__host__ __device__ constexpr bool is_general(int var) { return var >= VAR_FCG; }
__host__ __device__ constexpr int base_variant(int var) { return is_general(var) ? var - VAR_FCG + VAR_FC : var; }
__host__ __device__ constexpr int nsym(int dim) { return dim == 3 ? 6 : 3; }
__host__ __device__ constexpr int cache_values(int var, int dim) {
  return is_general(var) ? cache_values(base_variant(var), dim) + dim * dim + 1
       : var == VAR_T4 ? dim * dim + nsym(dim) + nsym(dim) * (nsym(dim) + 1) / 2
       : var == VAR_T2 ? dim * dim + nsym(dim) + 2
       : var == VAR_FC ? dim * dim
       : var == VAR_SC ? 1
       : 0;
}

// 1D tables of the Q_k element on [0,1] (built on the host in double, converted to T).
template <typename T>
struct Basis1D {
  T S[MAXN][MAXN];   // S[q][a]  = l_a(xg_q): GLL-nodal basis at Gauss point q
  T D[MAXN][MAXN];   // D[q][p]  = derivative at xg_q of the Lagrange polynomial through the Gauss points, p
  T Sd[MAXN][MAXN];  // Sd[q][a] = l_a'(xg_q)
  T w[MAXN];         // Gauss weights on [0,1]
};

// Geometry of one level.
struct Geom {
  int m;             // cells per direction
  int L;             // lattice nodes per direction = k m + 1
  int ncells;        // m^dim
  uint32_t fm[6];    // constrained-component bitmask per face (-x,+x,-y,+y,-z,+z)
  double h;          // cell size
  double inv_h;      // 1 / h
};

template <typename T>
struct Mat {
  T mu[MAXMAT];
  T lam[MAXMAT];
  int law;  // volumetric function: 0 the paper's lambda ln^2 J, 1 lambda/4 (J^2 - 1 - 2 ln J)
};

// Bitmask of the constrained components of lattice node (i0, i1, i2).
template <int DIM>
__device__ __forceinline__ uint32_t node_cmask(const Geom& g, int i0, int i1, int i2) {
  uint32_t r = 0;
  if (i0 == 0) r |= g.fm[0];
  if (i0 == g.L - 1) r |= g.fm[1];
  if (i1 == 0) r |= g.fm[2];
  if (i1 == g.L - 1) r |= g.fm[3];
  if (DIM == 3) {
    if (i2 == 0) r |= g.fm[4];
    if (i2 == g.L - 1) r |= g.fm[5];
  }
  return r;
}

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Cells per thread block for the cell kernels (thread per Gauss point / node, ~256 threads).
__host__ __device__ constexpr int cells_per_block(int dim, int n) {
  return (256 / ipow(n, dim)) < 1 ? 1 : (256 / ipow(n, dim));
}

// Gauss-point caches are stored per thread block of the cell kernels: block b holds, for every cached
// value v, the CB * NPT entries of its cells contiguously, padded to a multiple of 4 elements so that
// every row and every block's chunk starts on a 16-byte boundary (the granularity of a bulk copy):
//   index(b, v, t) = (b * NV + v) * BS + t,   BS = cache_row(dim, n),   t = local cell * NPT + q.
__host__ __device__ constexpr int cache_row(int dim, int n) {
  return (cells_per_block(dim, n) * ipow(n, dim) + 3) / 4 * 4;
}

// Cells per block of the tangent action and of its cache layout, per element type. Both forms of the
// action -- one thread per (cell, Gauss point) and one thread per x-line of a cell -- process the same
// cells per block for a given element type, so they read the same cache and the autotuner (csrc/capi.cu)
// can switch forms without rebuilding it. FP64 and double-float, bound by arithmetic, take ~256 threads in
// the point form (256 / (k+1)^dim cells); FP32, bound by memory latency, takes ~128 threads in the line
// form (128 / (k+1)^(dim-1) cells), which lets more blocks stream their cache chunks per SM.
template <typename T>
__host__ __device__ constexpr int layout_cells(int dim, int n) {
  return sizeof(T) == 4 ? ((128 / ipow(n, dim - 1)) < 1 ? 1 : (128 / ipow(n, dim - 1))) : cells_per_block(dim, n);
}
template <typename T>
__host__ __device__ constexpr int layout_row(int dim, int n) {
  return (layout_cells<T>(dim, n) * ipow(n, dim) + 3) / 4 * 4;
}

// Kernel forms of the tangent action: thread per (cell, Gauss point); thread per x-line of a cell; the line
// form as a persistent grid whose blocks copy their next cache chunk in while they finish the current one
// (FP32 only: elsewhere it runs as FORM_LINE); thread per z-plane of a cell (FP32 in 3D only: elsewhere it
// runs as FORM_LINE).
enum KernelForm { FORM_POINT = 0, FORM_LINE = 1, FORM_LINE_PERSIST = 2, FORM_PLANE = 3 };

// Device-side error word bits.
enum : unsigned { ERRBIT_JNEG = 1u, ERRBIT_NAN = 2u, ERRBIT_TIMEOUT = 4u, ERRBIT_NONSPD = 8u };

// A bounded mbarrier wait gives up after MBAR_WAIT_NS of GPU wall time (the global timer) or
// MBAR_POLL_LIMIT polls, whichever comes first: seconds, far above any real copy time.
constexpr unsigned MBAR_POLL_LIMIT = 1u << 24;
constexpr unsigned long long MBAR_WAIT_NS = 4000000000ull;

}  // namespace hy
