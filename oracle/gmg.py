"""Geometric multigrid of Sec. 6 with the smoother settings of Sec. 7, on assembled matrices.

Test infrastructure (see oracle/__init__.py).
  * transfers: standard geometric prolongation between nested Q_k spaces (coarse basis evaluated
    at fine nodes); restriction is its transpose; rows/columns of constrained dofs are zeroed.
  * level tangents: the current displacement is carried down to every level (Sec. 6) by nodal
    interpolation (reading O8) and each level operator is the tangent linearised about it.
  * smoother: Jacobi-preconditioned Chebyshev of degree 4 on [0.6 lmax, 1.2 lmax], lmax the largest
    Ritz value of 30 CG iterations on D^{-1} A (Sec. 7); one sweep per pre-/post-smoothing by default.
  * coarse level: the same Chebyshev used as a solver, with its degree chosen so that the polynomial
    bound reduces the residual by 1e-3 on the estimated spectrum [lmin, 1.2 lmax] (Sec. 7).
  * V-cycle and PCG in their textbook forms.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import gll_nodes, lagrange
from .fem import Problem
from .rng import splitmix64_uniform


def _lattice(k, m):
    g = gll_nodes(k)
    x = np.concatenate([(c + g[:k]) / m for c in range(m)] + [np.array([1.0])])
    return x


def _eval_1d(k, m_src, x_dst):
    """Matrix (len(x_dst) x (k m_src + 1)) evaluating a Q_k lattice field of m_src cells at points x_dst."""
    g = gll_nodes(k)
    M = np.zeros((len(x_dst), k * m_src + 1))
    for i, x in enumerate(x_dst):
        c = min(int(math.floor(x * m_src)), m_src - 1)
        V, _ = lagrange(g, np.array([x * m_src - c]))
        M[i, k * c : k * c + k + 1] = V[0]
    M[np.abs(M) < 1e-15] = 0.0
    return M


def prolongation_1d(k, m_coarse):
    """Coarse (m_coarse cells) to fine (2 m_coarse cells) prolongation along one axis."""
    return _eval_1d(k, m_coarse, _lattice(k, 2 * m_coarse))


def interpolation_1d(k, m_coarse):
    """Fine (2 m_coarse cells) field evaluated at the coarse lattice nodes (carries u down)."""
    return _eval_1d(k, 2 * m_coarse, _lattice(k, m_coarse))


def lattice_operator(M1, dim):
    """M1 applied along every axis of an interleaved vector field: M1 (x) ... (x) M1 (x) I_dim."""
    M = sp.csr_matrix(M1)
    for _ in range(dim - 1):
        M = sp.kron(sp.csr_matrix(M1), M)
    return sp.kron(M, sp.identity(dim)).tocsr()


def chebyshev(A, Dinv, b, x0, degree, lo, hi):
    """Jacobi-preconditioned Chebyshev iteration of the given degree on [lo, hi] (Saad, Alg. 12.1).

    Degree s means s polynomial steps; with x0 = None the start is zero and the first residual
    is b itself. Returns x.
    """
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - A @ x
    d = Dinv * r / theta
    x = x + d
    for _ in range(degree - 1):
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv * r)
        x = x + d
        rho = rho_new
    return x


def cg_ritz(A, Dinv, v, iters):
    """Ritz values of D^{-1} A from `iters` Jacobi-PCG iterations on A x = v, x0 = 0.

    Lanczos tridiagonal from the CG coefficients: T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    T_{j,j+1} = sqrt(beta_j)/alpha_j. Stops early once (r,z) <= 1e-28 (r0,z0).
    """
    r = v.copy()
    z = Dinv * r
    p = z.copy()
    rz = r @ z
    rz0 = rz
    alphas, betas = [], []
    for _ in range(iters):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        r = r - alpha * Ap
        z = Dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        if rz_new <= 1e-28 * rz0:
            break
        p = z + beta * p
        rz = rz_new
    n = len(alphas)
    T = np.zeros((n, n))
    for j in range(n):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < n:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]
    return np.linalg.eigvalsh(T)


def coarse_degree(lo, hi, reduction=1e-3):
    """Smallest s with 1 / T_s((hi+lo)/(hi-lo)) <= reduction (Chebyshev polynomial bound)."""
    sigma = (hi + lo) / (hi - lo)
    return max(1, int(math.ceil(math.acosh(1.0 / reduction) / math.acosh(sigma) - 1e-12)))


class Hierarchy:
    """Level problems from coarsest (0) to finest (L-1), each halving the cells per direction."""

    def __init__(self, dim, k, levels_m, ids, mu_tab, lam_tab, masks, degree=4, sweeps=1, smooth_lo=0.6,
                 smooth_hi=1.2, eig_iters=30, coarse_eig_iters=None, coarse_reduction=1e-3, coarse_solver="chebyshev",
                 law=0, X=None):
        self.dim, self.k = dim, k
        # a curved geometry (finest-level nodal coordinates) is carried down by the same nodal interpolation
        # as the displacement (reading O8), so every level has its own isoparametric map
        Xl = [None] * len(levels_m)
        if X is not None:
            Xl[-1] = np.asarray(X, dtype=float).reshape(-1)
            for l in range(len(levels_m) - 1, 0, -1):
                Xl[l - 1] = lattice_operator(interpolation_1d(k, levels_m[l - 1]), dim) @ Xl[l]
        self.levels = [Problem(dim, k, ml, ids[l], mu_tab, lam_tab, masks, law=law, X=Xl[l])
                       for l, ml in enumerate(levels_m)]
        self.degree, self.sweeps = degree, sweeps
        self.smooth_lo, self.smooth_hi = smooth_lo, smooth_hi
        self.eig_iters = eig_iters
        self.coarse_eig_iters = coarse_eig_iters
        self.coarse_reduction = coarse_reduction
        self.coarse_solver = coarse_solver  # "chebyshev" (Sec. 7) or "direct" (exact solve, an option)
        self.P = [None]
        self.I = [None]
        for l in range(1, len(levels_m)):
            mc = levels_m[l - 1]
            assert levels_m[l] == 2 * mc
            Pl = lattice_operator(prolongation_1d(k, mc), dim)
            zf = sp.diags(self.levels[l].free.astype(float))
            zc = sp.diags(self.levels[l - 1].free.astype(float))
            self.P.append((zf @ Pl @ zc).tocsr())
            self.I.append(lattice_operator(interpolation_1d(k, mc), dim))

    def set_displacement(self, u_fine, lmax=None, coarse_bounds=None):
        """Carry u down, linearise every level, estimate eigenvalues (or take the given ones)."""
        L = len(self.levels)
        self.u = [None] * L
        self.u[L - 1] = np.asarray(u_fine, dtype=float)
        for l in range(L - 1, 0, -1):
            self.u[l - 1] = self.I[l] @ self.u[l]
        self.A = [p.tangent(ul) for p, ul in zip(self.levels, self.u)]
        self.Dinv = [1.0 / A.diagonal() for A in self.A]
        self.lmax = [0.0] * L
        for l in range(1, L):
            if lmax is not None:
                self.lmax[l] = lmax[l]
            else:
                self.lmax[l] = self.estimate(l, self.eig_iters).max()
        if self.coarse_solver == "direct":
            self.coarse_lo = self.coarse_hi = 0.0
            self.coarse_spd = bool(np.all(np.linalg.eigvalsh(self.A[0].toarray()) > 0))
            self.coarse_deg = 0
            return
        if coarse_bounds is not None:
            self.coarse_lo, self.coarse_hi = coarse_bounds
        else:
            nfree = int(self.levels[0].free.sum())
            it = nfree if self.coarse_eig_iters is None else min(nfree, self.coarse_eig_iters)
            ritz = self.estimate(0, it)
            self.coarse_lo, self.coarse_hi = ritz.min(), self.smooth_hi * ritz.max()
        # an indefinite coarsest level (tangent about an unstable state) cannot be solved by Chebyshev;
        # the V-cycle refuses it
        self.coarse_spd = self.coarse_lo > 0
        self.coarse_deg = coarse_degree(self.coarse_lo, self.coarse_hi, self.coarse_reduction) if self.coarse_spd else 0

    def start_vector(self, l):
        v = splitmix64_uniform(l, self.levels[l].n_dofs)
        v[self.levels[l].constrained] = 0.0
        return v

    def estimate(self, l, iters):
        return cg_ritz(self.A[l], self.Dinv[l], self.start_vector(l), iters)

    def smooth(self, l, b, x0):
        lo, hi = self.smooth_lo * self.lmax[l], self.smooth_hi * self.lmax[l]
        x = x0
        for _ in range(self.sweeps):
            x = chebyshev(self.A[l], self.Dinv[l], b, x, self.degree, lo, hi)
        return x

    def vcycle(self, b, l=None):
        """One V-cycle on level l (default finest) for right-hand side b, zero initial guess."""
        if l is None:
            l = len(self.levels) - 1
            if not self.coarse_spd:
                raise ValueError("coarsest-level tangent is not positive definite")
        if l == 0:
            if self.coarse_solver == "direct":
                return spla.spsolve(self.A[0].tocsc(), b)
            return chebyshev(self.A[0], self.Dinv[0], b, None, self.coarse_deg, self.coarse_lo, self.coarse_hi)
        x = self.smooth(l, b, None)
        r = b - self.A[l] @ x
        e = self.vcycle(self.P[l].T @ r, l - 1)
        x = x + self.P[l] @ e
        return self.smooth(l, b, x)


def pcg(A, b, precond, rtol=1e-8, maxit=1000):
    """Preconditioned CG from x0 = 0; stops when ||r|| <= rtol ||b||. Returns (x, iterations, converged)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, True
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= rtol * nb:
            return x, it, True
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, False
