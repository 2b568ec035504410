"""Finite-element definitions of energy, residual, tangent and its action (Secs. 2-3, 5).

Test infrastructure (see oracle/__init__.py). Everything is computed with the full
tensor-product tables of oracle.basis (O(n^{2d}) per cell, no sum factorisation) and
integrated in the reference configuration: the paper's division by J after integrating
over the spatial configuration (Sec. 5) is the same integral, so it is absent here.

Notation (per cell K, quadrature point q, node a, component c):
  Grad N_a  = dN[q,a,:] / h           reference gradient of a shape function
  F         = I + Grad u              (Sec. 2.1)
  g_a       = F^{-T} Grad N_a         so that grad(N_a e_c) = e_c (x) g_a   (Sec. 2.1: grad = Grad . F^{-1})
  residual  R_{a,c} = sum_q w_q h^d  tau : grad^s(N_a e_c)                    (Eq. weak_form)
  tangent   A_{ac,be} = sum_q w_q h^d [ grad^s(N_a e_c) : JC : grad^s(N_b e_e)
                                      + grad(N_a e_c) : (grad(N_b e_e) . tau) ] (Eq. algebraic_tangent)
Dirichlet treatment (reading O9 / Sec. 3): the constrained operator is Z A Z + (I - Z) with
Z the diagonal mask of free dofs; residual rows of constrained dofs are zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import material
from .basis import CellTables, gauss_rule, gll_nodes, lagrange


class Problem:
    """A uniform m^dim mesh of Q_k cells on the unit square/cube with per-cell materials.

    ids: uint8 material id per cell (x fastest); mu_tab, lam_tab: per-id moduli;
    masks: per-face bitmask of constrained components, faces (-x,+x,-y,+y,-z,+z).
    """

    def __init__(self, dim, k, m, ids, mu_tab, lam_tab, masks, chunk=512, law=0, X=None):
        self.dim, self.k, self.m = dim, k, m
        self.n = k + 1
        self.h = 1.0 / m
        self.L = k * m + 1
        self.n_nodes = self.L**dim
        self.n_dofs = dim * self.n_nodes
        self.tab = CellTables(dim, k)
        self.chunk = chunk
        self.law = law  # 0: the paper's volumetric function lambda ln^2 J; 1: lambda/4 (J^2 - 1 - 2 ln J)
        # reference geometry: None = the uniform lattice of cells of side h; else the nodal coordinates
        # (n_nodes, dim) of an isoparametric Q_k map of the cells (curved cells)
        self.X = None if X is None else np.asarray(X, dtype=float).reshape(-1, dim)
        ids = np.asarray(ids)
        self.mu = np.asarray(mu_tab, dtype=float)[ids]
        self.lam = np.asarray(lam_tab, dtype=float)[ids]
        self.masks = list(masks)
        # connectivity: cell multi-index (c0,c1,..), local node multi-index (a0,a1,..), both x fastest
        n, L = self.n, self.L
        cells = np.indices((m,) * dim).reshape(dim, -1)[::-1]       # cells[i][K] = c_i
        loc = np.indices((n,) * dim).reshape(dim, -1)[::-1]         # loc[i][a]  = a_i
        gnode = np.zeros((m**dim, n**dim), dtype=np.int64)
        for i in range(dim):
            gnode += (k * cells[i][:, None] + loc[i][None, :]) * L**i
        self.cell_nodes = gnode
        self.cell_dofs = (gnode[:, :, None] * dim + np.arange(dim)[None, None, :]).reshape(m**dim, -1)
        # constrained dofs from the face masks
        lat = np.indices((L,) * dim).reshape(dim, -1)[::-1]
        cons = np.zeros((self.n_nodes, dim), dtype=bool)
        for a in range(dim):
            for side, val in ((0, 0), (1, L - 1)):
                for c in range(dim):
                    if masks[2 * a + side] >> c & 1:
                        cons[lat[a] == val, c] = True
        self.constrained = cons.reshape(-1)
        self.free = ~self.constrained

    # ---- per-cell kinematics -------------------------------------------------------------
    def _chunks(self):
        nc = self.m**self.dim
        for s in range(0, nc, self.chunk):
            yield np.arange(s, min(nc, s + self.chunk))

    def _geom(self, cells):
        """(invJ[K,q,J,I] = d xi_J / d X_I, wdV[K,q] = w_q det(dX/dxi)) of the reference map at the Gauss
        points: the uniform lattice gives I/h and w_q h^d; a curved geometry its isoparametric map."""
        nq = self.tab.w.shape[0]
        if self.X is None:
            invJ = np.broadcast_to(np.eye(self.dim) / self.h, (len(cells), nq, self.dim, self.dim))
            return invJ, np.broadcast_to(self.tab.w * self.h**self.dim, (len(cells), nq))
        XK = self.X[self.cell_nodes[cells]]                                  # [K, a, I]
        Jm = np.einsum("KaI,qaJ->KqIJ", XK, self.tab.dN)                     # dX_I / dxi_J
        det = np.linalg.det(Jm)
        if np.any(det <= 0):
            raise FloatingPointError("reference map not invertible at a quadrature point")
        return np.linalg.inv(Jm), self.tab.w[None, :] * det

    def grad_at_qp(self, v, cells):
        """Grad v[K,q,i,J] = sum_a v_{a,i} dN_a/dxi . dxi/dX for the given cells."""
        vK = v[self.cell_dofs[cells]].reshape(len(cells), -1, self.dim)
        invJ, _ = self._geom(cells)
        return np.einsum("Kai,qaL,KqLJ->KqiJ", vK, self.tab.dN, invJ)

    def deformation(self, u, cells):
        """F = I + Grad u at every quadrature point of the cells (Sec. 2.1); raises if J <= 0."""
        F = np.eye(self.dim) + self.grad_at_qp(u, cells)
        J = np.linalg.det(F)
        if np.any(J <= 0):
            raise FloatingPointError("J <= 0 at a quadrature point")
        return F

    def min_jacobian(self, u):
        return min(np.linalg.det(np.eye(self.dim) + self.grad_at_qp(u, c)).min() for c in self._chunks())

    def _qp_params(self, cells):
        nq = self.n**self.dim
        return (np.repeat(self.mu[cells][:, None], nq, axis=1), np.repeat(self.lam[cells][:, None], nq, axis=1))

    def _g(self, F, cells):
        """g[K,q,a,j] = sum_J Grad N_a[J] F^{-1}[J,j], Grad N_a = dN_a/dxi . dxi/dX."""
        Finv = np.linalg.inv(F)
        invJ, _ = self._geom(cells)
        return np.einsum("qaL,KqLJ,KqJj->Kqaj", self.tab.dN, invJ, Finv)

    # ---- energy, residual --------------------------------------------------------------------
    def energy(self, u):
        """E = sum_K sum_q psi(F_q) w_q h^d (Sec. 2.1 potential without traction term)."""
        E = 0.0
        for cells in self._chunks():
            F = self.deformation(u, cells)
            mu, lam = self._qp_params(cells)
            _, wdV = self._geom(cells)
            E += np.einsum("Kq,Kq->", material.psi(F, mu, lam, self.law), wdV)
        return E

    def face_load(self, tractions):
        """External force of dead tractions (reference configuration, per unit reference area), the surface
        term of the weak form (Eq. weak_form; the paper loads its benchmark this way, Sec. 7):
        f_{a,c} = sum over faces of t_c * int_face N_a dA, with tractions[face][c] for the faces (-x, +x, -y,
        +y, -z, +z). On a face of a cell, N_a is the product of 1D Lagrange polynomials on the GLL nodes; the
        integral uses the (k+1)-point Gauss rule along every in-face axis."""
        t = np.asarray(tractions, dtype=float).reshape(2 * self.dim, self.dim)
        xg, wg = gauss_rule(self.n)
        V, _ = lagrange(gll_nodes(self.k), xg)  # V[q, j] = l_j(xg_q)
        f = np.zeros(self.n_nodes * self.dim)
        n, m, L, dim = self.n, self.m, self.L, self.dim
        for face in range(2 * dim):
            if not np.any(t[face]):
                continue
            ax, side = face // 2, face % 2
            inplane = [i for i in range(dim) if i != ax]
            # every cell on the face and every node of the cell on the face
            for cidx in np.ndindex(*([m] * (dim - 1))):
                c = [0] * dim
                for i, ci in zip(inplane, cidx):
                    c[i] = ci
                c[ax] = 0 if side == 0 else m - 1
                for aidx in np.ndindex(*([n] * (dim - 1))):
                    a = [0] * dim
                    for i, ai in zip(inplane, aidx):
                        a[i] = ai
                    a[ax] = 0 if side == 0 else n - 1
                    # int over the cell face of prod_i l_{a_i}(x_i): a product of 1D Gauss sums
                    wgt = self.h ** (dim - 1)
                    for i in inplane:
                        wgt *= float(np.dot(wg, V[:, a[i]]))
                    node = sum((self.k * c[i] + a[i]) * L**i for i in range(dim))
                    f[node * dim:(node + 1) * dim] += wgt * t[face]
        return f

    def residual_raw(self, u):
        """R_i = sum_K sum_q tau : grad^s N_i w_q h^d for every dof, constrained rows included (Eq. weak_form)."""
        R = np.zeros(self.n_dofs)
        for cells in self._chunks():
            F = self.deformation(u, cells)
            mu, lam = self._qp_params(cells)
            tau = material.kirchhoff(F, mu, lam, self.law)
            g = self._g(F, cells)
            # tau : grad^s(N_a e_c) = tau : grad(N_a e_c) (tau symmetric) = sum_j tau_cj g_a,j
            _, wdV = self._geom(cells)
            RK = np.einsum("Kqcj,Kqaj,Kq->Kac", tau, g, wdV)
            np.add.at(R, self.cell_dofs[cells].reshape(-1), RK.reshape(-1))
        return R

    def residual(self, u):
        """Residual with constrained rows set to zero."""
        R = self.residual_raw(u)
        R[self.constrained] = 0.0
        return R

    # ---- tangent --------------------------------------------------------------------------------
    def _local_tangent(self, u, cells):
        """Element tangent matrices [K, a*d+c, b*d+e] from Eq. algebraic_tangent, literal double contractions."""
        d = self.dim
        F = self.deformation(u, cells)
        mu, lam = self._qp_params(cells)
        tau = material.kirchhoff(F, mu, lam, self.law)
        JC = material.spatial_tangent(F, mu, lam, self.law)
        ga = self._g(F, cells)
        I = np.eye(d)
        G = np.einsum("ic,Kqaj->Kqacij", I, ga)                         # grad(N_a e_c)_{ij} = d_ic g_a,j
        Gs = 0.5 * (G + np.swapaxes(G, -1, -2))                           # grad^s(N_a e_c)
        _, w = self._geom(cells)
        # (optimize=True only lets numpy pick the contraction order of these library contractions)
        CGs = np.einsum("Kqijkl,Kqbekl->Kqijbe", JC, Gs, optimize=True)  # JC : grad^s(N_b e_e)
        mat = np.einsum("Kqacij,Kqijbe,Kq->Kacbe", Gs, CGs, w, optimize=True)
        Gt = np.einsum("Kqbeim,Kqmj->Kqbeij", G, tau, optimize=True)    # grad(N_b e_e) . tau
        geo = np.einsum("Kqacij,Kqbeij,Kq->Kacbe", G, Gt, w, optimize=True)
        nloc = self.cell_dofs.shape[1]
        return (mat + geo).reshape(len(cells), nloc, nloc)

    def tangent_raw(self, u):
        """Assembled tangent A (scipy CSR), no boundary conditions applied."""
        rows, cols, vals = [], [], []
        for cells in self._chunks():
            AK = self._local_tangent(u, cells)
            dofs = self.cell_dofs[cells]
            rows.append(np.repeat(dofs[:, :, None], dofs.shape[1], axis=2).reshape(-1))
            cols.append(np.repeat(dofs[:, None, :], dofs.shape[1], axis=1).reshape(-1))
            vals.append(AK.reshape(-1))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_dofs, self.n_dofs))
        return A.tocsr()

    def constrain(self, A):
        """Z A Z + (I - Z): identity rows/columns on constrained dofs."""
        z = self.free.astype(float)
        Z = sp.diags(z)
        return (Z @ A @ Z + sp.diags(1.0 - z)).tocsr()

    def tangent(self, u):
        return self.constrain(self.tangent_raw(u))

    def apply(self, u, x, constrained=True):
        """Element-by-element action y = A(u) x of Eq. mf_vmult (no assembled matrix).

        Per cell and quadrature point: grad x = Grad x . F^{-1}; Q = grad x . tau + JC : grad^s x;
        y_{a,c} += w_q h^d grad(N_a e_c) : Q = w_q h^d sum_j g_a,j Q_cj.
        With constrained=True, x is read as zero on constrained dofs and y_c = x_c there.
        """
        xin = np.where(self.constrained, 0.0, x) if constrained else np.asarray(x, dtype=float)
        y = np.zeros(self.n_dofs)
        for cells in self._chunks():
            self.apply_cells(u, xin, cells, y)
        if constrained:
            y[self.constrained] = x[self.constrained]
        return y

    def apply_cells(self, u, xin, cells, y):
        """Adds the contributions of the given cells to y (the loop body of apply; xin already has the
        constrained entries zeroed if they are to be read as zero)."""
        F = self.deformation(u, cells)
        mu, lam = self._qp_params(cells)
        tau = material.kirchhoff(F, mu, lam, self.law)
        JC = material.spatial_tangent(F, mu, lam, self.law)
        Finv = np.linalg.inv(F)
        gx = np.einsum("KqiJ,KqJj->Kqij", self.grad_at_qp(xin, cells), Finv)
        gxs = 0.5 * (gx + np.swapaxes(gx, -1, -2))
        Q = np.einsum("Kqim,Kqmj->Kqij", gx, tau) + np.einsum("Kqijkl,Kqkl->Kqij", JC, gxs)
        ga = self._g(F, cells)
        _, wdV = self._geom(cells)
        yK = np.einsum("Kqaj,Kqcj,Kq->Kac", ga, Q, wdV)
        np.add.at(y, self.cell_dofs[cells].reshape(-1), yK.reshape(-1))

    def diagonal(self, u):
        """diag of the constrained tangent, summed element by element (1 on constrained dofs)."""
        d = self.dim
        D = np.zeros(self.n_dofs)
        for cells in self._chunks():
            F = self.deformation(u, cells)
            mu, lam = self._qp_params(cells)
            tau = material.kirchhoff(F, mu, lam, self.law)
            JC = material.spatial_tangent(F, mu, lam, self.law)
            ga = self._g(F, cells)
            I = np.eye(d)
            G = np.einsum("ic,Kqaj->Kqacij", I, ga)
            Gs = 0.5 * (G + np.swapaxes(G, -1, -2))
            _, w = self._geom(cells)
            mat = np.einsum("Kqacij,Kqijkl,Kqackl,Kq->Kac", Gs, JC, Gs, w)
            geo = np.einsum("Kqaj,Kqmj,Kqam,Kq->Ka", ga, tau, ga, w)  # d_cc = 1: same for every c
            DK = mat + geo[:, :, None]
            np.add.at(D, self.cell_dofs[cells].reshape(-1), DK.reshape(-1))
        D[self.constrained] = 1.0
        return D
