"""Pins of oracle.fem against what the paper and the mathematics fix (Secs. 2-3, 5).

  * R(0) = 0 exactly, R(finite rigid rotation) ~ 0           (tau = 0 when b = I)
  * affine patch test: nodal reactions in closed form          (divergence theorem, GLL weights)
  * R = dE/du and A = dR/du by central differences            (Eqs. weak_form, tangent)
  * symmetry of A, translations in ker A(u), rotations in ker A(0)
  * small-strain limit: A(0) equals an exactly integrated (sympy) linear-elasticity stiffness with
    Lame (mu, 2 lambda) -- the paper's psi carries lambda ln^2 J (Sec. 2.3) -- and (mu, lambda) for the
    second volumetric function lambda/4 (J^2 - 1 - 2 ln J)
  * brute force: pure-Python loops over every index on one cell
"""
import itertools
import math

import numpy as np
import pytest

from oracle import material
from oracle.basis import CellTables
from oracle.fem import Problem
from paper_1904_13131_gb300 import inputs


def make(dim, k, m, ratio=10.0, masks=None, uniform=False):
    mu, lam = inputs.material_table(ratio)
    ids = np.zeros(m**dim, np.uint8) if uniform else inputs.inclusion_ids(dim, m)
    return Problem(dim, k, m, ids, mu, lam, masks if masks is not None else [0] * (2 * dim))


def coords(p):
    return inputs.node_coords(p.dim, p.k, p.m)


@pytest.mark.parametrize("dim,k,m", [(2, 1, 3), (2, 3, 2), (3, 2, 2)])
def test_zero_residual_at_rest_and_rigid_rotation(dim, k, m):
    p = make(dim, k, m)
    assert np.all(p.residual_raw(np.zeros(p.n_dofs)) == 0.0)
    th = 0.5
    Q = np.eye(dim)
    Q[:2, :2] = [[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]
    if dim == 3:
        R2 = np.eye(3)
        R2[1:, 1:] = [[math.cos(0.3), -math.sin(0.3)], [math.sin(0.3), math.cos(0.3)]]
        Q = Q @ R2
    X = coords(p)
    u = (X @ (Q - np.eye(dim)).T).reshape(-1)
    assert np.abs(p.residual_raw(u)).max() < 1e-13


def _gll_weights_unit(k):
    """Closed form w_j = 2 / (k (k+1) P_k(x_j)^2) on [-1,1], halved for [0,1]."""
    from numpy.polynomial import legendre
    x = 2 * inputs.gll_unit(k) - 1
    Pk = legendre.Legendre.basis(k)(x)
    return 1.0 / (k * (k + 1) * Pk**2)


@pytest.mark.parametrize("dim,k,m", [(2, 2, 3), (2, 4, 2), (3, 1, 3), (3, 3, 1)])
def test_affine_patch_reactions(dim, k, m):
    p = make(dim, k, m, uniform=True)
    rng = np.random.default_rng(5)
    H = 0.1 * rng.standard_normal((dim, dim))
    u = (coords(p) @ H.T).reshape(-1)
    R = p.residual_raw(u).reshape(-1, dim)
    P = material.piola(np.eye(dim) + H, 1.0, inputs.lame_lambda(1.0, 0.3))
    # integral of each 1D lattice hat function, from GLL weights in closed form
    wg = _gll_weights_unit(k) / m
    W1 = np.zeros(p.L)
    for c in range(m):
        W1[k * c : k * c + k + 1] += wg
    idx = np.indices((p.L,) * dim).reshape(dim, -1)[::-1]
    expect = np.zeros((p.n_nodes, dim))
    for J in range(dim):
        other = np.prod([W1[idx[a]] for a in range(dim) if a != J], axis=0)
        sgn = (idx[J] == p.L - 1).astype(float) - (idx[J] == 0).astype(float)
        expect += np.outer(other * sgn, P[:, J])
    np.testing.assert_allclose(R, expect, atol=1e-13)


@pytest.mark.parametrize("dim,k,m", [(2, 2, 3), (3, 1, 2), (3, 2, 1)])
def test_residual_is_energy_gradient(dim, k, m):
    p = make(dim, k, m)
    u = inputs.smooth_field(dim, k, m, seed=3, amplitude=0.08)
    v = inputs.gaussian_vector(p.n_dofs, 4)
    R = p.residual_raw(u)
    g = R @ v
    errs = []
    for eps in (4e-5, 2e-5):
        fd = (p.energy(u + eps * v) - p.energy(u - eps * v)) / (2 * eps)
        errs.append(abs(fd - g))
    assert errs[1] < 1e-6 * np.linalg.norm(R) * np.linalg.norm(v)
    assert errs[1] < 0.3 * errs[0]


@pytest.mark.parametrize("dim,k,m", [(2, 2, 3), (2, 3, 2), (3, 1, 2), (3, 2, 1)])
def test_tangent_is_residual_derivative(dim, k, m):
    p = make(dim, k, m)
    u = inputs.smooth_field(dim, k, m, seed=6, amplitude=0.08)
    v = inputs.gaussian_vector(p.n_dofs, 7)
    Av = p.tangent_raw(u) @ v
    errs = []
    for eps in (2e-4, 1e-4):
        fd = (p.residual_raw(u + eps * v) - p.residual_raw(u - eps * v)) / (2 * eps)
        errs.append(np.abs(fd - Av).max())
    assert errs[1] < 1e-5 * np.abs(Av).max()
    assert 3.0 < errs[0] / errs[1] < 5.0  # error ~ eps^2


@pytest.mark.parametrize("dim,k,m", [(2, 2, 4), (3, 2, 2)])
def test_symmetry_and_kernel(dim, k, m):
    p = make(dim, k, m)
    u = inputs.smooth_field(dim, k, m, seed=8)
    A = p.tangent_raw(u)
    v, w = inputs.gaussian_vector(p.n_dofs, 1), inputs.gaussian_vector(p.n_dofs, 2)
    nA = abs(A).max()
    assert abs(v @ (A @ w) - w @ (A @ v)) < 1e-13 * np.linalg.norm(v) * np.linalg.norm(w) * nA * 10
    for c in range(dim):  # translations at any u
        t = np.zeros((p.n_nodes, dim)); t[:, c] = 1.0
        assert np.abs(A @ t.reshape(-1)).max() < 1e-12 * nA
    A0 = p.tangent_raw(np.zeros(p.n_dofs))
    X = coords(p)
    for a, b in itertools.combinations(range(dim), 2):  # infinitesimal rotations at u = 0
        W = np.zeros((dim, dim)); W[a, b], W[b, a] = 1.0, -1.0
        assert np.abs(A0 @ (X @ W.T).reshape(-1)).max() < 1e-12 * nA
    # the constrained operator keeps symmetry and has unit rows on constrained dofs
    p2 = make(dim, k, m, masks=inputs.face_masks(dim, top=inputs.normal_top_mask(dim)))
    Ac = p2.tangent(u)
    assert abs(Ac - Ac.T).max() < 1e-12 * nA
    np.testing.assert_allclose(Ac.diagonal()[p2.constrained], 1.0)


def _sympy_linear_elastic_cell(dim, k, mu, lam):
    sympy = pytest.importorskip("sympy")
    xs = sympy.symbols("x0:%d" % dim)
    nodes = [sympy.Rational(j, k) for j in range(k + 1)]  # equispaced = GLL for k <= 2

    def l1(j, x):
        return sympy.prod([(x - nodes[m_]) / (nodes[j] - nodes[m_]) for m_ in range(k + 1) if m_ != j])

    n = k + 1
    Ns = []
    for a in range(n**dim):
        at = [(a // n**i) % n for i in range(dim)]
        Ns.append(sympy.prod([l1(at[i], xs[i]) for i in range(dim)]))
    dN = [[sympy.diff(N, xs[J]) for J in range(dim)] for N in Ns]

    def integ(e):
        for x in xs:
            e = sympy.integrate(sympy.expand(e), (x, 0, 1))
        return float(e)

    nl = n**dim * dim
    K = np.zeros((nl, nl))
    for a in range(n**dim):
        for b in range(a, n**dim):
            grad_dot = integ(sum(dN[a][J] * dN[b][J] for J in range(dim)))
            for c in range(dim):
                for e in range(dim):
                    val = lam * integ(dN[a][c] * dN[b][e]) + mu * integ(dN[a][e] * dN[b][c])
                    if c == e:
                        val += mu * grad_dot
                    K[a * dim + c, b * dim + e] = val
                    K[b * dim + e, a * dim + c] = val
    return K


@pytest.mark.parametrize("law,lame2", [(0, 2.0), (1, 1.0)])
@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1)])
def test_small_strain_limit_matches_exact_linear_elasticity(dim, k, law, lame2):
    """The paper's law linearises to Lame (mu, 2 lambda); the second volumetric function to (mu, lambda)."""
    p = make(dim, k, 1, uniform=True)
    p.law = law
    mu, lam = 1.0, inputs.lame_lambda(1.0, 0.3)
    A0 = p.tangent_raw(np.zeros(p.n_dofs)).toarray()
    K = _sympy_linear_elastic_cell(dim, k, mu, lame2 * lam)
    np.testing.assert_allclose(A0, K, atol=1e-13 * np.abs(K).max())


def _brute_cell(dim, k, u_cell, mu, lam, law=0):
    """Residual and tangent of one unit cell with explicit loops over every index."""
    t = CellTables(dim, k)
    na = (k + 1) ** dim
    R = np.zeros(na * dim)
    A = np.zeros((na * dim, na * dim))
    for q in range(na):
        F = np.eye(dim)
        for a in range(na):
            for i in range(dim):
                for J in range(dim):
                    F[i, J] += u_cell[a * dim + i] * t.dN[q, a, J]
        Finv = np.linalg.inv(F)
        J_ = np.linalg.det(F)
        b = F @ F.T
        pv = 2 * lam * math.log(J_) if law == 0 else 0.5 * lam * (J_ * J_ - 1.0)  # J U'(J)
        jdp = 2 * lam if law == 0 else lam * J_ * J_                             # J d(J U')/dJ
        tau = mu * b - (mu - pv) * np.eye(dim)
        cc = 2 * (mu - pv)
        g = np.zeros((na, dim))
        for a in range(na):
            for j in range(dim):
                for J in range(dim):
                    g[a, j] += t.dN[q, a, J] * Finv[J, j]
        for a in range(na):
            for c in range(dim):
                for j in range(dim):
                    R[a * dim + c] += t.w[q] * tau[c, j] * g[a, j]
        for a in range(na):
            for c in range(dim):
                for b_ in range(na):
                    for e in range(dim):
                        s = 0.0
                        for i in range(dim):
                            for j in range(dim):
                                gi = (g[a, j] if i == c else 0.0)
                                gs_i = 0.5 * ((g[a, j] if i == c else 0.0) + (g[a, i] if j == c else 0.0))
                                for kk in range(dim):
                                    for ll in range(dim):
                                        gs_j = 0.5 * ((g[b_, ll] if kk == e else 0.0) + (g[b_, kk] if ll == e else 0.0))
                                        Cijkl = cc * 0.5 * ((i == kk) * (j == ll) + (i == ll) * (j == kk)) \
                                            + jdp * (i == j) * (kk == ll)
                                        s += gs_i * Cijkl * gs_j
                                # geometric: grad(N_a e_c)_{ij} (grad(N_b e_e) . tau)_{ij}
                                gt = sum((g[b_, mm] if i == e else 0.0) * tau[mm, j] for mm in range(dim))
                                s += gi * gt
                        A[a * dim + c, b_ * dim + e] += t.w[q] * s
    return R, A


@pytest.mark.parametrize("law", [0, 1])
@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1)])
def test_brute_force_single_cell(dim, k, law):
    p = make(dim, k, 1, uniform=True)
    p.law = law
    u = 0.1 * inputs.gaussian_vector(p.n_dofs, 11)
    mu, lam = 1.0, inputs.lame_lambda(1.0, 0.3)
    R, A = _brute_cell(dim, k, u, mu, lam, law)
    np.testing.assert_allclose(p.residual_raw(u), R, atol=1e-13)
    np.testing.assert_allclose(p.tangent_raw(u).toarray(), A, atol=1e-12)


@pytest.mark.parametrize("dim,k,m", [(2, 2, 3), (3, 2, 2)])
def test_element_apply_and_diagonal_match_assembled(dim, k, m):
    p = make(dim, k, m, masks=inputs.face_masks(dim, top=inputs.normal_top_mask(dim)))
    u = inputs.smooth_field(dim, k, m, seed=2)
    x = inputs.gaussian_vector(p.n_dofs, 3)
    A = p.tangent(u)
    np.testing.assert_allclose(p.apply(u, x), A @ x, atol=1e-13 * np.abs(A @ x).max())
    np.testing.assert_allclose(p.diagonal(u), A.diagonal(), atol=1e-14 * abs(A).max())


@pytest.mark.parametrize("k,m", [(1, 4), (2, 3), (3, 2)])
def test_sampled_action_from_the_cells_of_each_node(k, m):
    """The sampled-output check of the largest meshes: y at a dof from only the cells holding its node
    (apply_cells) equals the full element-by-element action there; the cell lists match a brute-force
    search of the connectivity."""
    from paper_1904_13131_gb300 import inputs

    from .mesh_util import cells_of_node
    pr = inputs.problem(3, k, m, top=0)
    P = Problem(3, k, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
    L = k * m + 1
    for node in range(P.n_nodes):
        idx = (node % L, (node // L) % L, node // (L * L))
        assert sorted(cells_of_node(k, m, idx)) == np.nonzero((P.cell_nodes == node).any(axis=1))[0].tolist()
    u = inputs.smooth_field(3, k, m, seed=0)
    x = inputs.gaussian_vector(P.n_dofs, 1)
    full = P.apply(u, x)
    dofs = np.arange(0, P.n_dofs, 7)
    cells = sorted({c for d in dofs for c in cells_of_node(k, m, ((d // 3) % L, (d // 3 // L) % L, d // 3 // (L * L)))})
    y = np.zeros(P.n_dofs)
    P.apply_cells(u, np.where(P.constrained, 0.0, x), np.array(cells), y)
    sampled = np.where(P.constrained[dofs], x[dofs], y[dofs])
    np.testing.assert_allclose(sampled, full[dofs], rtol=1e-13, atol=1e-13 * np.abs(full).max())
