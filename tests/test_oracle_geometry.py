"""Pins of the oracle on curved (isoparametric) cells (the paper's meshes are curved, Sec. 7).

* Patch test: on a curved mesh of one material, an affine displacement u = A X + b gives a uniform F =
  I + A, so the internal forces vanish at every node not on the boundary (a Q_k map reproduces fields
  linear in X exactly).
* A finite rotation u = (Q - I) X gives F = Q and zero internal forces everywhere.
* Volume: the bump vanishes on the boundary, so the curved mesh still fills the unit square / cube; under a
  uniform F the stored energy is psi(F) times that volume (1), which pins the weights det(dX/dxi).
* Energy -> residual and residual -> tangent by central differences on the curved mesh (second-order
  error ratio), which ties the volume weights det(dX/dxi) and the gradients dxi/dX together.
* With the lattice coordinates passed explicitly, the results equal the uniform-lattice path.
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.material import psi
from paper_1904_13131_gb300 import inputs


def make(dim, k, m, X=None, uniform=False, masks=None):
    mu, lam = inputs.material_table(10.0)
    ids = np.zeros(m**dim, np.uint8) if uniform else inputs.inclusion_ids(dim, m)
    return Problem(dim, k, m, ids, mu, lam, masks if masks is not None else [0] * (2 * dim), X=X)


@pytest.mark.parametrize("dim,k,m", [(2, 1, 4), (2, 2, 3), (2, 3, 2), (3, 1, 3), (3, 2, 2)])
def test_affine_patch_and_rotation_on_curved_cells(dim, k, m):
    X = inputs.curved_coords(dim, k, m)
    p = make(dim, k, m, X=X, uniform=True)
    rng = np.random.default_rng(dim + k)
    A = 0.05 * rng.standard_normal((dim, dim))
    u = (X @ A.T + 0.01).reshape(-1)
    R = p.residual_raw(u).reshape(-1, dim)
    lat = inputs.node_coords(dim, k, m)
    interior = np.all((lat > 1e-12) & (lat < 1 - 1e-12), axis=1)
    assert np.abs(R[~interior]).max() > 1e-6  # the boundary carries the reactions
    np.testing.assert_allclose(R[interior], 0.0, atol=1e-13)
    th = 0.4
    Q = np.eye(dim)
    Q[:2, :2] = [[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]
    ur = (X @ (Q - np.eye(dim)).T).reshape(-1)
    np.testing.assert_allclose(p.residual_raw(ur), 0.0, atol=1e-13)


@pytest.mark.parametrize("dim,k,m", [(2, 1, 4), (2, 3, 2), (3, 2, 2)])
def test_energy_of_a_uniform_deformation_is_psi_times_the_volume(dim, k, m):
    X = inputs.curved_coords(dim, k, m)
    p = make(dim, k, m, X=X, uniform=True)
    A = 0.08 * np.random.default_rng(7 + dim).standard_normal((dim, dim))
    F = np.eye(dim) + A
    mu, lam = inputs.material_table(10.0)
    np.testing.assert_allclose(p.energy((X @ A.T).reshape(-1)), psi(F, mu[0], lam[0]), rtol=1e-13)
    # the curved mesh is not the lattice: a field that is not affine in X integrates differently
    q = (np.sin(3.0 * X) * 0.02).reshape(-1)
    assert abs(p.energy(q) - make(dim, k, m, uniform=True).energy(q)) > 1e-8


@pytest.mark.parametrize("dim,k,m", [(2, 2, 3), (3, 1, 2)])
def test_finite_differences_on_curved_cells(dim, k, m):
    X = inputs.curved_coords(dim, k, m)
    p = make(dim, k, m, X=X)
    u = inputs.smooth_field(dim, k, m, seed=9, amplitude=0.03)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(p.n_dofs)
    R = p.residual_raw(u)
    errs = []
    for eps in (4e-5, 2e-5):
        fd = (p.energy(u + eps * d) - p.energy(u - eps * d)) / (2 * eps)
        errs.append(abs(fd - R @ d))
    assert errs[1] < 1e-5 * np.linalg.norm(R) * np.linalg.norm(d) and 3.0 < errs[0] / errs[1] < 5.0  # ~ eps^2
    A = p.tangent_raw(u)
    errs = []
    for eps in (2e-4, 1e-4):
        fd = (p.residual_raw(u + eps * d) - p.residual_raw(u - eps * d)) / (2 * eps)
        errs.append(np.linalg.norm(fd - A @ d))
    assert errs[1] < 1e-5 * np.linalg.norm(A @ d) and 3.0 < errs[0] / errs[1] < 5.0


def test_explicit_lattice_coordinates_equal_the_uniform_path():
    dim, k, m = 3, 2, 2
    lat = inputs.node_coords(dim, k, m)
    p0, p1 = make(dim, k, m), make(dim, k, m, X=lat)
    u = inputs.smooth_field(dim, k, m, seed=1)
    x = inputs.gaussian_vector(p0.n_dofs, 2)
    np.testing.assert_allclose(p1.residual_raw(u), p0.residual_raw(u), atol=1e-14)
    np.testing.assert_allclose(p1.apply(u, x), p0.apply(u, x), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(p1.diagonal(u), p0.diagonal(u), rtol=1e-13)
