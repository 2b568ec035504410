"""Pins of the dead-traction load (the surface term of Eq. weak_form) and of Newton under it.

* Closed forms on the unit square / cube: the total force on a face is t * (face area = 1); its first
  moments are t * int x_i dA (1/2 along the face, the face position across it), exact because Q_k
  reproduces linear functions and the Gauss rule integrates N_a exactly; the second moments t/3 for k >= 2.
* Nodes off the loaded faces carry nothing.
* Newton under a shear traction on the free top face: the converged internal forces balance the load
  (R_int = f_ext on the free dofs), and the reactions at the clamped bottom carry the whole load, since the
  internal forces of a free body sum to zero (translation invariance).
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs


def make(dim, k, m, masks=None):
    mu, lam = inputs.material_table(10.0)
    return Problem(dim, k, m, inputs.inclusion_ids(dim, m), mu, lam,
                   masks if masks is not None else inputs.face_masks(dim))


@pytest.mark.parametrize("dim,k,m", [(2, 1, 3), (2, 2, 4), (2, 3, 2), (3, 1, 2), (3, 2, 2)])
def test_face_load_moments(dim, k, m):
    p = make(dim, k, m)
    X = inputs.node_coords(dim, k, m)
    rng = np.random.default_rng(5)
    for face in range(2 * dim):
        t = np.zeros((2 * dim, dim))
        t[face] = rng.standard_normal(dim)
        f = p.face_load(t).reshape(-1, dim)
        ax, side = face // 2, face % 2
        on = np.isclose(X[:, ax], float(side))
        assert np.all(f[~on] == 0.0)
        np.testing.assert_allclose(f.sum(axis=0), t[face], atol=1e-14)
        for i in range(dim):
            expect = 0.5 if i != ax else float(side)
            np.testing.assert_allclose(X[:, i] @ f, expect * t[face], atol=1e-14)
            if k >= 2 and i != ax:
                np.testing.assert_allclose((X[:, i] ** 2) @ f, t[face] / 3.0, atol=1e-14)


@pytest.mark.parametrize("dim,k,m", [(2, 2, 4), (3, 1, 3)])
def test_newton_under_shear_traction_balances(dim, k, m):
    p = make(dim, k, m)  # bottom clamped, everything else free
    t = np.zeros((2 * dim, dim))
    t[2 * (dim - 1) + 1][0] = 0.05  # shear on the top face along x
    f = p.face_load(t)
    u, rep = newton_solve(p, np.zeros(p.n_dofs), load_steps=3, f_ext=f)
    R = p.residual_raw(u)
    free, cons = p.free, p.constrained
    assert np.linalg.norm(R[free] - f[free]) <= 1e-9 * np.linalg.norm(f)
    total_internal = R.reshape(-1, dim).sum(axis=0)
    np.testing.assert_allclose(total_internal, 0.0, atol=1e-12)
    # reactions at the clamped face equal minus the applied load
    np.testing.assert_allclose(R.reshape(-1, dim)[cons.reshape(-1, dim).all(axis=1)].sum(axis=0),
                               -f.reshape(-1, dim).sum(axis=0), atol=1e-9)
    assert np.abs(u).max() > 1e-3  # it deformed
