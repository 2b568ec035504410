"""Pins of oracle.newton: exact affine solution, quadratic convergence, load stepping (Secs. 3, 7)."""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs


@pytest.mark.parametrize("dim,k,m", [(2, 2, 3), (3, 1, 2)])
def test_affine_dirichlet_gives_affine_solution(dim, k, m):
    """Homogeneous body, every boundary dof prescribed by u = H X: the solution is that affine field."""
    mu, lam = inputs.material_table(1.0)
    masks = [(1 << dim) - 1] * (2 * dim)
    p = Problem(dim, k, m, np.zeros(m**dim, np.uint8), mu, lam, masks)
    rng = np.random.default_rng(1)
    H = 0.1 * rng.standard_normal((dim, dim))
    u_aff = (inputs.node_coords(dim, k, m) @ H.T).reshape(-1)
    u, rep = newton_solve(p, np.where(p.constrained, u_aff, 0.0), load_steps=2)
    np.testing.assert_allclose(u, u_aff, atol=1e-12)


def test_config1_newton_converges_quadratically():
    """2D 16x16 Q2 inclusion problem, top displaced by -0.1 in 5 load steps."""
    dim, k, m = 2, 2, 16
    pr = inputs.problem(dim, k, m, top=inputs.normal_top_mask(dim))
    p = Problem(dim, k, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
    X = inputs.node_coords(dim, k, m)
    ubc = np.zeros((p.n_nodes, dim))
    ubc[np.isclose(X[:, 1], 1.0), 1] = -0.1
    u, rep = newton_solve(p, ubc.reshape(-1), load_steps=5)
    assert all(2 <= it <= 6 for it in rep["iterations"])
    for hist in rep["residuals"]:
        for r0, r1 in zip(hist[:-1], hist[1:]):
            if r0 > 1e-8 * hist[0]:
                assert r1 <= 10.0 * r0**2 + 1e-14
    # the converged state is an equilibrium: free residual tiny, prescribed values met
    R = p.residual(u)
    assert np.linalg.norm(R) < 1e-9
    np.testing.assert_allclose(u.reshape(-1, dim)[np.isclose(X[:, 1], 1.0), 1], -0.1, atol=0)
    assert p.min_jacobian(u) > 0
