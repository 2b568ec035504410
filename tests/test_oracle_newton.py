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


def uniaxial_masks(dim):
    """Bottom clamped, every side face constrained in its own normal component, the top face held laterally
    and free along its normal: a homogeneous body under a normal traction on the top then deforms in
    uniaxial strain, F = diag(1, .., 1, s). (With the top free laterally as well, the compressed block's
    tangent turns indefinite -- a surface instability -- before s = 0.5, which every halved step reaches.)"""
    masks = [0] * (2 * dim)
    for a in range(dim - 1):
        masks[2 * a] = masks[2 * a + 1] = 1 << a
    masks[2 * (dim - 1)] = (1 << dim) - 1
    masks[2 * (dim - 1) + 1] = (1 << (dim - 1)) - 1
    return masks


def uniaxial_newton(t, mu, lam, rtol=1e-10):
    """Newton with the J > 0 halving rule (reading O15) on the scalar equilibrium of uniaxial strain under a
    dead compressive traction t on the top face: dpsi/ds (s) = -t, with psi(s) = mu/2 (s^2 - 1 - 2 ln s) +
    lam ln^2 s, the energy of Sec. 2.3 at F = diag(1, .., 1, s) (tr C = d - 1 + s^2, J = s). Differentiated
    by hand from psi, not from the stress formula: P(s) = mu (s - 1/s) + 2 lam ln s / s and
    P'(s) = mu (1 + 1/s^2) + 2 lam (1 - ln s) / s^2. Returns (s, iterations, halvings per iteration)."""
    P = lambda s: mu * (s - 1.0 / s) + 2.0 * lam * np.log(s) / s
    dP = lambda s: mu * (1.0 + 1.0 / s**2) + 2.0 * lam * (1.0 - np.log(s)) / s**2
    s, ref, its, halv = 1.0, None, 0, []
    while True:
        g = P(s) + t
        ref = abs(g) if ref is None else ref
        if its > 0 and abs(g) <= rtol * ref:
            return s, its, halv
        ds, step = -g / dP(s), 1.0
        for h in range(6):
            if s + step * ds > 0:
                break
            step *= 0.5
        else:
            raise FloatingPointError("J <= 0 after 5 halvings")
        s, its = s + step * ds, its + 1
        halv.append(h)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1), (3, 2)])
@pytest.mark.parametrize("t,first_halvings", [(7.5, 1), (12.0, 2)])
def test_newton_halves_steps_that_fold_a_cell(dim, k, t, first_halvings):
    """Reading O15 pinned on a problem with a closed-form Newton path. The first Newton step about u = 0 is
    the linear-elastic one, a strain of -t/(2 mu + 2 lam) = -t/5, so for t = 7.5 (12) it would fold every
    cell (J = -0.5 (-1.4)): the accepted update is the first halving (the second) with J > 0. Every iterate
    stays homogeneous, so the finite-element Newton must retrace the scalar Newton of uniaxial strain:
    same halvings, same iteration count, and the converged field u = (s - 1) X_d e_d exactly."""
    m = 2
    mu, lam = inputs.material_table(1.0)
    p = Problem(dim, k, m, np.zeros(m**dim, np.uint8), mu, lam, uniaxial_masks(dim))
    tr = np.zeros((2 * dim, dim))
    tr[2 * dim - 1][dim - 1] = -t
    u, rep = newton_solve(p, np.zeros(p.n_dofs), load_steps=1, f_ext=p.face_load(tr))
    s, its, halv = uniaxial_newton(t, mu[0], lam[0])
    assert halv[0] == first_halvings and rep["halvings"] == [halv]
    assert rep["iterations"] == [its]
    X = inputs.node_coords(dim, k, m)
    expect = np.zeros((p.n_nodes, dim))
    expect[:, dim - 1] = (s - 1.0) * X[:, dim - 1]
    np.testing.assert_allclose(u.reshape(-1, dim), expect, atol=1e-13)
    assert 0.3 < s < 0.5 and abs(p.min_jacobian(u) - s) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_newton_gives_up_after_five_halvings(dim):
    """t = 200: even 1/32 of the linear-elastic step (strain -40/32) folds the cells, so the solve fails."""
    m, k = 2, 1
    mu, lam = inputs.material_table(1.0)
    p = Problem(dim, k, m, np.zeros(m**dim, np.uint8), mu, lam, uniaxial_masks(dim))
    tr = np.zeros((2 * dim, dim))
    tr[2 * dim - 1][dim - 1] = -200.0
    with pytest.raises(FloatingPointError):
        newton_solve(p, np.zeros(p.n_dofs), load_steps=1, f_ext=p.face_load(tr))
    with pytest.raises(FloatingPointError):
        uniaxial_newton(200.0, mu[0], lam[0])
