"""Pins of oracle.gmg: transfers, Chebyshev polynomial, Ritz estimate, V-cycle, PCG (Secs. 6-7)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import gmg
from oracle.basis import gll_nodes
from paper_1904_13131_gb300 import inputs


@pytest.mark.parametrize("k,mc", [(1, 3), (2, 2), (3, 2), (4, 1)])
def test_prolongation_reproduces_polynomials(k, mc):
    xc = inputs.lattice_1d(k, mc)
    xf = inputs.lattice_1d(k, 2 * mc)
    P1 = gmg.prolongation_1d(k, mc)
    for p in range(k + 1):
        np.testing.assert_allclose(P1 @ xc**p, xf**p, atol=1e-13)
    # carrying a prolongated coarse field back down returns it (nested spaces)
    I1 = gmg.interpolation_1d(k, mc)
    np.testing.assert_allclose(I1 @ P1, np.eye(len(xc)), atol=1e-13)
    # a fine field with a kink inside a coarse cell is not a coarse field: interpolation samples it
    f = np.abs(xf - 0.5 / mc) if mc > 1 else xf**(k + 1)
    assert np.abs(P1 @ (I1 @ f) - f).max() > 1e-6


def test_lattice_operator_layout():
    P1 = gmg.prolongation_1d(2, 1)
    P = gmg.lattice_operator(P1, 2)
    xc = inputs.node_coords(2, 2, 1)
    xf = inputs.node_coords(2, 2, 2)
    uc = np.stack([xc[:, 0] ** 2 * xc[:, 1], xc[:, 1] - xc[:, 0] * xc[:, 1] ** 2], 1).reshape(-1)
    uf = np.stack([xf[:, 0] ** 2 * xf[:, 1], xf[:, 1] - xf[:, 0] * xf[:, 1] ** 2], 1).reshape(-1)
    np.testing.assert_allclose(P @ uc, uf, atol=1e-14)


def test_chebyshev_error_polynomial_closed_form():
    lam = np.linspace(0.05, 2.0, 40)
    A = sp.diags(lam)
    x_star = np.ones_like(lam)
    b = A @ x_star
    lo, hi = 0.6, 2.4
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    for s in (1, 2, 4, 7):
        x = gmg.chebyshev(A, np.ones_like(lam), b, None, s, lo, hi)

        def T(s_, t):
            t = np.asarray(t, dtype=float)
            return np.where(np.abs(t) <= 1, np.cos(s_ * np.arccos(np.clip(t, -1, 1))),
                            np.sign(t) ** s_ * np.cosh(s_ * np.arccosh(np.maximum(np.abs(t), 1))))
        p = T(s, (theta - lam) / delta) / T(s, theta / delta)
        np.testing.assert_allclose(x_star - x, p * x_star, atol=1e-13)
    # with a start vector the same polynomial acts on the initial error
    x0 = np.linspace(-1, 1, 40)
    x = gmg.chebyshev(A, np.ones_like(lam), b, x0, 4, lo, hi)
    p = T(4, (theta - lam) / delta) / T(4, theta / delta)
    np.testing.assert_allclose(x_star - x, p * (x_star - x0), atol=1e-13)


def test_ritz_values_and_coarse_degree():
    rng = np.random.default_rng(0)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1, 50, n)) @ Q.T
    A = 0.5 * (A + A.T)
    Dinv = 1.0 / np.diag(A)
    ritz = gmg.cg_ritz(A, Dinv, rng.standard_normal(n), n)
    ev = np.sort(np.linalg.eigvals(Dinv[:, None] * A).real)
    np.testing.assert_allclose(ritz.max(), ev.max(), rtol=1e-8)
    np.testing.assert_allclose(ritz.min(), ev.min(), rtol=1e-6)
    few = gmg.cg_ritz(A, Dinv, rng.standard_normal(n), 5)
    assert few.max() <= ev.max() * (1 + 1e-12) and few.min() >= ev.min() * (1 - 1e-12)
    for lo, hi in ((0.01, 3.0), (0.5, 2.0)):
        s = gmg.coarse_degree(lo, hi)
        sig = (hi + lo) / (hi - lo)
        assert 1.0 / math.cosh(s * math.acosh(sig)) <= 1e-3
        assert s == 1 or 1.0 / math.cosh((s - 1) * math.acosh(sig)) > 1e-3


@pytest.fixture(scope="module")
def hier2d():
    pr = inputs.problem(2, 2, 8, n_levels=3, top=inputs.normal_top_mask(2))
    H = gmg.Hierarchy(2, 2, pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"])
    u = 0.5 * inputs.smooth_field(2, 2, 8, seed=1)
    H.set_displacement(u)
    return H


def test_level_displacement_and_eigen_estimate(hier2d):
    H = hier2d
    for l in range(1, 3):  # u_l is the nodal interpolation of u_{l+1}
        X = inputs.node_coords(2, 2, H.levels[l - 1].m)
        Xf = inputs.node_coords(2, 2, H.levels[l].m)
        idx = [int(np.argmin(np.abs(Xf - x).sum(1))) for x in X]  # k = 2: coarse nodes are fine nodes
        np.testing.assert_array_equal(H.u[l - 1].reshape(-1, 2), H.u[l].reshape(-1, 2)[idx])
        A = H.A[l].toarray()
        ev = np.linalg.eigvals(A * H.Dinv[l][:, None]).real.max()
        assert ev * (1 - 1e-2) <= H.lmax[l] <= ev * (1 + 1e-12)


def _dense_vcycle(H):
    f = H.levels[-1].free
    cols = np.where(f)[0]
    V = np.zeros((len(cols), len(cols)))
    e = np.zeros(len(f))
    for i, c in enumerate(cols):
        e[:] = 0.0
        e[c] = 1.0
        V[:, i] = H.vcycle(e)[f]
    return V, H.A[-1].toarray()[np.ix_(f, f)]


def test_vcycle_symmetric_positive_definite(hier2d):
    """With an unresolved inclusion the coarse levels are not Galerkin operators (Sec. 6 assumes the
    coarsest mesh resolves the heterogeneity), so the cycle may overshoot; it must stay SPD."""
    V, A = _dense_vcycle(hier2d)
    assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0
    assert np.linalg.eigvals(V @ A).real.min() > 0


def test_vcycle_contracts_on_homogeneous_material():
    pr = inputs.problem(2, 2, 8, n_levels=3, top=inputs.normal_top_mask(2), ratio=1.0)
    H = gmg.Hierarchy(2, 2, pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"])
    H.set_displacement(0.5 * inputs.smooth_field(2, 2, 8, seed=1))
    V, A = _dense_vcycle(H)
    ev = np.linalg.eigvals(V @ A).real
    assert ev.min() > 0.3 and ev.max() < 1.1  # rho(I - V A) < 0.7


def test_pcg_matches_direct_solve(hier2d):
    H = hier2d
    A = H.A[-1]
    b = inputs.gaussian_vector(A.shape[0], 9)
    b[H.levels[-1].constrained] = 0
    x, its, ok = gmg.pcg(A, b, H.vcycle, rtol=1e-12)
    assert ok and its < 40
    xd = spla.spsolve(A.tocsc(), b)
    np.testing.assert_allclose(x, xd, atol=1e-10 * np.abs(xd).max())


def test_gll_nodes_used_by_transfers_match_inputs():
    for k in (1, 2, 3, 4):
        np.testing.assert_allclose(gll_nodes(k), inputs.gll_unit(k), atol=1e-15)


def test_direct_coarse_option():
    """Exact coarse solve: one level makes the V-cycle the inverse; with more levels it stays SPD."""
    pr = inputs.problem(2, 2, 4, n_levels=1, top=inputs.normal_top_mask(2))
    H = gmg.Hierarchy(2, 2, pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"], coarse_solver="direct")
    u = 0.3 * inputs.smooth_field(2, 2, 4, seed=1)
    H.set_displacement(u)
    b = inputs.gaussian_vector(H.levels[0].n_dofs, 2)
    b[H.levels[0].constrained] = 0
    np.testing.assert_allclose(H.A[0] @ H.vcycle(b), b, atol=1e-12 * np.abs(b).max())
    pr = inputs.problem(2, 2, 8, n_levels=3, top=inputs.normal_top_mask(2))
    H = gmg.Hierarchy(2, 2, pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"], coarse_solver="direct")
    H.set_displacement(0.5 * inputs.smooth_field(2, 2, 8, seed=1))
    V, A = _dense_vcycle(H)
    assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0
