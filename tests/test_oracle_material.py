"""Pins of oracle.material: the closed-form tau and J*C against derivatives of psi, for the paper's law
(Sec. 2.3) and the second volumetric function (law 1).

psi, tau and J*C are three separately written formulas; finite differences tie each one to the
next, so a dropped term or a wrong factor in any of them fails here.
"""
import numpy as np
import pytest

from oracle import material


def _random_F(rng, d, scale=0.3):
    while True:
        F = np.eye(d) + scale * rng.standard_normal((d, d))
        if np.linalg.det(F) > 0.3:
            return F


@pytest.mark.parametrize("law", material.LAWS)
@pytest.mark.parametrize("d", [2, 3])
def test_tau_is_push_forward_of_dpsi(d, law):
    rng = np.random.default_rng(0)
    mu, lam = 1.3, 2.1
    for _ in range(5):
        F = _random_F(rng, d)
        P = np.zeros((d, d))
        errs = []
        for eps in (1e-4, 5e-5):
            for i in range(d):
                for j in range(d):
                    E = np.zeros((d, d)); E[i, j] = eps
                    P[i, j] = (material.psi(F + E, mu, lam, law=law) - material.psi(F - E, mu, lam, law=law)) / (2 * eps)
            errs.append(np.abs(P @ F.T - material.kirchhoff(F, mu, lam, law=law)).max())
        assert errs[1] < 1e-7
        np.testing.assert_allclose(material.piola(F, mu, lam, law=law), P, atol=1e-7)


@pytest.mark.parametrize("law", material.LAWS)
@pytest.mark.parametrize("d", [2, 3])
def test_linearisation_of_piola(d, law):
    """D_H P = [grad H . tau + J*C : grad^s H] F^{-T} with grad H = H F^{-1} (Eq. tangent and its footnote)."""
    rng = np.random.default_rng(1)
    mu, lam = 0.7, 1.9
    for _ in range(5):
        F = _random_F(rng, d)
        H = rng.standard_normal((d, d))
        Finv = np.linalg.inv(F)
        g = H @ Finv
        gs = 0.5 * (g + g.T)
        pred = (g @ material.kirchhoff(F, mu, lam, law=law)
                + np.einsum("ijkl,kl->ij", material.spatial_tangent(F, mu, lam, law=law), gs)) @ Finv.T
        errs = []
        for eps in (2e-4, 1e-4):
            fd = (material.piola(F + eps * H, mu, lam, law=law) - material.piola(F - eps * H, mu, lam, law=law)) / (2 * eps)
            errs.append(np.abs(fd - pred).max())
        assert errs[1] < 1e-6 * np.abs(pred).max()
        assert errs[1] < 0.3 * errs[0]  # second-order convergence of the central difference


@pytest.mark.parametrize("law", material.LAWS)
@pytest.mark.parametrize("d", [2, 3])
def test_stress_free_reference_and_rotation(d, law):
    mu, lam = 1.0, 1.5
    I = np.eye(d)
    assert material.psi(I, mu, lam, law=law) == 0.0
    assert np.all(material.kirchhoff(I, mu, lam, law=law) == 0.0)
    th = 0.7
    Q = np.eye(d)
    Q[:2, :2] = [[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]
    assert abs(material.psi(Q, mu, lam, law=law)) < 1e-15
    assert np.abs(material.kirchhoff(Q, mu, lam, law=law)).max() < 1e-15


@pytest.mark.parametrize("law", material.LAWS)
@pytest.mark.parametrize("d", [2, 3])
def test_symmetries_and_objectivity(d, law):
    rng = np.random.default_rng(2)
    F = _random_F(rng, d)
    C = material.spatial_tangent(F, 1.0, 1.5, law=law)
    np.testing.assert_allclose(C, C.transpose(1, 0, 2, 3), atol=0)
    np.testing.assert_allclose(C, C.transpose(0, 1, 3, 2), atol=0)
    np.testing.assert_allclose(C, C.transpose(2, 3, 0, 1), atol=0)
    tau = material.kirchhoff(F, 1.0, 1.5, law=law)
    np.testing.assert_allclose(tau, tau.T, atol=1e-15)
    th = 0.4
    Q = np.eye(d)
    Q[:2, :2] = [[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]
    np.testing.assert_allclose(material.kirchhoff(Q @ F, 1.0, 1.5, law=law), Q @ tau @ Q.T, atol=1e-13)
