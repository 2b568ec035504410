"""Compressible neo-Hooke laws, batched over leading axes.

Test infrastructure (see oracle/__init__.py). Law 0 is the paper's (Sec. 2.3), written straight from the
printed closed forms:
    psi(C) = mu/2 [tr C - tr I - 2 ln J] + lambda ln^2 J,
    tau = mu b - (mu - 2 lambda ln J) I,   J*C = 2 (mu - 2 lambda ln J) S + 2 lambda I (x) I.
Law 1 keeps the isochoric-plus-log part and replaces the volumetric function by
U(J) = lambda/4 (J^2 - 1 - 2 ln J) (the Simo-Taylor form); with p(J) = J U'(J) = lambda/2 (J^2 - 1):
    tau = mu b - (mu - p) I,   J*C = 2 (mu - p) S + J p'(J) I (x) I = 2 (mu - p) S + lambda J^2 I (x) I.
(The paper's law fits the same pattern with p = 2 lambda ln J and J p' = 2 lambda.) Its small-strain limit
is linear elasticity with Lame parameters (mu, lambda); law 0 gives (mu, 2 lambda).
In 2D (plane strain) all tensors are 2x2 and tr I = 2.
"""
from __future__ import annotations

import numpy as np

LAWS = (0, 1)


def _volumetric(J, lam, law):
    """(U(J), p(J) = J U'(J), J p'(J)) of the volumetric function."""
    lam = np.asarray(lam, dtype=float)
    if law == 0:
        lnJ = np.log(J)
        return lam * lnJ**2, 2.0 * lam * lnJ, 2.0 * lam * np.ones_like(lnJ)
    if law == 1:
        return 0.25 * lam * (J**2 - 1.0 - 2.0 * np.log(J)), 0.5 * lam * (J**2 - 1.0), lam * J**2
    raise ValueError(f"unknown law {law}")


def psi(F, mu, lam, law=0):
    """Strain energy per unit reference volume, F shaped (..., d, d); mu, lam broadcast to (...)."""
    d = F.shape[-1]
    C = np.swapaxes(F, -1, -2) @ F
    J = np.linalg.det(F)
    U, _, _ = _volumetric(J, lam, law)
    return 0.5 * mu * (np.trace(C, axis1=-2, axis2=-1) - d - 2.0 * np.log(J)) + U


def kirchhoff(F, mu, lam, law=0):
    """Kirchhoff stress tau = mu b - (mu - p(J)) I."""
    d = F.shape[-1]
    b = F @ np.swapaxes(F, -1, -2)
    _, p, _ = _volumetric(np.linalg.det(F), lam, law)
    mu = np.asarray(mu, dtype=float)[..., None, None]
    return mu * b - (mu - p[..., None, None]) * np.eye(d)


def spatial_tangent(F, mu, lam, law=0):
    """Material part of the spatial tangent J*C_ijkl = 2 (mu - p) S_ijkl + J p'(J) d_ij d_kl."""
    d = F.shape[-1]
    I = np.eye(d)
    S = 0.5 * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))
    II = np.einsum("ij,kl->ijkl", I, I)
    _, p, Jdp = _volumetric(np.linalg.det(F), lam, law)
    c = 2.0 * (np.asarray(mu, dtype=float) - p)
    return c[..., None, None, None, None] * S + Jdp[..., None, None, None, None] * II


def piola(F, mu, lam, law=0):
    """First Piola stress P = tau F^{-T} (Sec. 2.1: tau := P F^T)."""
    return kirchhoff(F, mu, lam, law) @ np.swapaxes(np.linalg.inv(F), -1, -2)
