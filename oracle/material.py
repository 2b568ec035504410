"""Compressible neo-Hooke law of Sec. 2.3, batched over leading axes.

Test infrastructure (see oracle/__init__.py). Written straight from the printed
closed forms: psi(C) = mu/2 [tr C - tr I - 2 ln J] + lambda ln^2 J,
tau = mu b - (mu - 2 lambda ln J) I, J*C = 2 (mu - 2 lambda ln J) S + 2 lambda I (x) I.
In 2D (plane strain) all tensors are 2x2 and tr I = 2.
"""
from __future__ import annotations

import numpy as np


def psi(F, mu, lam):
    """Strain energy per unit reference volume (Sec. 2.3), F shaped (..., d, d); mu, lam broadcast to (...)."""
    d = F.shape[-1]
    C = np.swapaxes(F, -1, -2) @ F
    J = np.linalg.det(F)
    lnJ = np.log(J)
    return 0.5 * mu * (np.trace(C, axis1=-2, axis2=-1) - d - 2.0 * lnJ) + lam * lnJ**2


def kirchhoff(F, mu, lam):
    """Kirchhoff stress tau = mu b - (mu - 2 lambda ln J) I (Sec. 2.3)."""
    d = F.shape[-1]
    b = F @ np.swapaxes(F, -1, -2)
    lnJ = np.log(np.linalg.det(F))
    mu = np.asarray(mu, dtype=float)[..., None, None]
    c1 = (mu - 2.0 * np.asarray(lam, dtype=float)[..., None, None] * lnJ[..., None, None])
    return mu * b - c1 * np.eye(d)


def spatial_tangent(F, mu, lam):
    """Material part of the spatial tangent J*C_ijkl = 2(mu - 2 lambda ln J) S_ijkl + 2 lambda d_ij d_kl (Sec. 2.3)."""
    d = F.shape[-1]
    I = np.eye(d)
    S = 0.5 * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))
    II = np.einsum("ij,kl->ijkl", I, I)
    lnJ = np.log(np.linalg.det(F))
    c = 2.0 * (np.asarray(mu, dtype=float) - 2.0 * np.asarray(lam, dtype=float) * lnJ)
    lam2 = 2.0 * np.asarray(lam, dtype=float)
    return c[..., None, None, None, None] * S + lam2[..., None, None, None, None] * II


def piola(F, mu, lam):
    """First Piola stress P = tau F^{-T} (Sec. 2.1: tau := P F^T)."""
    return kirchhoff(F, mu, lam) @ np.swapaxes(np.linalg.inv(F), -1, -2)
