"""Adaptive explicit time step (Section 3.1: the LES runs with adaptive time
stepping; the stage coefficients of the paper's integrator are in its cited
work, not in the paper, so the step size rule is what is built here).

Reading: each step takes dt = cfl / max_e lambda_e over the candidate, with
lambda_e = max_sp (|V| + c) (p+1)^2 / h_e + max_sp (mu / rho) (p+1)^4 / h_e^2
and the element length h_e = min over solution points and directions d of
2 |J| / |S[d, :]| (the physical extent of the reference interval [-1, 1]
along xi_d; exact for an affine element).

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def element_length(mesh):
    """h_e [E] = min over sp, d of 2 |J| / |S[d, :]|."""
    Snorm = np.linalg.norm(mesh.S, axis=2)           # [E, d, Nsp]
    return np.min(2.0 * mesh.J[:, None, :] / Snorm, axis=(1, 2))


def spectral_rate(mesh, phys, u):
    """lambda_e [E] of the reading above for the state u [E, nvar, Nsp]."""
    dim = mesh.dim
    rho = u[:, 0]
    V = u[:, 1:1 + dim] / rho[:, None]
    vmag = np.sqrt(np.sum(V * V, axis=1))
    p = phys.pressure(np.moveaxis(u, 1, 0))
    c = np.sqrt(phys.gamma * p / rho)
    h = element_length(mesh)
    k = (mesh.p + 1) ** 2
    lam = np.max(vmag + c, axis=1) * k / h
    if phys.viscous and phys.mu > 0.0:
        lam = lam + np.max(phys.mu / rho, axis=1) * k * k / (h * h)
    return lam


def cfl_dt(mesh, phys, u, cfl):
    """dt = cfl / max_e lambda_e."""
    return cfl / float(np.max(spectral_rate(mesh, phys, u)))
