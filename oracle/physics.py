"""Pointwise physics: compressible Navier-Stokes fluxes (Section 2.1, Eqs. 1-7),
the Rusanov common flux, boundary states, and linear advection (used only by
the pins that compare FR with nodal DG).

Arrays carry variables on axis 0 ([nvar, ...]) and vector components on the
axis given explicitly.  Conserved variables u = [rho, rho V_i, rho E] (Eq. 2).

Readings taken (the paper is silent or inconsistent):

* Viscous flux sign (Eq. 4 prints the energy entry as -q_j - u_i tau_ij,
  which is inconsistent with the momentum entry): the standard form
  F_vis,j = [0, tau_ij, V_i tau_ij - q_j] with the total flux
  F = F_inv - F_vis.
* Heat flux Eq. 7: E + p/rho - V^2/2 = gamma e with e the specific internal
  energy, so q_j = -(mu gamma / Pr) d e / d x_j; mu constant.
* Rusanov wave speed lambda = max(|V_L.n| + c_L, |V_R.n| + c_R).
* Wall: adiabatic no-slip (viscous) or slip (inviscid) reflection ghost for
  the inviscid flux; boundary state (rho, 0, rho e) (no-slip) or the
  tangential-velocity state (slip) for the common solution.
* Far field: subsonic/supersonic characteristic (Riemann-invariant) state
  from the free stream (Appendix D.1 names Riemann-invariant boundaries).

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

BC_WALL = 1
BC_FARFIELD = 2


class NavierStokes:
    """Compressible Euler / Navier-Stokes in 2D or 3D."""

    def __init__(self, dim, gamma=1.4, mu=0.0, prandtl=0.71, viscous=None, eta=1.0,
                 freestream=None):
        self.dim = dim
        self.nvar = dim + 2
        self.gamma = gamma
        self.mu = mu
        self.prandtl = prandtl
        self.viscous = (mu > 0.0) if viscous is None else viscous
        self.eta = eta
        # free stream (rho, V[dim], p), used by the far-field boundary
        if freestream is None:
            freestream = (1.0, np.zeros(dim), 1.0)
        self.rho_inf = float(freestream[0])
        self.V_inf = np.asarray(freestream[1], float)[:dim]
        self.p_inf = float(freestream[2])

    # ---- primitive helpers -------------------------------------------
    def pressure(self, u):
        rho = u[0]
        mom = u[1:1 + self.dim]
        return (self.gamma - 1.0) * (u[-1] - 0.5 * np.sum(mom * mom, axis=0) / rho)

    def conserved(self, rho, V, p):
        ke = 0.5 * rho * np.sum(V * V, axis=0)
        return np.concatenate([rho[None], rho[None] * V, (p / (self.gamma - 1.0) + ke)[None]])

    # ---- inviscid flux, Eq. 3 -----------------------------------------
    def flux_inv(self, u):
        """F_inv [nvar, dim, ...]."""
        d = self.dim
        rho = u[0]
        V = u[1:1 + d] / rho
        p = self.pressure(u)
        F = np.empty((self.nvar, d) + rho.shape)
        F[0] = u[1:1 + d]
        for i in range(d):
            F[1 + i] = u[1 + i][None] * V
            F[1 + i, i] += p
        F[-1] = (u[-1] + p)[None] * V
        return F

    def rusanov(self, uL, uR, N):
        """Common inviscid flux F^c . N for area-weighted normal N [dim, ...].

        F^c.n = 1/2 (F_L + F_R).n - 1/2 lambda (u_R - u_L),  n = N/|N|.
        """
        d = self.dim
        area = np.sqrt(np.sum(N * N, axis=0))
        n = N / area
        FL = self.flux_inv(uL)
        FR = self.flux_inv(uR)
        Fn = 0.5 * (np.einsum("vd...,d...->v...", FL, n) + np.einsum("vd...,d...->v...", FR, n))
        cL = np.sqrt(self.gamma * self.pressure(uL) / uL[0])
        cR = np.sqrt(self.gamma * self.pressure(uR) / uR[0])
        vL = np.abs(np.sum(uL[1:1 + d] * n, axis=0) / uL[0])
        vR = np.abs(np.sum(uR[1:1 + d] * n, axis=0) / uR[0])
        lam = np.maximum(vL + cL, vR + cR)
        return (Fn - 0.5 * lam * (uR - uL)) * area

    # ---- viscous flux, Eqs. 4, 6, 7 ------------------------------------
    def flux_vis(self, u, gu):
        """F_vis [nvar, dim, ...] from u and its gradient gu [nvar, dim, ...]."""
        d = self.dim
        rho = u[0]
        V = u[1:1 + d] / rho
        Et = u[-1]
        grho = gu[0]
        gV = (gu[1:1 + d] - V[:, None] * grho[None]) / rho       # gV[i, j] = dV_i/dx_j
        gEr = (gu[-1] - (Et / rho)[None] * grho) / rho            # grad(E/rho)
        ge = gEr - np.einsum("i...,ij...->j...", V, gV)           # grad e
        div = sum(gV[i, i] for i in range(d))
        tau = self.mu * (gV + np.swapaxes(gV, 0, 1))
        for i in range(d):
            tau[i, i] -= (2.0 / 3.0) * self.mu * div
        kappa = self.mu * self.gamma / self.prandtl
        F = np.zeros((self.nvar, d) + rho.shape)
        F[1:1 + d] = tau
        F[-1] = np.einsum("i...,ij...->j...", V, tau) + kappa * ge
        return F

    # ---- boundaries ------------------------------------------------------
    def farfield_state(self, uL, N):
        """Characteristic far-field boundary state from the free stream."""
        d = self.dim
        g = self.gamma
        n = N / np.sqrt(np.sum(N * N, axis=0))
        rhoL = uL[0]
        VL = uL[1:1 + d] / rhoL
        pL = self.pressure(uL)
        cL = np.sqrt(g * pL / rhoL)
        vnL = np.sum(VL * n, axis=0)
        Vinf = self.V_inf.reshape((d,) + (1,) * (n.ndim - 1))
        vnI = np.sum(Vinf * n, axis=0)
        cI = np.sqrt(g * self.p_inf / self.rho_inf)
        Rp = vnL + 2.0 * cL / (g - 1.0)
        Rm = vnI - 2.0 * cI / (g - 1.0)
        vnb = 0.5 * (Rp + Rm)
        cb = 0.25 * (g - 1.0) * (Rp - Rm)
        out = vnb > 0.0
        s = np.where(out, pL / rhoL ** g, self.p_inf / self.rho_inf ** g)
        Vt = np.where(out[None], VL - vnL[None] * n, Vinf - vnI[None] * n)
        rhob = (cb * cb / (g * s)) ** (1.0 / (g - 1.0))
        pb = rhob * cb * cb / g
        Vb = Vt + vnb[None] * n
        ub = self.conserved(rhob, Vb, pb)
        # supersonic normal free stream: take the free stream (inflow) or interior (outflow)
        uI = self.conserved(np.full(rhoL.shape, self.rho_inf), np.broadcast_to(Vinf, VL.shape),
                            np.full(rhoL.shape, self.p_inf))
        sup_in = (np.abs(vnI) >= cI) & (vnI < 0.0)
        sup_out = (np.abs(vnI) >= cI) & (vnI >= 0.0)
        ub = np.where(sup_in[None], uI, ub)
        ub = np.where(sup_out[None], uL, ub)
        return ub

    def wall_ghost(self, uL, N):
        """Reflection ghost state for the inviscid common flux at a wall."""
        d = self.dim
        uR = uL.copy()
        if self.viscous:
            uR[1:1 + d] = -uL[1:1 + d]
        else:
            n = N / np.sqrt(np.sum(N * N, axis=0))
            mn = np.sum(uL[1:1 + d] * n, axis=0)
            uR[1:1 + d] = uL[1:1 + d] - 2.0 * mn[None] * n
        return uR

    def wall_state(self, uL, N):
        """Common solution at a wall: zero (no-slip) or tangential (slip) velocity,
        interior density and internal energy."""
        d = self.dim
        ub = uL.copy()
        rho = uL[0]
        mom = uL[1:1 + d]
        if self.viscous:
            ub[1:1 + d] = 0.0
            ub[-1] = uL[-1] - 0.5 * np.sum(mom * mom, axis=0) / rho
        else:
            n = N / np.sqrt(np.sum(N * N, axis=0))
            mn = np.sum(mom * n, axis=0)
            mt = mom - mn[None] * n
            ub[1:1 + d] = mt
            ub[-1] = uL[-1] - 0.5 * mn * mn / rho
        return ub

    def bc_states(self, tag, uL, N):
        """(ghost state for the inviscid flux, boundary common solution)."""
        if tag == BC_WALL:
            return self.wall_ghost(uL, N), self.wall_state(uL, N)
        if tag == BC_FARFIELD:
            ub = self.farfield_state(uL, N)
            return ub, ub
        raise ValueError(f"unknown boundary tag {tag}")

    def bc_viscous_flux(self, tag, ub, G, N):
        """Common viscous normal flux F_vis(u_b, G).N at a boundary face point;
        at an adiabatic wall the energy entry (V_b.tau.n - q.n) is zero."""
        F = self.flux_vis(ub, G)
        Fn = np.einsum("vd...,d...->v...", F, N)
        if tag == BC_WALL:
            Fn[-1] = 0.0
        return Fn


class Advection:
    """Linear advection du/dt + a.grad u = 0 (scalar); Rusanov = upwind."""

    def __init__(self, a):
        self.a = np.asarray(a, float)
        self.dim = self.a.size
        self.nvar = 1
        self.viscous = False

    def flux_inv(self, u):
        return u[:, None] * self.a.reshape((1, -1) + (1,) * (u.ndim - 1))

    def rusanov(self, uL, uR, N):
        an = np.einsum("d,d...->...", self.a, N)
        return 0.5 * an * (uL + uR) - 0.5 * np.abs(an) * (uR - uL)
