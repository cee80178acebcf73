"""FR residual, classic RK4 update and wall forces (plain FP64, vectorised over
elements).

The semi-discrete system du/dt = R(u) discretises Eq. 1 (Section 2.1) with
Huynh's Flux Reconstruction (cited in Section 1).  The paper gives no FR
details; the reading taken (tensor GL points, DG or g2 correction, Rusanov
inviscid flux, BR2 viscous flux) is spelled out step by step below.

Notation (per element, reference coordinates xi in [-1, 1]^dim):

* u_f: the solution polynomial extrapolated to the flux points of a face;
  with GL points each face point needs only the line of solution points
  normal to it.
* For a face f = 2 d + s (xi_d = -1 for s = 0, +1 for s = 1), nsign = -1 / +1
  and h_f = h_- / h_+ the correction-derivative profile along that line
  (``Ref1D.hm`` / ``Ref1D.hp``).
* Common solution u_c = (u_L + u_R)/2 (interior) or the boundary state.
* Corrected gradient (FR form of the auxiliary equation):
  q_d = D_d u + sum over the two faces normal to d of nsign h_f (u_c - u_f);
  grad u = (1/|J|) sum_d S[d, :] q_d.
* BR2 face gradient on each side: G = I_f[grad_D u] + eta I_f[r_f] with
  grad_D u the uncorrected gradient and r_f the correction of face f alone;
  common viscous flux 1/2 (F_v(u_L, G_L) + F_v(u_R, G_R)).N.
* Residual R = -(1/|J|) [ sum_d D_d Ft_d + sum_f h_f (Fc.N - nsign I_f[Ft_d]) ]
  with Ft_d = sum_i S[d, i] F_i, F = F_inv - F_vis, and Fc.N the common
  normal flux (inviscid minus viscous) scaled by the face area.

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from . import mixed
from .mixed import MortarOps
from .physics import BC_FARFIELD, BC_WALL


def _contract(a, vec, d, dim):
    """Contract direction d of tensor data a [..., Np,.., Np] with vec [Np]."""
    return np.tensordot(a, vec, axes=([a.ndim - 1 - d], [0]))


def _deriv(a, D, d, dim):
    ax = a.ndim - 1 - d
    return np.moveaxis(np.tensordot(a, D, axes=([ax], [1])), -1, ax)


def _expand(fv, h, d, dim, Np):
    """Spread face-point values fv [..., Nfp] along the lines normal to a face of
    direction d with profile h [Np]: out[..., sp] = fv[fp(sp)] * h[i_d(sp)]."""
    lead = fv.shape[:-1]
    t = fv.reshape(lead + (Np,) * (dim - 1))
    t = np.expand_dims(t, axis=-1 - d)
    return t * h.reshape((Np,) + (1,) * d)


class FRSolver:
    """Residual, RK4 and forces on one mesh for one physics.

    ``caps``: optional per-element polynomial degrees q <= p; an element of
    degree q < p is a degree-q FR element whose faces keep the degree-p flux
    points (``oracle.mixed``).
    ``source``: optional list of Gaussian monopoles (A, k, (xs, ys, zs), freq)
    added to the energy equation (Appendix D, Eq. D.1):
    s(x, t) = sum_m A_m exp(-k_m |x - x_m|^2) sin(2 pi freq_m t), evaluated at
    the solution points at the stage time."""

    def __init__(self, mesh, phys, source=None, caps=None):
        self.m = mesh
        self.ph = phys
        self.source = list(source) if source else []
        # per-element degrees: the elements of each reduced degree q < p and
        # their degree-q operators
        self.caps = None if caps is None else np.asarray(caps, np.int64)
        self.reduced = []
        if self.caps is not None:
            for q in range(mesh.p):
                sel = np.nonzero(self.caps == q)[0]
                if sel.size:
                    self.reduced.append((sel, MortarOps(mesh.p, q, mesh.ref.kind)))
        if self.source and self.reduced:
            raise ValueError("the energy source is defined on elements of the full degree only")

    def source_term(self, t):
        """s(x_sp, t) [E, Nsp] of Eq. D.1 (zeros without sources)."""
        x = self.m.xsp
        s = np.zeros(x.shape[:2])
        for A, k, xs, freq in self.source:
            r2 = np.sum((x - np.asarray(xs, float)[None, None, :x.shape[2]]) ** 2, axis=-1)
            s += A * np.exp(-k * r2) * np.sin(2.0 * np.pi * freq * t)
        return s

    # -------------------------------------------------------------------
    def residual(self, u, want_faces=False, t=0.0):
        """R(u) for u [E, nvar, Nsp] at time t (the time enters only through
        the source term); optionally also face data: the traces ``uf``
        [E, nface, nvar, Nfp], the common viscous normal flux ``Fv_common``
        and the BR2 face gradients ``Gface`` [E, nface, nvar, dim, Nfp]
        (None for inviscid physics), and the boundary states ``bc``."""
        m, ph = self.m, self.ph
        ref = m.ref
        E, dim, Np, Nfp, nf = m.E, m.dim, m.Np, m.Nfp, m.nface
        nv = ph.nvar
        tshape = (Np,) * dim
        ut = u.reshape((E, nv) + tshape)
        J = m.J                                  # [E, Nsp]
        S = m.S                                  # [E, d, i, Nsp]

        # 1. traces at flux points
        uf = np.empty((E, nf, nv, Nfp))
        for d in range(dim):
            for s in (0, 1):
                lv = ref.lp if s else ref.lm
                uf[:, 2 * d + s] = _contract(ut, lv, d, dim).reshape(E, nv, Nfp)

        # 2. outside state: neighbour trace, or boundary ghost / boundary state
        conn = m.conn
        inner = conn[:, :, 0] >= 0
        ei, fi = np.nonzero(inner)
        ne, nfc = conn[ei, fi, 0], conn[ei, fi, 1]
        uo = np.zeros_like(uf)
        uo[ei, fi] = np.moveaxis(uf[ne[:, None], nfc[:, None], :, m.fpmap[ei, fi]], -1, 1)
        uc = 0.5 * (uf + uo)
        ughost = uo.copy()
        N = m.N                                  # [E, nf, Nfp, dim]
        bc = {}
        for tag in (BC_WALL, BC_FARFIELD):
            be, bfc = m.bc_faces(tag)
            if be.size == 0:
                continue
            uL = np.moveaxis(uf[be, bfc], 1, 0)              # [nv, K, Nfp]
            Nb = np.moveaxis(N[be, bfc], -1, 0)              # [dim, K, Nfp]
            g, ub = ph.bc_states(tag, uL, Nb)
            ughost[be, bfc] = np.moveaxis(g, 0, 1)
            uc[be, bfc] = np.moveaxis(ub, 0, 1)
            bc[tag] = (be, bfc, ub, Nb)
        jmp = uc - uf                            # [E, nf, nv, Nfp]

        # 3. common inviscid normal flux (area-weighted)
        Fc = np.moveaxis(ph.rusanov(np.moveaxis(uf, 2, 0), np.moveaxis(ughost, 2, 0),
                                    np.moveaxis(N, 3, 0)), 0, 2)

        # 4. viscous terms (BR2)
        grad = None
        Fv_common = None
        Gface = None
        if ph.viscous:
            qD = [_deriv(ut, ref.D, d, dim).reshape(E, nv, -1) for d in range(dim)]
            gD = np.zeros((E, nv, dim, m.Nsp))
            for i in range(dim):
                for d in range(dim):
                    gD[:, :, i] += (S[:, d, i] / J)[:, None] * qD[d]
            gDt = gD.reshape((E, nv, dim) + tshape)
            Fv_own = np.zeros((E, nf, nv, Nfp))
            Gface = np.zeros((E, nf, nv, dim, Nfp))
            for d in range(dim):
                for s in (0, 1):
                    f = 2 * d + s
                    lv = ref.lp if s else ref.lm
                    h = ref.hp if s else ref.hm
                    nsg = 1.0 if s else -1.0
                    Gi = _contract(gDt, lv, d, dim).reshape(E, nv, dim, Nfp)
                    line = _expand(jmp[:, f], h, d, dim, Np).reshape(E, nv, -1)  # [E, nv, Nsp]
                    lift = nsg * (S[:, d] / J[:, None])[:, None] * line[:, :, None]  # [E,nv,i,Nsp]
                    Li = _contract(lift.reshape((E, nv, dim) + tshape), lv, d, dim).reshape(E, nv, dim, Nfp)
                    Gface[:, f] = Gi + ph.eta * Li
            for sel, ops in self.reduced:
                Gface[sel] = mixed.face_gradients(m, ph, sel, ops, u, jmp)
            for f in range(nf):
                G = Gface[:, f]
                Fvis = ph.flux_vis(np.moveaxis(uf[:, f], 1, 0), np.transpose(G, (1, 2, 0, 3)))  # [nv, dim, E, Nfp]
                Fv_own[:, f] = np.moveaxis(np.einsum("vdef,efd->vef", Fvis, N[:, f]), 0, 1)
            Fv_common = np.zeros_like(Fv_own)
            Fv_common[ei, fi] = 0.5 * (Fv_own[ei, fi] - np.moveaxis(
                Fv_own[ne[:, None], nfc[:, None], :, m.fpmap[ei, fi]], -1, 1))
            for tag, (be, bfc, ub, Nb) in bc.items():
                G = np.moveaxis(Gface[be, bfc], 1, 0)        # [nv, K, dim, Nfp]
                G = np.moveaxis(G, 2, 1)                     # [nv, dim, K, Nfp]
                Fv_common[be, bfc] = np.moveaxis(ph.bc_viscous_flux(tag, ub, G, Nb), 0, 1)
            Fc = Fc - Fv_common
            # corrected gradient at solution points
            grad = np.zeros((E, nv, dim, m.Nsp))
            for d in range(dim):
                q = qD[d].copy()
                for s in (0, 1):
                    h = ref.hp if s else ref.hm
                    nsg = 1.0 if s else -1.0
                    q += nsg * _expand(jmp[:, 2 * d + s], h, d, dim, Np).reshape(E, nv, -1)
                for i in range(dim):
                    grad[:, :, i] += (S[:, d, i] / J)[:, None] * q

        # 5. flux at solution points and its transformed components
        uu = np.moveaxis(u, 1, 0)                              # [nv, E, Nsp]
        F = ph.flux_inv(uu)                                    # [nv, dim, E, Nsp]
        if ph.viscous:
            F = F - ph.flux_vis(uu, np.moveaxis(np.moveaxis(grad, 1, 0), 2, 1))
        Ft = np.einsum("edin,vien->devn", S, F)               # [d, E, nv, Nsp]

        # 6. divergence plus face corrections
        div = np.zeros((E, nv) + tshape)
        for d in range(dim):
            Ftd = Ft[d].reshape((E, nv) + tshape)
            div += _deriv(Ftd, ref.D, d, dim)
            for s in (0, 1):
                f = 2 * d + s
                lv = ref.lp if s else ref.lm
                h = ref.hp if s else ref.hm
                nsg = 1.0 if s else -1.0
                FDn = nsg * _contract(Ftd, lv, d, dim).reshape(E, nv, Nfp)
                div += _expand(Fc[:, f] - FDn, h, d, dim, Np)
        R = -div.reshape(E, nv, -1) / J[:, None]
        if self.source:
            R[:, nv - 1, :] += self.source_term(t)
        red = []
        for sel, ops in self.reduced:
            R[sel], Rq, Jq = mixed.residual(m, ph, sel, ops, u, jmp, Fc)
            red.append((sel, ops.q, Rq, Jq))
        if not want_faces:
            return R
        return R, {"uf": uf, "Fv_common": Fv_common, "bc": bc, "Gface": Gface, "reduced": red}

    # -------------------------------------------------------------------
    def rk4_step(self, u, dt, t=0.0):
        """Classic RK4 from time t: k1 = R(u, t), k2 = R(u + dt/2 k1, t + dt/2),
        k3 = R(u + dt/2 k2, t + dt/2), k4 = R(u + dt k3, t + dt);
        u + dt (k1 + 2 k2 + 2 k3 + k4)/6."""
        k1 = self.residual(u, t=t)
        k2 = self.residual(u + 0.5 * dt * k1, t=t + 0.5 * dt)
        k3 = self.residual(u + 0.5 * dt * k2, t=t + 0.5 * dt)
        k4 = self.residual(u + dt * k3, t=t + dt)
        return u + dt * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0

    # -------------------------------------------------------------------
    @staticmethod
    def coef_stage_times(coef):
        """Stage abscissae tau_i of a scheme in coefficient form: the value of
        stage i's input when the scheme integrates du/dt = 1 from u = 0 with
        dt = 1 (so u equals the time), and the value reached after the step."""
        v, acc, taus = 0.0, 0.0, []
        for i, (a, b, c, d, e, f) in enumerate(np.asarray(coef, float).reshape(-1, 6)):
            taus.append(v)
            acc = (0.0 if i == 0 else e * acc) + f
            v = a * 0.0 + b * v + c + d * acc
        return np.array(taus), v

    def coef_step(self, u, dt, coef, t=0.0):
        """One step of an explicit scheme given in coefficient form (the reading
        taken for the optimal explicit integrator that Section 3.1 uses and
        whose coefficients are in the cited work): with u0 = u, v = u,
        acc = 0, for each stage (a, b, c, d, e, f):
            k = R(v, t + tau_i dt)
            acc = e acc + f dt k      (acc = f dt k at the first stage)
            v = a u0 + b v + c dt k + d acc
        and the new state is the last v."""
        coef = np.asarray(coef, float).reshape(-1, 6)
        taus, _ = self.coef_stage_times(coef)
        u0, v, acc = u, u, None
        for i, (a, b, c, d, e, f) in enumerate(coef):
            k = self.residual(v, t=t + taus[i] * dt)
            acc = f * dt * k if i == 0 else e * acc + f * dt * k
            v = a * u0 + b * v + c * dt * k + d * acc
        return v

    # -------------------------------------------------------------------
    def wall_force(self, u):
        """Force of the fluid on the walls, sum over wall face points of
        w_fp (p N - tau(G).N) with N the element's outward area-weighted
        normal (pointing into the body), p from the interior trace and
        tau.N the momentum part of the wall's common viscous flux
        (Section 3.2 lift and drag)."""
        m, ph = self.m, self.ph
        R, faces = self.residual(u, want_faces=True)
        be, bfc = m.bc_faces(BC_WALL)
        w = m.face_weights()
        if be.size == 0:
            return np.zeros(m.dim)
        uL = np.moveaxis(faces["uf"][be, bfc], 1, 0)       # [nv, K, Nfp]
        p = ph.pressure(uL)                                 # [K, Nfp]
        Nb = m.N[be, bfc]                                   # [K, Nfp, dim]
        F = np.einsum("kf,kfd,f->d", p, Nb, w)
        if ph.viscous:
            Fv = faces["Fv_common"][be, bfc][:, 1:1 + m.dim]  # [K, dim, Nfp]
            F -= np.einsum("kdf,f->d", Fv, w)
        return F
