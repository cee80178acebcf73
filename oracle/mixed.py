"""Elements of reduced polynomial degree inside a degree-p mesh (the variable
solution degree of Section 3.1: P0 far from the body up to P3 or P4 near it,
against reflections from the boundaries).

Reading (the paper shows only the degree distribution, as a figure, and
gives no interface treatment): an element of degree q < p is a degree-q FR
element on its own (q+1)^dim GL points, while every face of the mesh keeps
the (p+1)^(dim-1) GL flux points of degree p, so faces stay conforming.
The element's state is stored as the values of its degree-q polynomial at
the degree-p points (so traces, sampling and state transfers are those of a
degree-p element).  Its residual takes these steps:

1. u_q = I_qp u: the polynomial evaluated at the q points (exact).
2. Face data at the degree-p face points as for any element: trace u_f,
   common solution u_c, common normal flux Fc.N (Rusanov minus the common
   BR2 viscous flux), all with the shared degree-p normals.
3. Mortar: the face data are projected onto degree q along each tangential
   direction and evaluated at the q face points,
       Pi_qp[i, j] = sum_{k <= q} (2k + 1)/2 P_k(x^q_i) P_k(x^p_j) w^p_j,
   exact for the degrees involved; the jump u_c - u_f and Fc.N go through it.
4. Degree-q FR with those face values: corrected gradient, flux, divergence
   and correction with the degree-q operators (DG or g2 correction; at q = 0
   the only linear correction function, (1 - x)/2, whatever the kind), and
   the metric terms S and |J| taken as the degree-p interpolants of the
   element's metrics evaluated at the q points, R_q = -div / |J|_q.
5. R = I_pq R_q: the residual polynomial evaluated at the degree-p points.

For the neighbours' common viscous flux the element's BR2 face gradient on
face f is G = I_f[grad_D u_q] + eta I_f[r_f] built at the q face points
(degree-q lifting of face f's projected jump alone) and evaluated at the
degree-p face points.

With q = p every step reduces to the uniform degree-p scheme.  The common
fluxes stay shared at the degree-p points and Pi_qp keeps the face mean, so
the scheme is conservative; on affine elements it keeps a free stream.

Test infrastructure (see ``oracle/__init``).
"""
from __future__ import annotations

import numpy as np

from .basis import DG, Ref1D, gauss_legendre, lagrange
from .mesh import _apply
from .sponge import legendre_values


def _contract(a, vec, d):
    return np.tensordot(a, vec, axes=([a.ndim - 1 - d], [0]))


def _deriv(a, D, d):
    ax = a.ndim - 1 - d
    return np.moveaxis(np.tensordot(a, D, axes=([ax], [1])), -1, ax)


def _expand(fv, h, d, dim, n):
    """Face values fv [..., n^(dim-1)] spread along the lines normal to a face
    of direction d with the profile h [n]."""
    t = fv.reshape(fv.shape[:-1] + (n,) * (dim - 1))
    t = np.expand_dims(t, axis=-1 - d)
    return t * h.reshape((n,) + (1,) * d)


class MortarOps:
    """Degree-q operators of an element inside a degree-p mesh."""

    def __init__(self, p, q, kind):
        self.p, self.q = p, q
        self.ref = Ref1D(q, kind if q > 0 else DG)
        xp, wp = gauss_legendre(p + 1)
        xq = self.ref.x
        self.Iqp = lagrange(xp, xq)           # [q+1, p+1]: values at the q points
        self.Ipq = lagrange(xq, xp)           # [p+1, q+1]: values at the p points
        Pq = np.zeros((q + 1, p + 1))
        for k in range(q + 1):
            Pq += np.outer(legendre_values(k, xq), legendre_values(k, xp) * wp) * (2 * k + 1) / 2.0
        self.Pqp = Pq                         # [q+1, p+1]: L2 projection, values at the q points


def volume(a, M, dim):
    """Apply M [m, n] along every direction of [..., n^dim] -> [..., m^dim]."""
    n = M.shape[1]
    t = a.reshape(a.shape[:-1] + (n,) * dim)
    return _apply(t, [M] * dim, dim).reshape(a.shape[:-1] + (-1,))


def face(a, M, dim):
    """Apply M [m, n] along the dim - 1 tangential directions of face data [..., n^(dim-1)]."""
    if dim == 1:
        return a
    n = M.shape[1]
    t = a.reshape(a.shape[:-1] + (n,) * (dim - 1))
    return _apply(t, [M] * (dim - 1), dim - 1).reshape(a.shape[:-1] + (-1,))


def metrics(mesh, sel, ops):
    """S [K, d, i, Nq] and |J| [K, Nq] at the q points of elements sel: the
    degree-p interpolants of the element's metric terms evaluated there."""
    dim = mesh.dim
    S = volume(mesh.S[sel], ops.Iqp, dim)
    J = volume(mesh.J[sel], ops.Iqp, dim)
    return S, J


def face_gradients(mesh, ph, sel, ops, ut, jmp):
    """BR2 face gradients [K, nface, nv, dim, Nfp] (at the degree-p face
    points) of the elements sel of degree ops.q; ut [E, nv, Np^dim] the
    states at the degree-p points, jmp [E, nface, nv, Nfp] = u_c - u_f."""
    dim, nq, Npf = mesh.dim, ops.q + 1, mesh.Nfp
    ref = ops.ref
    K, nv = len(sel), ut.shape[1]
    S, J = metrics(mesh, sel, ops)
    uq = volume(ut[sel], ops.Iqp, dim)                          # [K, nv, Nq]
    tsh = (nq,) * dim
    uqt = uq.reshape((K, nv) + tsh)
    gD = np.zeros((K, nv, dim) + tsh)
    for d in range(dim):
        qd = _deriv(uqt, ref.D, d)
        for i in range(dim):
            gD[:, :, i] += (S[:, d, i] / J).reshape((K, 1) + tsh) * qd
    out = np.zeros((K, mesh.nface, nv, dim, Npf))
    for d in range(dim):
        for s in (0, 1):
            f = 2 * d + s
            lv = ref.lp if s else ref.lm
            h = ref.hp if s else ref.hm
            nsg = 1.0 if s else -1.0
            jq = face(jmp[sel, f], ops.Pqp, dim)                   # [K, nv, Nfq]
            Gi = _contract(gD, lv, d).reshape(K, nv, dim, -1)
            line = _expand(jq, h, d, dim, nq).reshape(K, nv, -1)   # [K, nv, Nq]
            lift = nsg * (S[:, d] / J[:, None])[:, None] * line[:, :, None]   # [K, nv, i, Nq]
            Li = _contract(lift.reshape((K, nv, dim) + tsh), lv, d).reshape(K, nv, dim, -1)
            out[:, f] = face(Gi + ph.eta * Li, ops.Ipq, dim)
    return out


def gradient(mesh, sel, ops, ut, jmp):
    """Corrected gradient [K, nv, dim, Nq] at the q points of the elements sel:
    q_d = D_d u_q + sum over the faces normal to d of nsign h_f (Pi_qp jump),
    grad = (1/|J|) sum_d S[d, :] q_d."""
    dim, nq = mesh.dim, ops.q + 1
    ref = ops.ref
    K, nv = len(sel), ut.shape[1]
    S, J = metrics(mesh, sel, ops)
    uqt = volume(ut[sel], ops.Iqp, dim).reshape((K, nv) + (nq,) * dim)
    grad = np.zeros((K, nv, dim, nq ** dim))
    for d in range(dim):
        q = _deriv(uqt, ref.D, d).reshape(K, nv, -1)
        for s in (0, 1):
            h = ref.hp if s else ref.hm
            nsg = 1.0 if s else -1.0
            jq = face(jmp[sel, 2 * d + s], ops.Pqp, dim)
            q = q + nsg * _expand(jq, h, d, dim, nq).reshape(K, nv, -1)
        for i in range(dim):
            grad[:, :, i] += (S[:, d, i] / J)[:, None] * q
    return grad


def residual(mesh, ph, sel, ops, ut, jmp, Fc):
    """Residual of the elements sel of degree ops.q: returns R [K, nv, Nsp]
    at the degree-p points, R_q [K, nv, Nq] at the q points and |J|_q.
    Fc [E, nface, nv, Nfp]: common normal flux (inviscid minus viscous)."""
    dim, nq = mesh.dim, ops.q + 1
    ref = ops.ref
    K, nv = len(sel), ut.shape[1]
    S, J = metrics(mesh, sel, ops)
    uq = volume(ut[sel], ops.Iqp, dim)
    tsh = (nq,) * dim
    Fq = [face(Fc[sel, f], ops.Pqp, dim) for f in range(mesh.nface)]
    uu = np.moveaxis(uq, 1, 0)                                    # [nv, K, Nq]
    F = ph.flux_inv(uu)                                           # [nv, dim, K, Nq]
    if ph.viscous:
        grad = gradient(mesh, sel, ops, ut, jmp)
        F = F - ph.flux_vis(uu, np.moveaxis(np.moveaxis(grad, 1, 0), 2, 1))
    Ft = np.einsum("edin,vien->devn", S, F)                      # [d, K, nv, Nq]
    div = np.zeros((K, nv) + tsh)
    for d in range(dim):
        Ftd = Ft[d].reshape((K, nv) + tsh)
        div += _deriv(Ftd, ref.D, d)
        for s in (0, 1):
            f = 2 * d + s
            lv = ref.lp if s else ref.lm
            h = ref.hp if s else ref.hm
            nsg = 1.0 if s else -1.0
            FDn = nsg * _contract(Ftd, lv, d).reshape(K, nv, -1)
            div += _expand(Fq[f] - FDn, h, d, dim, nq)
    Rq = -div.reshape(K, nv, -1) / J[:, None]
    return volume(Rq, ops.Ipq, dim), Rq, J
