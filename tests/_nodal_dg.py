"""Independent nodal DG for 2D linear advection on a uniform periodic quad mesh.

Used only to pin the oracle: FR with the DG correction function, GL points
and an upwind (Rusanov) flux must reproduce the nodal DG semi-discretisation
of a linear flux on affine elements (Huynh 2007, as cited in Section 1).

Weak form per element K with the tensor Lagrange basis phi_k on the GL nodes:
    M du/dt = sum_K int_K grad(phi_k) . a u dx - int_dK phi_k (a.n) u* ds
with u* the upwind trace.  Every integral uses a Gauss rule of p+3 points per
direction, so nothing here shares the FR construction (no correction
functions, no extrapolation lines).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def _lag(xs, ys):
    L = np.ones((len(ys), len(xs)))
    for j in range(len(xs)):
        for m in range(len(xs)):
            if m != j:
                L[:, j] *= (ys - xs[m]) / (xs[j] - xs[m])
    return L


def _lagd(xs, ys):
    n = len(xs)
    D = np.zeros((len(ys), n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            t = np.full(len(ys), 1.0 / (xs[j] - xs[k]))
            for m in range(n):
                if m not in (j, k):
                    t = t * (ys - xs[m]) / (xs[j] - xs[m])
            D[:, j] += t
    return D


def dg_rhs(u, nx, ny, hx, hy, p, a):
    """du/dt for u [E, Np*Np] (node index i + Np j, element e = ex + nx ey)."""
    Np = p + 1
    xn, _ = npleg.leggauss(Np)
    xq, wq = npleg.leggauss(p + 3)
    B = _lag(xn, xq)                 # [nq, Np]
    Bd = _lagd(xn, xq)
    Bm = _lag(xn, np.array([-1.0]))[0]
    Bp = _lag(xn, np.array([1.0]))[0]
    # 2D basis at volume quadrature points: phi_{i + Np j}(xq_a, xq_b)
    Phi = np.einsum("ai,bj->abji", B, B).reshape(len(xq) ** 2, Np * Np)
    Phx = np.einsum("ai,bj->abji", Bd, B).reshape(len(xq) ** 2, Np * Np) * (2.0 / hx)
    Phy = np.einsum("ai,bj->abji", B, Bd).reshape(len(xq) ** 2, Np * Np) * (2.0 / hy)
    W = np.einsum("a,b->ab", wq, wq).ravel() * (hx * hy / 4.0)
    M = Phi.T @ (W[:, None] * Phi)
    K = (a[0] * Phx + a[1] * Phy).T @ (W[:, None] * Phi)
    E = nx * ny
    out = np.empty_like(u)
    ue = u.reshape(E, Np, Np)        # [e, j, i]
    for e in range(E):
        ex, ey = e % nx, e // nx
        rhs = K @ u[e]
        # four edges: (normal, own trace function of the other coordinate, neighbour)
        edges = [
            ((-1.0, 0.0), lambda U: U @ Bm, ((ex - 1) % nx) + nx * ey, lambda U: U @ Bp, hy, "x", Bm),
            ((1.0, 0.0), lambda U: U @ Bp, ((ex + 1) % nx) + nx * ey, lambda U: U @ Bm, hy, "x", Bp),
            ((0.0, -1.0), lambda U: Bm @ U, ex + nx * ((ey - 1) % ny), lambda U: Bp @ U, hx, "y", Bm),
            ((0.0, 1.0), lambda U: Bp @ U, ex + nx * ((ey + 1) % ny), lambda U: Bm @ U, hx, "y", Bp),
        ]
        for nrm, own, nb, other, length, axis, bedge in edges:
            an = a[0] * nrm[0] + a[1] * nrm[1]
            uo = B @ own(ue[e])              # trace at quadrature points along the edge
            un = B @ other(ue[nb])
            ustar = uo if an > 0 else un
            flux = an * ustar * wq * (length / 2.0)   # [nq]
            if axis == "x":
                # phi_{i + Np j} on the edge: l_i(+-1) l_j(s)
                contrib = np.einsum("i,sj,s->ji", bedge, B, flux).ravel()
            else:
                contrib = np.einsum("j,si,s->ji", bedge, B, flux).ravel()
            rhs -= contrib
        out[e] = np.linalg.solve(M, rhs)
    return out
