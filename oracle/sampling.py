"""FW-H data-surface sampling (Section 3.1: density, pressure and velocity are
collected on the permeable surface during the run).

Each surface point is located once: the element whose bounding box holds it
is searched by Newton iteration on x(xi) = y (tolerance 1e-13); when a point
lies on a shared face the lowest element id wins.  The sampled value is the
element's tensor Lagrange interpolant of the solution at the located xi,
converted to (rho, V_1..V_dim, p).

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .basis import lagrange, lagrange_deriv


def _map_and_jac(nodes_e, q, dim, xi):
    xe = np.linspace(-1.0, 1.0, q + 1)
    L = [lagrange(xe, [xi[d]])[0] for d in range(dim)]
    Ld = [lagrange_deriv(xe, [xi[d]])[0] for d in range(dim)]
    X = nodes_e.reshape((q + 1,) * dim + (dim,))  # [c, b, a, comp]
    x = np.zeros(dim)
    A = np.zeros((dim, dim))
    for idx in np.ndindex(*((q + 1,) * dim)):
        a = idx[::-1]  # direction 0 index last in the reshape
        w = 1.0
        for d in range(dim):
            w *= L[d][a[d]]
        x += w * X[idx]
        for k in range(dim):
            wk = 1.0
            for d in range(dim):
                wk *= Ld[d][a[d]] if d == k else L[d][a[d]]
            A[:, k] += wk * X[idx]
    return x, A


def locate(mesh, pts, tol=1e-13):
    """(element ids [N], reference coordinates [N, dim]) of physical points."""
    nodes = mesh.nodes
    q, dim = mesh.q, mesh.dim
    lo = nodes.min(axis=1)
    hi = nodes.max(axis=1)
    pad = 0.05 * (hi - lo).max(axis=1, keepdims=True)
    elems = np.full(len(pts), -1, np.int64)
    xis = np.zeros((len(pts), dim))
    for k, y in enumerate(pts):
        cand = np.nonzero(np.all((y >= lo - pad) & (y <= hi + pad), axis=1))[0]
        for e in cand:
            xi = np.zeros(dim)
            ok = False
            for _ in range(50):
                x, A = _map_and_jac(nodes[e], q, dim, xi)
                dx = np.linalg.solve(A, y - x)
                xi = xi + dx
                if np.max(np.abs(xi)) > 3.0:
                    break
                if np.max(np.abs(dx)) < tol:
                    ok = True
                    break
            if ok and np.all(np.abs(xi) <= 1.0 + 1e-10):
                elems[k] = e
                xis[k] = np.clip(xi, -1.0, 1.0)
                break
        if elems[k] < 0:
            raise ValueError(f"surface point {k} not found in the mesh")
    return elems, xis


def sample(mesh, phys, u, elems, xis):
    """Primitive values [N, dim+2] = (rho, V..., p) at located points."""
    ref = mesh.ref
    dim, Np = mesh.dim, mesh.Np
    out = np.zeros((len(elems), dim + 2))
    for k, (e, xi) in enumerate(zip(elems, xis)):
        L = [lagrange(ref.x, [xi[d]])[0] for d in range(dim)]
        w = L[0]
        for d in range(1, dim):
            w = np.multiply.outer(L[d], w)     # direction 0 fastest
        uk = u[e] @ w.ravel()                  # [nvar]
        rho = uk[0]
        V = uk[1:1 + dim] / rho
        p = phys.pressure(uk[:, None])[0]
        out[k] = np.concatenate([[rho], V, [p]])
    return out
