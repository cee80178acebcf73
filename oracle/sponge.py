"""Variable polynomial degree by element ("sponge zones", Section 3.1: a
variable solution polynomial degree, P0 far from the body up to P3 or P4 near
it, keeps acoustic waves from reflecting off the boundaries).

An element of degree q < p holds a polynomial of degree q in each direction,
stored as its values at the degree-p points; its residual is that of a
degree-q FR element (``oracle.mixed``).  A state set on such an element is
first projected onto that space with the L2 projection applied along every
direction (GL quadrature, exact for these degrees)

    Pi_q[i, j] = sum_{k <= q} P_k(x_i) P_k(x_j) w_j (2k + 1) / 2

(P_k the Legendre polynomials, x, w the degree-p GL points and weights).
Pi_q keeps the element mean (k = 0).

Test infrastructure (see ``oracle/__init``).
"""
from __future__ import annotations

import numpy as np

from .basis import gauss_legendre


def legendre_values(k, x):
    """P_k(x) by the three-term recurrence."""
    x = np.asarray(x, float)
    p0, p1 = np.ones_like(x), x
    if k == 0:
        return p0
    for n in range(1, k):
        p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
    return p1


def projection_1d(p, q):
    """Pi_q on the p+1 GL points (the identity when q >= p)."""
    x, w = gauss_legendre(p + 1)
    P = np.zeros((p + 1, p + 1))
    for k in range(min(q, p) + 1):
        v = legendre_values(k, x)
        P += np.outer(v, v * w) * (2 * k + 1) / 2.0
    return P


def project(mesh, a, caps):
    """Project a [E, ..., Nsp] element-wise: element e onto degree caps[e]
    (caps[e] >= p leaves it unchanged)."""
    a = np.array(a, float, copy=True)
    p, dim = mesh.p, mesh.dim
    for q in sorted(set(int(c) for c in np.asarray(caps)) - set(range(p, 10 ** 6))):
        sel = np.nonzero(np.asarray(caps) == q)[0]
        if sel.size == 0:
            continue
        Pq = projection_1d(p, q)
        blk = a[sel].reshape(a[sel].shape[:-1] + (p + 1,) * dim)
        for d in range(dim):
            ax = blk.ndim - 1 - d          # direction 0 is the last axis
            blk = np.moveaxis(np.tensordot(blk, Pq, axes=([ax], [1])), -1, ax)
        a[sel] = blk.reshape(a[sel].shape)
    return a
