"""Reference-element operators of Flux Reconstruction on [-1, 1]^dim.

The paper discretises Eq. 1 with Huynh's FR (Section 1, Section 2.1) but names
neither points nor correction functions.  Reading taken: tensor-product
Gauss-Legendre (GL) solution points, GL flux points on each face, and either
the DG correction function (right Radau polynomial) or Huynh's g2.

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg

DG = 0
HUYNH_G2 = 1


def gauss_legendre(n):
    """n GL points and weights on [-1, 1] (library primitive), made exactly
    symmetric about 0: P_n has definite parity, so its roots come in +-
    pairs (and 0 for odd n) and the weights pair up equally."""
    x, w = npleg.leggauss(n)
    x = 0.5 * (np.asarray(x, float) - np.asarray(x, float)[::-1])
    w = 0.5 * (np.asarray(w, float) + np.asarray(w, float)[::-1])
    return x, w


def gauss_lobatto(n):
    """n >= 2 Gauss-Lobatto points: -1, +1 and the roots of P'_{n-1}."""
    c = np.zeros(n)
    c[-1] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if n > 2 else np.zeros(0)
    return np.concatenate(([-1.0], inner, [1.0]))


def lagrange(xs, ys):
    """Matrix L[i, j] = l_j(ys[i]) of the Lagrange basis on nodes xs."""
    xs = np.asarray(xs, float)
    ys = np.atleast_1d(np.asarray(ys, float))
    n = xs.size
    L = np.ones((ys.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (ys - xs[m]) / (xs[j] - xs[m])
    return L


def lagrange_deriv(xs, ys):
    """Matrix D[i, j] = l_j'(ys[i]) (product rule, summed over the dropped factor)."""
    xs = np.asarray(xs, float)
    ys = np.atleast_1d(np.asarray(ys, float))
    n = xs.size
    D = np.zeros((ys.size, n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(ys.size, 1.0 / (xs[j] - xs[k]))
            for m in range(n):
                if m != j and m != k:
                    term = term * (ys - xs[m]) / (xs[j] - xs[m])
            D[:, j] += term
    return D


def _legendre(k):
    c = np.zeros(k + 1)
    c[k] = 1.0
    return c


def radau_right(k):
    """Legendre-series coefficients of R_{R,k} = ((-1)^k / 2)(P_k - P_{k-1}).

    R_{R,k}(-1) = 1 and R_{R,k}(1) = 0 (Huynh 2007): the left-boundary DG
    correction function for a degree k-1 solution.
    """
    c = np.zeros(k + 1)
    c[k] += 1.0
    c[k - 1] -= 1.0
    return 0.5 * (-1.0) ** k * c


def correction_left(p, kind):
    """Legendre coefficients of g_L for degree p (g_L(-1)=1, g_L(1)=0).

    kind=DG: g_L = R_{R,p+1}.  kind=HUYNH_G2: g2 = ((k-1) R_{R,k} + k R_{R,k-1})/(2k-1),
    k = p+1 (Huynh's g2).
    """
    k = p + 1
    if kind == DG:
        return radau_right(k)
    a = radau_right(k)
    b = np.zeros(k + 1)
    b[:k] = radau_right(k - 1)
    return ((k - 1) * a + k * b) / (2 * k - 1)


def correction_left_deriv(p, kind, xs):
    """g_L'(xs)."""
    return npleg.legval(np.asarray(xs, float), npleg.legder(correction_left(p, kind)))


class Ref1D:
    """1D ingredients of the tensor-product element of degree p.

    Attributes
    ----------
    x, w : GL solution points and quadrature weights (Np = p+1 of them)
    lm, lp : l_j(-1), l_j(+1) -- extrapolation of a line of solution-point
        values to the xi = -1 / +1 end (the flux point of that line)
    D : D[i, j] = l_j'(x_i), derivative of the solution polynomial at the points
    hm, hp : correction-derivative profiles h_-(x_i) = -g_L'(x_i) and
        h_+(x_i) = g_R'(x_i) = -g_L'(-x_i); a face of side s adds
        (common - own) * h_s along the line normal to it (see ``oracle.fr``)
    """

    def __init__(self, p, kind=DG):
        self.p = p
        self.Np = p + 1
        self.kind = kind
        self.x, self.w = gauss_legendre(self.Np)
        self.lm = lagrange(self.x, [-1.0])[0]
        self.lp = lagrange(self.x, [1.0])[0]
        self.D = lagrange_deriv(self.x, self.x)
        gLd = correction_left_deriv(p, kind, self.x)
        self.hm = -gLd
        self.hp = -correction_left_deriv(p, kind, -self.x)
        self.gll = gauss_lobatto(self.Np)
