"""Pins of the oracle's reference-element operators against closed forms."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import basis


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_gauss_lobatto_points(n):
    g = basis.gauss_lobatto(n)
    assert g[0] == -1.0 and g[-1] == 1.0
    assert np.allclose(g, -g[::-1], atol=1e-15)
    # interior points are the roots of P'_{n-1}: closed forms for n = 3, 4
    if n == 3:
        assert np.allclose(g, [-1, 0, 1])
    if n == 4:
        assert np.allclose(g, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_and_derivative_exact_on_polynomials(p):
    x, _ = basis.gauss_legendre(p + 1)
    ys = np.linspace(-1, 1, 7)
    L = basis.lagrange(x, ys)
    D = basis.lagrange_deriv(x, ys)
    for k in range(p + 1):
        assert np.allclose(L @ x ** k, ys ** k, atol=1e-13)
        dk = k * ys ** (k - 1) if k else np.zeros_like(ys)
        assert np.allclose(D @ x ** k, dk, atol=1e-12)
    assert np.allclose(basis.lagrange(x, x), np.eye(p + 1), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dg_correction_is_right_radau(p):
    c = basis.correction_left(p, basis.DG)
    assert abs(npleg.legval(-1.0, c) - 1.0) < 1e-14
    assert abs(npleg.legval(1.0, c)) < 1e-14
    # closed form g_DG'(-1) = -(p+1)^2 / 2
    assert abs(basis.correction_left_deriv(p, basis.DG, [-1.0])[0] + (p + 1) ** 2 / 2) < 1e-12
    # Radau property: orthogonal to every polynomial of degree <= p-1
    xq, wq = np.polynomial.legendre.leggauss(p + 4)
    for j in range(p):
        assert abs(np.dot(wq, npleg.legval(xq, c) * xq ** j)) < 1e-14
    # degree exactly p+1
    assert abs(c[-1]) > 0.1 and len(c) == p + 2


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_huynh_g2(p):
    c = basis.correction_left(p, basis.HUYNH_G2)
    assert abs(npleg.legval(-1.0, c) - 1.0) < 1e-14
    assert abs(npleg.legval(1.0, c)) < 1e-14
    d = basis.correction_left_deriv(p, basis.HUYNH_G2, [-1.0, 1.0])
    assert abs(d[0] + p * (p + 1) / 2) < 1e-12      # g2'(-1) = -p(p+1)/2
    assert abs(d[1]) < 1e-12                        # double root at +1


@pytest.mark.parametrize("kind", [basis.DG, basis.HUYNH_G2])
def test_correction_profiles_integrate_to_one(kind):
    # int_{-1}^{1} h_+ = g_R(1) - g_R(-1) = 1: GL quadrature of the profiles
    for p in range(1, 5):
        r = basis.Ref1D(p, kind)
        assert abs(np.dot(r.w, r.hp) - 1.0) < 1e-13
        assert abs(np.dot(r.w, r.hm) - 1.0) < 1e-13
        assert np.allclose(r.hp, r.hm[::-1], atol=1e-13)
