"""Pins of the variable-order (sponge zone) oracle: the 1D projection against
the Legendre closed forms, and the residual with order caps against free-stream
preservation, conservation and invariance of the capped spaces."""
import math

import numpy as np
import pytest

from oracle import sponge as SP
from oracle.basis import gauss_legendre
from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from paper_2501_05709_gb300 import workloads as W


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_projection_closed_forms(p):
    x, w = gauss_legendre(p + 1)
    for q in range(p + 1):
        P = SP.projection_1d(p, q)
        assert np.allclose(P @ P, P, atol=1e-14)                               # idempotent
        for k in range(p + 1):
            v = SP.legendre_values(k, x)
            ref = v if k <= q else np.zeros_like(v)
            assert np.allclose(P @ v, ref, atol=1e-13)                         # keeps modes <= q, drops the rest
        Wm = np.diag(w)
        assert np.allclose(Wm @ P, (Wm @ P).T, atol=1e-14)                     # orthogonal in the GL inner product
        for k in range(q + 1):                                                 # exact on monomials of degree <= q
            assert np.allclose(P @ x ** k, x ** k, atol=1e-13)
    assert np.allclose(SP.projection_1d(p, p), np.eye(p + 1), atol=1e-14)
    assert np.allclose(SP.legendre_values(3, np.array([0.3])), 0.5 * (5 * 0.3 ** 3 - 3 * 0.3))


def _periodic(p=3, n=3, curve=0.0, q=1, seed=2):
    nodes, conn = W.box_mesh(3, n, 0.0, 2 * math.pi, q=q, curve=curve, seed=seed)
    return Mesh(nodes, conn, p)


def test_uncapped_residual_is_unchanged():
    m = _periodic()
    ph = NavierStokes(3, mu=0.01)
    u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp, seed=3), 0, 1))
    R0 = FRSolver(m, ph).residual(u)
    R1 = FRSolver(m, ph, caps=np.full(m.E, 3)).residual(u)
    assert np.array_equal(R0, R1)


def test_free_stream_in_capped_elements():
    m = _periodic(curve=0.1, q=2)
    ph = NavierStokes(3, mu=0.01)
    caps = np.random.default_rng(0).integers(0, 4, m.E)
    u = W.perturbed_uniform(m.E, m.Nsp, 1.1, [0.3, -0.2, 0.1], 2.0, amplitude=0.0)
    R = FRSolver(m, ph, caps=caps).residual(u)
    assert np.max(np.abs(R)) < 1e-11


def test_conservation_with_caps():
    m = _periodic(p=3, n=3)
    ph = NavierStokes(3, mu=0.01)
    caps = np.random.default_rng(1).integers(0, 4, m.E)
    u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp, seed=4), 0, 1))
    u = SP.project(m, u, caps)
    R = FRSolver(m, ph, caps=caps).residual(u)
    tot = np.einsum("evs,es,s->v", R, m.J, m.sp_weights())
    scale = np.einsum("evs,es,s->v", np.abs(R), m.J, m.sp_weights())
    assert np.all(np.abs(tot) <= 1e-13 * scale.max())


def test_rk4_stays_in_the_capped_spaces():
    m = _periodic(p=3, n=2)
    ph = NavierStokes(3, mu=0.01)
    caps = np.array([0, 1, 2, 3, 1, 0, 2, 3])
    u = SP.project(m, np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp, seed=5), 0, 1)), caps)
    v = FRSolver(m, ph, caps=caps).rk4_step(u, 1e-3)
    assert np.max(np.abs(SP.project(m, v, caps) - v)) <= 1e-13 * np.max(np.abs(v))
    e0 = np.nonzero(caps == 0)[0][0]
    assert np.ptp(v[e0], axis=-1).max() <= 1e-13 * np.max(np.abs(v[e0]))   # P0: one value per element
    assert np.max(np.abs(v - u)) > 1e-6                                       # it did move
