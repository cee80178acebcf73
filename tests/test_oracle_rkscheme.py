"""Pins of the oracle's explicit integrator in coefficient form (the form that
takes Section 3.1's optimal scheme from its coefficients).

On a linear operator L (FR linear advection) one step of an s-stage scheme of
order s <= 4 is exactly the degree-s Taylor polynomial of exp(dt L) applied to
u; RK4 in coefficient form equals the classic RK4 step; a second-order scheme
converges at order 2 on the nonlinear Navier-Stokes residual; and the stage
times integrate a time-dependent source with the scheme's own quadrature
(trapezoid rule for Heun's method)."""
import math

import numpy as np
import pytest

from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import Advection, NavierStokes
from paper_2501_05709_gb300 import schemes as SC
from paper_2501_05709_gb300 import workloads as W


def _advection():
    nodes, conn = W.box_mesh(2, 3, 0.0, 1.0, q=1)
    m = Mesh(nodes, conn, 2)
    s = FRSolver(m, Advection(np.array([0.5, 0.2])))
    u = np.random.default_rng(3).standard_normal((m.E, 1, m.Nsp))
    return s, u


@pytest.mark.parametrize("name,order", [("euler", 1), ("heun2", 2), ("ssprk3", 3), ("williamson3", 3),
                                        ("rk4", 4)])
def test_step_is_the_taylor_polynomial_on_a_linear_operator(name, order):
    s, u = _advection()
    dt = 0.01
    term, taylor = u.copy(), u.copy()
    for k in range(1, order + 1):
        term = dt * s.residual(term) / k
        taylor = taylor + term
    assert np.max(np.abs(s.coef_step(u, dt, SC.SCHEMES[name]) - taylor)) < 1e-13
    taus, end = FRSolver.coef_stage_times(SC.SCHEMES[name])
    assert abs(end - 1.0) < 1e-15


def test_rk4_coefficients_equal_the_classic_step():
    nodes, conn = W.box_mesh(3, 3, 0.0, 1.0, q=2, curve=0.1, seed=3)
    m = Mesh(nodes, conn, 3)
    s = FRSolver(m, NavierStokes(3, mu=0.02))
    u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp, seed=5), 0, 1))
    a, b = s.coef_step(u, 1e-3, SC.RK4), s.rk4_step(u, 1e-3)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b - u)) + 1e-15 * np.max(np.abs(u))
    assert np.allclose(FRSolver.coef_stage_times(SC.RK4)[0], [0.0, 0.5, 0.5, 1.0], rtol=0, atol=1e-16)


def test_second_order_convergence_on_navier_stokes():
    nodes, conn = W.box_mesh(3, 2, 0.0, 1.0, q=2, curve=0.1, seed=3)
    m = Mesh(nodes, conn, 2)
    s = FRSolver(m, NavierStokes(3, mu=0.02))
    u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp, seed=5), 0, 1))
    T = 4e-3
    ref = u
    for _ in range(16):
        ref = s.rk4_step(ref, T / 16)
    err = []
    for n in (2, 4):
        v = u
        for _ in range(n):
            v = s.coef_step(v, T / n, SC.HEUN2)
        err.append(np.max(np.abs(v - ref)))
    rate = math.log2(err[0] / err[1])
    assert 1.8 < rate < 2.3, rate


def test_stage_times_give_the_trapezoid_rule_for_heun():
    # a spatially uniform energy source on a periodic quiescent box: one step
    # adds the scheme's quadrature of s(t); Heun's method is the trapezoid rule
    nodes, conn = W.box_mesh(3, 2, -1.0, 1.0, q=1)
    m = Mesh(nodes, conn, 2)
    A, f, t, dt = 0.05, 0.5, 0.21, 0.13
    ph = NavierStokes(3, mu=0.0, freestream=(1.0, np.zeros(3), 1.0 / 1.4))
    s = FRSolver(m, ph, source=[(A, 0.0, (0.0, 0.0, 0.0), f)])
    u = np.ascontiguousarray(np.moveaxis(W.uniform_state((m.E, m.Nsp), 1.0, [0.0, 0.0, 0.0], 1.0 / 1.4), 0, 1))
    sfun = lambda x: A * math.sin(2 * math.pi * f * x)
    v = s.coef_step(u, dt, SC.HEUN2, t=t)
    assert np.max(np.abs(v[:, 4] - u[:, 4] - dt / 2 * (sfun(t) + sfun(t + dt)))) <= 1e-14
    w = s.coef_step(u, dt, SC.RK4, t=t)
    simpson = dt / 6 * (sfun(t) + 4 * sfun(t + dt / 2) + sfun(t + dt))
    assert np.max(np.abs(w[:, 4] - u[:, 4] - simpson)) <= 1e-14
