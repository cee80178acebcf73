"""Pins of the oracle's energy source term (Appendix D, Eq. D.1) and of the
stage times of the classic RK4 update with a time-dependent source."""
import math

import numpy as np

from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from paper_2501_05709_gb300 import workloads as W

GAMMA = 1.4


def _quiescent(p=3, n=3, lo=-1.0, hi=1.0, periodic=False, source=None):
    nodes, conn = W.box_mesh(3, n, lo, hi, q=1, periodic=[periodic] * 3, bc_tag=W.BC_FARFIELD)
    m = Mesh(nodes, conn, p)
    ph = NavierStokes(3, mu=0.0, viscous=False, freestream=(1.0, np.zeros(3), 1.0 / GAMMA))
    s = FRSolver(m, ph, source=source)
    u = np.ascontiguousarray(np.moveaxis(W.uniform_state((m.E, m.Nsp), 1.0, [0, 0, 0], 1.0 / GAMMA), 0, 1))
    return m, s, u


def test_quiescent_residual_is_the_source():
    # a uniform state at rest in a far-field box has R = 0: only Eq. D.1 remains
    src = [(0.05, 100.0, (0.1, -0.2, 0.05), 0.5)]
    m, s, u = _quiescent(source=src)
    t = 0.37
    R = s.residual(u, t=t)
    r2 = np.sum((m.xsp - np.array([0.1, -0.2, 0.05])) ** 2, axis=-1)
    ex = 0.05 * np.exp(-100.0 * r2) * math.sin(2 * math.pi * 0.5 * t)
    # round-off of the flux divergence of the uniform state (p = 1/gamma) is ~1e-14
    assert np.max(np.abs(R[:, 4] - ex)) <= 1e-12
    assert np.max(np.abs(R[:, :4])) <= 1e-12


def test_gaussian_source_volume_integral():
    # sum_sp w |J| s = A (pi/k)^(3/2) sin(2 pi f t) for a Gaussian well inside the box
    A, k, f, t = 0.05, 10.0, 0.5, 0.3
    m, s, u = _quiescent(n=8, lo=-2.0, hi=2.0, source=[(A, k, (0.0, 0.0, 0.0), f)])
    R = s.residual(u, t=t)
    w = m.sp_weights()
    tot = np.sum(R[:, 4] * m.J * w[None, :])
    ex = A * (math.pi / k) ** 1.5 * math.sin(2 * math.pi * f * t)
    assert abs(tot - ex) <= 1e-3 * abs(ex)   # GL quadrature of the Gaussian: 1.2e-4 here


def test_rk4_stage_times_simpson():
    # a spatially uniform source (k = 0) keeps a periodic uniform state uniform,
    # so one RK4 step adds Simpson's rule of s(t): dt/6 (s(t) + 4 s(t+dt/2) + s(t+dt))
    A, f, t, dt = 0.05, 0.5, 0.21, 0.13
    m, s, u = _quiescent(n=2, periodic=True, source=[(A, 0.0, (0.0, 0.0, 0.0), f)])
    v = s.rk4_step(u, dt, t=t)
    sfun = lambda x: A * math.sin(2 * math.pi * f * x)
    simpson = dt / 6 * (sfun(t) + 4 * sfun(t + dt / 2) + sfun(t + dt))
    assert np.max(np.abs(v[:, 4] - u[:, 4] - simpson)) <= 1e-14
    assert np.max(np.abs(v[:, :4] - u[:, :4])) <= 1e-14


def test_no_source_is_unchanged():
    m, s, u = _quiescent(source=None)
    assert np.max(np.abs(s.residual(u, t=1.0))) <= 1e-12
