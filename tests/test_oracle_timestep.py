"""Pins of the adaptive time-step oracle against closed forms: the element
length of affine boxes, the rate of a uniform flow, scaling and the viscous
term."""
import math

import numpy as np

from oracle import timestep as T
from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from paper_2501_05709_gb300 import workloads as W

GAMMA = 1.4


def _box(n, lo, hi, p, curve=0.0, q=1):
    nodes, conn = W.box_mesh(3, n, lo, hi, q=q, curve=curve, seed=1)
    return Mesh(nodes, conn, p)


def test_element_length_of_affine_boxes():
    m = _box([4, 2, 5], 0.0, [2.0, 3.0, 1.0], 2)
    assert np.allclose(T.element_length(m), min(2.0 / 4, 3.0 / 2, 1.0 / 5), rtol=1e-13, atol=0)
    m = _box(3, -1.0, 2.0, 3)
    assert np.allclose(T.element_length(m), 1.0, rtol=1e-13, atol=0)


def test_uniform_flow_closed_form():
    p, n, L = 3, 4, 2.0
    m = _box(n, 0.0, L, p)
    vel, pr, rho = np.array([0.3, -0.4, 1.2]), 2.5, 1.3
    u = W.perturbed_uniform(m.E, m.Nsp, rho, vel, pr, amplitude=0.0)
    ph = NavierStokes(3, mu=0.01, viscous=True)
    h = L / n
    lam = (np.linalg.norm(vel) + math.sqrt(GAMMA * pr / rho)) * (p + 1) ** 2 / h + 0.01 / rho * (p + 1) ** 4 / h ** 2
    assert abs(T.cfl_dt(m, ph, u, 0.5) - 0.5 / lam) <= 1e-13 * 0.5 / lam
    ph0 = NavierStokes(3, mu=0.0, viscous=False)
    lam0 = (np.linalg.norm(vel) + math.sqrt(GAMMA * pr / rho)) * (p + 1) ** 2 / h
    assert abs(T.cfl_dt(m, ph0, u, 0.5) - 0.5 / lam0) <= 1e-13 * 0.5 / lam0


def test_scaling_and_local_maximum():
    # doubling every coordinate doubles the inviscid step; a fast spot sets the step
    m1 = _box(3, 0.0, 1.0, 2, curve=0.1, q=2)
    m2 = _box(3, 0.0, 2.0, 2, curve=0.1, q=2)
    u = W.perturbed_uniform(m1.E, m1.Nsp, 1.0, [0.2, 0.0, 0.0], 1.0, amplitude=0.0)
    ph = NavierStokes(3, mu=0.0, viscous=False)
    assert abs(T.cfl_dt(m2, ph, u, 1.0) / T.cfl_dt(m1, ph, u, 1.0) - 2.0) <= 1e-12
    u2 = u.copy()
    u2[5, 1, 7] *= 10.0                       # one point 10x faster (and more energetic)
    lam = T.spectral_rate(m1, ph, u2)
    assert np.argmax(lam) == 5
    assert T.cfl_dt(m1, ph, u2, 1.0) < T.cfl_dt(m1, ph, u, 1.0)
