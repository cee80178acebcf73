"""Design geometry of the optimisation loop (Section 3.4): NACA 4-digit
sections of either camber sign and the angle of attack as a turn of the
section about the quarter chord (host only)."""
import math

import numpy as np

from paper_2501_05709_gb300 import cases as C
from paper_2501_05709_gb300 import workloads as W


def test_negative_camber_mirrors_positive_camber():
    beta = np.linspace(0.0, 2 * np.pi, 401)[:-1]
    xp, yp = W.naca4_surface(0.05, 0.4, 0.12, beta)
    xn, yn = W.naca4_surface(-0.05, 0.4, 0.12, beta)
    # the lower surface of -m is the mirrored upper surface of +m (beta -> 2pi - beta)
    mirror = (2 * np.pi - beta) % (2 * np.pi)
    xm, ym = W.naca4_surface(0.05, 0.4, 0.12, mirror)
    assert np.allclose(xn, xm, atol=1e-12) and np.allclose(yn, -ym, atol=1e-12)
    assert np.max(yp) > np.max(yn)                 # positive camber lifts the upper surface


def test_angle_of_attack_turns_the_section_nose_up():
    X0 = [2.0, 4.0, 12.0, 0.0]
    X1 = [2.0, 4.0, 12.0, 8.0]
    n0, c0, te0 = C.design_mesh(X0, n_theta=24, n_r=4, n_z=1)
    n1, c1, te1 = C.design_mesh(X1, n_theta=24, n_r=4, n_z=1)
    assert np.array_equal(c0, c1)
    a = math.radians(8.0)
    assert np.allclose(te0, (1.0, 0.0), atol=1e-12)
    assert np.allclose(te1, (0.25 + 0.75 * math.cos(a), -0.75 * math.sin(a)), atol=1e-12)
    # a rigid turn about the quarter chord: distances to it kept, z untouched,
    # the trailing edge below the chord line and the leading edge above it
    r0 = np.hypot(n0[..., 0] - 0.25, n0[..., 1])
    r1 = np.hypot(n1[..., 0] - 0.25, n1[..., 1])
    assert np.allclose(r0, r1, atol=1e-12) and np.array_equal(n0[..., 2], n1[..., 2])
    ang0 = np.arctan2(n0[..., 1], n0[..., 0] - 0.25)
    ang1 = np.arctan2(n1[..., 1], n1[..., 0] - 0.25)
    d = np.angle(np.exp(1j * (ang1 - ang0)))
    assert np.allclose(d[r0 > 1e-9], -a, atol=1e-9)
