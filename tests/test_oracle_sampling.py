"""Pins of the oracle's data-surface location and sampling."""
import numpy as np

from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from oracle.sampling import locate, sample
from paper_2501_05709_gb300 import workloads as W


def test_sampling_exact_for_linear_field_on_curved_ogrid():
    nodes, conn = W.ogrid_mesh(24, 4, 2, 0.2, r_outer=3.0, first_cell=0.05)
    m = Mesh(nodes, conn, 3)
    x = m.xsp
    rho = 1.0 + 0.1 * x[..., 0] - 0.05 * x[..., 1]
    # conserved variables linear in x (rho, rho V, rho E): of degree 2 in xi
    # on these quadratic elements, so this checks the point location and the
    # interpolation up to degree 2 (test_oracle_boundaries checks exactness on
    # tensor polynomials of the full degree p)
    u = np.zeros((m.E, 5, m.Nsp))
    u[:, 0] = rho
    u[:, 1] = 0.5 + 0.02 * x[..., 1]
    u[:, 2] = -0.1 + 0.03 * x[..., 0]
    u[:, 3] = 0.01 * x[..., 2]
    u[:, 4] = 5.0 + 0.2 * x[..., 0]
    y, nrm, area = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.1, span=0.2)
    el, xi = locate(m, y)
    s = sample(m, NavierStokes(3), u, el, xi)
    r = 1.0 + 0.1 * y[:, 0] - 0.05 * y[:, 1]
    mom = np.stack([0.5 + 0.02 * y[:, 1], -0.1 + 0.03 * y[:, 0], 0.01 * y[:, 2]], axis=1)
    Et = 5.0 + 0.2 * y[:, 0]
    p = 0.4 * (Et - 0.5 * np.sum(mom ** 2, axis=1) / r)
    assert np.allclose(s[:, 0], r, atol=1e-12, rtol=0)
    assert np.allclose(s[:, 1:4], mom / r[:, None], atol=1e-12, rtol=0)
    assert np.allclose(s[:, 4], p, atol=1e-12, rtol=0)


def test_locate_recovers_solution_point_positions():
    nodes, conn = W.box_mesh(3, 3, 0.0, 1.0, q=2, curve=0.1, seed=4)
    m = Mesh(nodes, conn, 2)
    pick = [(0, 5), (7, 13), (26, 0)]
    pts = np.array([m.xsp[e, s] for e, s in pick])
    el, xi = locate(m, pts)
    gl = m.ref.x
    for (e, s), ee, xx in zip(pick, el, xi):
        assert ee == e
        want = [gl[s % 3], gl[(s // 3) % 3], gl[s // 9]]
        assert np.allclose(xx, want, atol=1e-12)
