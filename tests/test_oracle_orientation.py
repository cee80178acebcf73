"""Pins of the oracle on meshes whose neighbouring elements have turned local
frames (face orientation codes 1-7 in 3D, 1 in 2D).

The FR discretisation on tensor elements with Gauss-Legendre points is
invariant under the rotations of the reference element (the points are
symmetric, g_R(xi) = g_L(-xi), and the conservative-curl metrics are a vector
identity), so a mesh whose elements are relabelled by such rotations must give
the same residual, point by point after relabelling, as the base mesh.  A
wrong face-point map for any code breaks that equality; conservation and free
stream preservation must also survive the relabelling."""
import numpy as np
import pytest

from oracle.basis import DG, HUYNH_G2
from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from paper_2501_05709_gb300 import workloads as W


def _state(x, **kw):
    return np.ascontiguousarray(np.moveaxis(W.random_smooth_state(x, **kw), 0, 1))


def test_reorient_covers_every_code():
    nodes, conn = W.box_mesh(3, 3, 0.0, 1.0, q=2, curve=0.1, seed=3)
    _, c3, _ = W.reorient(nodes, conn, 3, seed=5)
    assert set(c3[:, :, 2].ravel().tolist()) == set(range(8))
    nodes, conn = W.box_mesh(2, 3, 0.0, 1.0, q=2, curve=0.1, seed=3)
    _, c2, _ = W.reorient(nodes, conn, 2, seed=5)
    assert set(c2[:, :, 2].ravel().tolist()) == {0, 1}


@pytest.mark.parametrize("dim,q,p,curve,kind,mu", [
    (2, 2, 3, 0.12, DG, 0.02), (2, 1, 2, 0.0, HUYNH_G2, 0.0),
    (3, 1, 3, 0.0, DG, 0.02), (3, 2, 3, 0.1, DG, 0.02), (3, 2, 2, 0.08, HUYNH_G2, 0.0),
    (3, 2, 4, 0.1, DG, 0.01)])
def test_residual_equivariant_under_element_rotations(dim, q, p, curve, kind, mu):
    nodes, conn = W.box_mesh(dim, 3, 0.0, 1.0, q=q, curve=curve, seed=3)
    n2, c2, rots = W.reorient(nodes, conn, dim, seed=5)
    m1, m2 = Mesh(nodes, conn, p, kind=kind), Mesh(n2, c2, p, kind=kind)
    assert m2.normal_mismatch < 1e-13
    assert np.allclose(W.relabel_points(np.moveaxis(m1.xsp, 2, 1), rots, p + 1, dim),
                       np.moveaxis(m2.xsp, 2, 1), rtol=0, atol=1e-14)
    u = _state(m1.xsp, seed=2)
    ph = NavierStokes(dim, mu=mu)
    R1 = FRSolver(m1, ph).residual(u)
    R2 = FRSolver(m2, ph).residual(W.relabel_points(u, rots, p + 1, dim))
    assert np.max(np.abs(W.relabel_points(R1, rots, p + 1, dim) - R2)) <= 1e-12 * np.max(np.abs(R1))


@pytest.mark.parametrize("mu", [0.0, 1.0 / 2300.0])
def test_ogrid_with_walls_and_far_field_equivariant(mu):
    # the boundary faces move to other local faces with the rotation
    nodes, conn = W.ogrid_mesh(12, 3, 2, 0.2, r_outer=3.0, first_cell=0.05)
    n2, c2, rots = W.reorient(nodes, conn, 3, seed=8)
    assert set(c2[:, :, 2][c2[:, :, 0] >= 0].tolist()) == set(range(8))
    p = 2
    m1, m2 = Mesh(nodes, conn, p), Mesh(n2, c2, p)
    rho, vel, pr = W.freestream(0.2, 3.0)
    ph = NavierStokes(3, mu=mu, freestream=(rho, vel, pr))
    u = W.perturbed_uniform(m1.E, m1.Nsp, rho, vel, pr, amplitude=0.02, seed=0)
    R1 = FRSolver(m1, ph).residual(u)
    R2 = FRSolver(m2, ph).residual(W.relabel_points(u, rots, p + 1, 3))
    assert np.max(np.abs(W.relabel_points(R1, rots, p + 1, 3) - R2)) <= 1e-11 * np.max(np.abs(R1))
    # the wall force is a sum over the same wall points
    f1 = FRSolver(m1, ph).wall_force(u)
    f2 = FRSolver(m2, ph).wall_force(W.relabel_points(u, rots, p + 1, 3))
    assert np.allclose(f1, f2, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim,q,p,curve", [(2, 2, 3, 0.12), (3, 2, 3, 0.1)])
def test_conservation_and_free_stream_on_turned_elements(dim, q, p, curve):
    nodes, conn = W.box_mesh(dim, 3, 0.0, 1.0, q=q, curve=curve, seed=7)
    n2, c2, _ = W.reorient(nodes, conn, dim, seed=11)
    m = Mesh(n2, c2, p)
    ph = NavierStokes(dim, mu=0.02)
    u = _state(m.xsp, seed=2)
    R = FRSolver(m, ph).residual(u)
    tot = np.einsum("evs,es,s->v", R, m.J, m.sp_weights())
    scale = np.einsum("evs,es,s->v", np.abs(R), m.J, m.sp_weights())
    assert np.all(np.abs(tot) <= 1e-13 * scale.max())
    vel = [0.4, -0.3, 0.25][:dim]
    uu = np.ascontiguousarray(np.moveaxis(W.uniform_state((m.E, m.Nsp), 1.2, vel, 0.9), 0, 1))
    assert np.max(np.abs(FRSolver(m, ph).residual(uu))) < 1e-11
