"""Pin of the sampled-residual helper used by the full-size GPU parity tests:
on a small mesh it must reproduce the full oracle residual of the sample."""
import numpy as np

from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from paper_2501_05709_gb300 import workloads as W

from ._subset import sampled_residual


def test_sampled_residual_equals_full_residual():
    nodes, conn = W.ogrid_mesh(10, 3, 3, 0.2, r_outer=3.0, first_cell=0.05)
    rho, vel, p = W.freestream(0.2, 3.0)
    ph = NavierStokes(3, mu=1e-3, freestream=(rho, vel, p))
    m = Mesh(nodes, conn, 2)
    u = W.perturbed_uniform(m.E, m.Nsp, rho, vel, p, amplitude=0.02, seed=3)
    R = FRSolver(m, ph).residual(u)
    sample = [0, 7, 15, 31, 44, 89]

    def make(n, c):
        mm = Mesh(n, c, 2)
        return mm, FRSolver(mm, ph)

    Rs, ids = sampled_residual(make, nodes, conn, lambda ids, mm: u[ids], sample)
    assert np.max(np.abs(Rs - R[ids])) <= 1e-12 * np.max(np.abs(R))
