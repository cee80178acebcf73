"""Batched candidates (Section 2.2's two-layer parallelism: all candidates of a
MADS poll advance together) against the FP64 oracle, candidate by candidate.

Three NACA 4-digit O-grids of uneven sizes (one with turned element frames)
share one FP64 context; each has its own time step.  Every candidate's
residual, three RK4 steps, wall forces and surface samples must match an
oracle run on that candidate alone."""
import math

import numpy as np
import pytest

from ._cases import fp64_tol

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    B.build()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


MU = 1.0 / 2300.0
DTS = [2e-4, 1.5e-4, 2.5e-4]


def _candidates():
    from paper_2501_05709_gb300 import workloads as W
    shapes = [((0.02, 0.4, 0.12), 12, 3), ((0.05, 0.3, 0.09), 16, 4), ((0.0, 0.4, 0.15), 10, 3)]
    out = []
    for k, (naca, nt, nr) in enumerate(shapes):
        nodes, conn = W.ogrid_mesh(nt, nr, 2, 0.2, r_outer=3.0, first_cell=0.05, naca=naca)
        if k == 1:
            nodes, conn, _ = W.reorient(nodes, conn, 3, seed=4)
        out.append((nodes, conn))
    return out


def _setup():
    from oracle.fr import FRSolver
    from oracle.mesh import Mesh
    from oracle.physics import NavierStokes
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    rho, vel, p = W.freestream(0.2, 3.0)
    a = math.radians(3.0)
    opts = F.options(order=3, precision=F.FR_FP64, viscous=True, mu=MU, rho_inf=rho, p_inf=p, vel_inf=tuple(vel),
                     dt=DTS[0], lift_dir=(-math.sin(a), math.cos(a), 0.0), drag_dir=(math.cos(a), math.sin(a), 0.0),
                     ref_area=0.2)
    meshes = _candidates()
    ph = NavierStokes(3, mu=MU, freestream=(rho, vel, p))
    solvers, states = [], []
    for k, (n, c) in enumerate(meshes):
        m = Mesh(n, c, 3)
        solvers.append(FRSolver(m, ph))
        states.append(W.perturbed_uniform(m.E, m.Nsp, rho, vel, p, amplitude=0.02, seed=k))
    return meshes, opts, solvers, states, (rho, vel, p), a


def test_batched_residual_and_steps_match_oracle_per_candidate():
    from paper_2501_05709_gb300 import fr as F
    meshes, opts, solvers, states, _, _ = _setup()
    u = np.concatenate(states)
    with F.fr_mesh_load(meshes, opts) as ctx:
        assert ctx.ncand == 3
        ud = torch.tensor(u, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.cpu().numpy()
        for k, d in enumerate(DTS):
            F.fr_set_cand_dt(ctx, k, d)
        F.fr_state_set(ctx, u)
        F.fr_rk_step(ctx, 3)
        out = [F.fr_state_get(ctx, cand=k) for k in range(3)]
    off = 0
    for k, (s, uk) in enumerate(zip(solvers, states)):
        E = len(uk)
        assert _rel(R[off:off + E], s.residual(uk)) <= fp64_tol(s.residual, uk), k
        ref = uk
        for _ in range(3):
            ref = s.rk4_step(ref, DTS[k])

        def three(v, s=s, k=k):
            for _ in range(3):
                v = s.rk4_step(v, DTS[k])
            return v - uk
        assert _rel(out[k] - uk, ref - uk) <= fp64_tol(three, uk, base=1e-11), k
        off += E


def test_batched_forces_and_samples_match_oracle_per_candidate():
    from oracle.sampling import locate, sample
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    meshes, opts, solvers, states, (rho, vel, p), a = _setup()
    y, _, _ = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.1, span=0.2)
    q = 0.5 * rho * np.dot(vel, vel) * 0.2
    with F.fr_mesh_load(meshes, opts) as ctx:
        F.fr_state_set(ctx, np.concatenate(states))
        hs = [F.fwh_register(ctx, k, y, 2) for k in range(3)]
        F.fr_rk_step(ctx, 1)
        fo = [F.fr_forces(ctx, k) for k in range(3)]
        hist = [F.fwh_history(ctx, h, len(y)) for h in hs]
    for k, (s, uk) in enumerate(zip(solvers, states)):
        Fo = s.wall_force(uk)
        cl = (Fo[0] * -np.sin(a) + Fo[1] * np.cos(a)) / q
        cd = (Fo[0] * np.cos(a) + Fo[1] * np.sin(a)) / q
        assert abs(fo[k][0] - cl) <= 1e-12 * max(1.0, abs(cl)), k
        assert abs(fo[k][1] - cd) <= 1e-12 * max(1.0, abs(cd)), k
        el, xi = locate(s.m, y)
        ref = sample(s.m, s.ph, uk, el, xi)
        assert hist[k].shape == (1, len(y), 5)
        assert np.max(np.abs(hist[k][0] - ref)) <= 1e-12 * np.max(np.abs(ref)), k
