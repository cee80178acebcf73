"""Seeded parity cases shared by the GPU tests: a mesh from the workload
generators, physics constants, and a state evaluated at the solution points."""
import math

import numpy as np

from paper_2501_05709_gb300 import workloads as W

GAMMA = 1.4


def _conserved_at(xsp, fn, **kw):
    return np.ascontiguousarray(np.moveaxis(fn(xsp, **kw), 0, 1))


def make_case(name):
    """Returns dict(nodes, conn, p, kind, mu, visc, freestream, state(xsp) -> u, dt)."""
    c = {"kind": 0, "mu": 0.0, "visc": False, "freestream": (1.0, np.zeros(3), 1.0), "dt": 1e-3}
    if name == "vortex2d_p2":
        c["nodes"], c["conn"] = W.box_mesh(2, 16, -5.0, 5.0, q=1)
        c["p"] = 2
        c["freestream"] = (1.0, np.array([0.5 * math.sqrt(GAMMA), 0.0, 0.0]), 1.0)
        c["state"] = lambda x: _conserved_at(x, W.isentropic_vortex, t=0.0)
    elif name == "ns2d_curved_p3_g2":
        c["nodes"], c["conn"] = W.box_mesh(2, [5, 3], 0.0, 1.0, q=2, curve=0.1, seed=2)
        c.update(p=3, kind=1, mu=0.01, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=4)
    elif name == "tgv3d_p3":
        c["nodes"], c["conn"] = W.box_mesh(3, [5, 5, 3], 0.0, 2 * math.pi, q=1)
        c.update(p=3, mu=1.0 / 1600.0, visc=True, dt=2.5e-4)
        c["state"] = lambda x: _conserved_at(x, W.taylor_green, mach=0.1)
    elif name == "tgv3d_p4":
        # affine box at p = 4: two warps per element, the pipelined face kernel
        c["nodes"], c["conn"] = W.box_mesh(3, [4, 3, 3], 0.0, 2 * math.pi, q=1)
        c.update(p=4, mu=1.0 / 1600.0, visc=True, dt=1.5e-4)
        c["state"] = lambda x: _conserved_at(x, W.taylor_green, mach=0.1)
    elif name == "rot3d_p4":
        ax = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + math.sin(0.5) * K + (1 - math.cos(0.5)) * K @ K
        nodes, c["conn"] = W.box_mesh(3, [3, 3, 2], 0.0, 1.0, q=1)
        c["nodes"] = np.ascontiguousarray(np.asarray(nodes) @ R.T)
        c.update(p=4, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(np.asarray(x) @ R, W.random_smooth_state, seed=15)
    elif name == "ns3d_curved_p3":
        c["nodes"], c["conn"] = W.box_mesh(3, 3, 0.0, 1.0, q=2, curve=0.1, seed=3)
        c.update(p=3, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=5)
    elif name == "ns3d_walls_p2":
        c["nodes"], c["conn"] = W.box_mesh(3, [3, 4, 2], 0.0, [1.5, 1.0, 0.5], q=2, walls_y=True, curve=0.05)
        c.update(p=2, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=6, periods=[1.5, 1.0, 0.5])
    elif name in ("ns3d_ogrid_p3", "euler3d_ogrid_p2", "ns3d_ogrid_p4"):
        # curved O-grid with a no-slip body and a characteristic far field (at
        # p = 4 the boundary kernels on two warps per element)
        c["nodes"], c["conn"] = W.ogrid_mesh(12, 3, 2, 0.2, r_outer=3.0, first_cell=0.05)
        rho, vel, p = W.freestream(0.2, 3.0)
        c["freestream"] = (rho, vel, p)
        if name == "ns3d_ogrid_p3":
            c.update(p=3, mu=1.0 / 2300.0, visc=True, dt=2e-4)
        elif name == "ns3d_ogrid_p4":
            c.update(p=4, mu=1.0 / 2300.0, visc=True, dt=1e-4)
        else:
            c.update(p=2, dt=2e-4)
        nsp = (c["p"] + 1) ** 3
        E = len(c["nodes"])
        c["state"] = lambda x: W.perturbed_uniform(E, nsp, rho, vel, p, amplitude=0.02, seed=0)
    elif name in ("rot3d_p3", "rot3d_euler_p2"):
        # a periodic box turned about (1, 2, 3): affine but not axis-aligned
        # (full metric matrices); the state is periodic in the box's own frame
        ax = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + math.sin(0.5) * K + (1 - math.cos(0.5)) * K @ K
        nodes, c["conn"] = W.box_mesh(3, [4, 3, 3], 0.0, 1.0, q=1)
        c["nodes"] = np.ascontiguousarray(np.asarray(nodes) @ R.T)
        if name == "rot3d_p3":
            c.update(p=3, mu=0.02, visc=True)
        else:
            c.update(p=2)
        c["state"] = lambda x: _conserved_at(np.asarray(x) @ R, W.random_smooth_state, seed=10)
    elif name in ("walls3d_p2", "rotwalls3d_p3", "rotwalls3d_p4"):
        # straight-sided channel with no-slip walls on both y faces: axis-aligned
        # (walls3d_p2) or turned about (1, 2, 3) (rotwalls3d_p3, rotwalls3d_p4)
        nodes, c["conn"] = W.box_mesh(3, [3, 4, 2], 0.0, [1.5, 1.0, 0.5], q=1, walls_y=True)
        R = np.eye(3)
        if name != "walls3d_p2":
            ax = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
            K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
            R = np.eye(3) + math.sin(0.5) * K + (1 - math.cos(0.5)) * K @ K
        c["nodes"] = np.ascontiguousarray(np.asarray(nodes) @ R.T)
        c.update(p={"walls3d_p2": 2, "rotwalls3d_p3": 3, "rotwalls3d_p4": 4}[name], mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(np.asarray(x) @ R, W.random_smooth_state, seed=11,
                                             periods=[1.5, 1.0, 0.5])
    elif name == "farfield3d_euler_p2":
        # axis-aligned box with characteristic far field on every face, Euler
        c["nodes"], c["conn"] = W.box_mesh(3, [3, 3, 2], -1.0, 1.0, q=1, periodic=[False] * 3,
                                           bc_tag=W.BC_FARFIELD)
        rho, vel, p = W.freestream(0.3, 5.0)
        c["freestream"] = (rho, vel, p)
        c.update(p=2)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=12, periods=[2.0, 2.0, 2.0])
    elif name == "walls2d_p3":
        c["nodes"], c["conn"] = W.box_mesh(2, [4, 3], 0.0, [2.0, 1.0], q=1, walls_y=True)
        c.update(p=3, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=13, periods=[2.0, 1.0])
    elif name == "ns3d_p1":
        c["nodes"], c["conn"] = W.box_mesh(3, 3, 0.0, 1.0, q=1, curve=0.08, seed=8)
        c.update(p=1, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=7)
    elif name == "ns3d_p4_g2":
        c["nodes"], c["conn"] = W.box_mesh(3, [3, 2, 2], 0.0, 1.0, q=2, curve=0.1, seed=9)
        c.update(p=4, kind=1, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=8)
    elif name in ("turned3d_curved_p3", "turned3d_affine_p3", "turned2d_curved_p2_g2", "turned3d_affine_p4",
                  "turned3d_curved_p4"):
        # every element's local frame turned by a seeded rotation of the
        # reference element: faces carry all orientation codes (at p = 4 the
        # face phases run on two warps per element)
        if name == "turned3d_curved_p3":
            nodes, conn = W.box_mesh(3, 3, 0.0, 1.0, q=2, curve=0.1, seed=3)
            c.update(p=3, mu=0.02, visc=True)
        elif name == "turned3d_affine_p3":
            nodes, conn = W.box_mesh(3, [4, 3, 3], 0.0, 1.0, q=1)
            c.update(p=3, mu=0.02, visc=True)
        elif name == "turned3d_affine_p4":
            nodes, conn = W.box_mesh(3, [3, 3, 2], 0.0, 1.0, q=1)
            c.update(p=4, mu=0.02, visc=True)
        elif name == "turned3d_curved_p4":
            nodes, conn = W.box_mesh(3, [3, 2, 2], 0.0, 1.0, q=2, curve=0.1, seed=4)
            c.update(p=4, mu=0.02, visc=True)
        else:
            nodes, conn = W.box_mesh(2, [4, 3], 0.0, 1.0, q=2, curve=0.1, seed=2)
            c.update(p=2, kind=1, mu=0.01, visc=True)
        c["nodes"], c["conn"], _ = W.reorient(nodes, conn, len(nodes[0][0]), seed=5)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=14)
    elif name in ("turned_ogrid_p3", "turned_ogrid_euler_p2"):
        nodes, conn = W.ogrid_mesh(12, 3, 2, 0.2, r_outer=3.0, first_cell=0.05)
        c["nodes"], c["conn"], _ = W.reorient(nodes, conn, 3, seed=8)
        rho, vel, p = W.freestream(0.2, 3.0)
        c["freestream"] = (rho, vel, p)
        if name == "turned_ogrid_p3":
            c.update(p=3, mu=1.0 / 2300.0, visc=True, dt=2e-4)
        else:
            c.update(p=2, dt=2e-4)
        nsp = (c["p"] + 1) ** 3
        E = len(c["nodes"])
        c["state"] = lambda x: W.perturbed_uniform(E, nsp, rho, vel, p, amplitude=0.02, seed=1)
    elif name == "single_element":
        c["nodes"], c["conn"] = W.box_mesh(3, 1, 0.0, 1.0, q=1)
        c.update(p=3, mu=0.02, visc=True)
        c["state"] = lambda x: _conserved_at(x, W.random_smooth_state, seed=9)
    else:
        raise KeyError(name)
    return c


CASES = ["vortex2d_p2", "ns2d_curved_p3_g2", "tgv3d_p3", "ns3d_curved_p3", "ns3d_walls_p2", "ns3d_ogrid_p3",
         "euler3d_ogrid_p2", "ns3d_p1", "ns3d_p4_g2", "single_element", "rot3d_p3", "walls3d_p2", "rotwalls3d_p3",
         "farfield3d_euler_p2", "walls2d_p3", "rot3d_euler_p2", "turned3d_curved_p3", "turned3d_affine_p3",
         "turned2d_curved_p2_g2", "turned_ogrid_p3", "turned_ogrid_euler_p2", "tgv3d_p4", "rot3d_p4",
         "turned3d_affine_p4", "turned3d_curved_p4", "rotwalls3d_p4", "ns3d_ogrid_p4"]


def ulp_floor(fn, u, draws=2, seed=0):
    """Relative L2 change of fn(u) when every input value moves by one unit in
    the last place: the round-off floor of the computation itself."""
    rng = np.random.default_rng(seed)
    ref = fn(u)
    worst = 0.0
    for _ in range(draws):
        up = u * (1.0 + rng.choice([-1.0, 1.0], size=u.shape) * 2.0 ** -53)
        d = fn(up) - ref
        worst = max(worst, float(np.linalg.norm(d.ravel()) / np.linalg.norm(ref.ravel())))
    return worst


def coef_floor(solver, u, pick=None, draws=2, seed=1):
    """Relative L2 change of the oracle residual when every operator
    coefficient (D, extrapolation and correction weights) and every metric
    value (S, |J|, normals) moves by one unit in the last place: the floor set
    by how the data of the discretisation itself is rounded.  The solver's
    energy sources and per-element degrees are kept."""
    import copy

    from oracle.fr import FRSolver
    rng = np.random.default_rng(seed)

    def jig(a):
        return a * (1.0 + rng.choice([-1.0, 1.0], size=np.shape(a)) * 2.0 ** -53)

    ref = solver.residual(u)
    if pick is not None:
        ref = ref[pick]
    worst = 0.0
    for _ in range(draws):
        m2 = copy.copy(solver.m)
        r2 = copy.copy(solver.m.ref)
        for name in ("D", "lm", "lp", "hm", "hp"):
            setattr(r2, name, jig(getattr(r2, name)))
        m2.ref = r2
        for name in ("S", "J", "N"):
            setattr(m2, name, jig(getattr(m2, name)))
        R2 = FRSolver(m2, solver.ph, source=solver.source, caps=solver.caps).residual(u)
        if pick is not None:
            R2 = R2[pick]
        worst = max(worst, float(np.linalg.norm((R2 - ref).ravel()) / np.linalg.norm(ref.ravel())))
    return worst


def fp64_tol(fn, u, base=1e-12, solver=None, pick=None):
    """The FP64 parity bar: 1e-12 relative L2, or 4x the oracle's own floor
    where the problem's conditioning puts that floor above 2.5e-13.  The floor
    is the larger of the 1-ulp state floor and (when the solver is given) the
    1-ulp operator/metric floor."""
    floor = ulp_floor(fn, u)
    if solver is not None:
        floor = max(floor, coef_floor(solver, u, pick))
    return max(base, 4.0 * floor)


def oracle_for(c):
    from oracle.fr import FRSolver
    from oracle.mesh import Mesh
    from oracle.physics import NavierStokes
    m = Mesh(c["nodes"], c["conn"], c["p"], kind=c["kind"])
    dim = m.dim
    rho, vel, p = c["freestream"]
    ph = NavierStokes(dim, mu=c["mu"], viscous=c["visc"], freestream=(rho, np.asarray(vel)[:dim], p))
    return m, FRSolver(m, ph)


def gpu_options(c, precision=0):
    from paper_2501_05709_gb300 import fr as F
    rho, vel, p = c["freestream"]
    return F.options(order=c["p"], correction=c["kind"], precision=precision, viscous=c["visc"], mu=c["mu"],
                     rho_inf=rho, p_inf=p, vel_inf=tuple(vel), dt=c["dt"])
