"""GPU parity of variable polynomial degree by element (the sponge zones of
Section 3.1: degree-q elements with faces at the degree-p points) through the
C-ABI, against the oracle: residual, state projection, RK4 steps, graph
replay, per-candidate degrees, removal, conservation, the Euler path, the FP32
bound, and that the reduced elements run their own kernels."""
import numpy as np
import pytest

from ._cases import fp64_tol, gpu_options, make_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    B.build()


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _caps(E, p, seed):
    # every degree 0..p present, the rest drawn at random
    rng = np.random.default_rng(seed)
    caps = rng.integers(0, p + 1, size=E)
    caps[: min(E, p + 1)] = np.arange(min(E, p + 1))
    return caps.astype(np.int32)


def _oracle(c, caps):
    from oracle.fr import FRSolver
    from oracle.mesh import Mesh
    from oracle.physics import NavierStokes
    m = Mesh(c["nodes"], c["conn"], c["p"], kind=c["kind"])
    rho, vel, p = c["freestream"]
    ph = NavierStokes(m.dim, mu=c["mu"], viscous=c["visc"], freestream=(rho, np.asarray(vel)[:m.dim], p))
    return m, FRSolver(m, ph, caps=caps)


@pytest.mark.parametrize("name", ["ns3d_curved_p3", "vortex2d_p2", "ns3d_walls_p2", "ns3d_p4_g2", "ns3d_p1"])
def test_residual_with_orders_fp64(name):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=3)
    m, s = _oracle(c, caps)
    u = c["state"](m.xsp)
    R_or = s.residual(u)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_set_element_order(ctx, caps)
        ud = torch.tensor(u, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.cpu().numpy()
    assert relerr(R, R_or) <= fp64_tol(s.residual, u)
    # elements of degree q carry no modes above q
    from oracle.sponge import project
    assert np.abs(project(m, R, caps) - R).max() <= 1e-12 * np.abs(R).max()


def test_state_is_projected_on_order_set_and_state_set():
    from oracle.sponge import project
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=5)
    m, _ = _oracle(c, None)
    u = c["state"](m.xsp)
    ref = project(m, u, caps)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_set_element_order(ctx, caps)
        a = F.fr_state_get(ctx)
        F.fr_state_set(ctx, u)
        b = F.fr_state_get(ctx)
    assert relerr(a, ref) <= 1e-14
    assert np.array_equal(a, b)
    full = caps == c["p"]
    assert np.array_equal(a[full], u[full])


def test_rk4_steps_with_orders_fp64():
    from oracle.sponge import project
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=7)
    m, s = _oracle(c, caps)
    u = project(m, c["state"](m.xsp), caps)
    dt = 2e-3
    ref = u.copy()
    for _ in range(3):
        ref = s.rk4_step(ref, dt)
    opts = gpu_options(c)
    opts.dt = dt
    with F.fr_mesh_load((c["nodes"], c["conn"]), opts) as ctx:
        F.fr_set_element_order(ctx, caps)
        F.fr_state_set(ctx, u)
        F.fr_rk_step(ctx, 3)
        out = F.fr_state_get(ctx)
    assert relerr(out - u, ref - u) <= 1e-11
    assert np.abs(project(m, out, caps) - out).max() <= 1e-12 * np.abs(out).max()
    # the orders did act: without them the increment differs
    _, s0 = _oracle(c, None)
    ref0 = u.copy()
    for _ in range(3):
        ref0 = s0.rk4_step(ref0, dt)
    assert relerr(ref0 - u, ref - u) > 1e-6


def test_graph_replay_with_orders_matches_direct():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_p1")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=11)
    m, _ = _oracle(c, None)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as a, \
            F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as b:
        for ctx in (a, b):
            F.fr_set_element_order(ctx, caps)
            F.fr_state_set(ctx, u)
        F.fr_rk_step(a, 5)
        F.fr_rk_step_graph(b, 5)
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))


def test_serial_and_forked_reduced_kernels_agree():
    # a step runs the reduced-degree kernels on their own streams beside the
    # degree-p kernels; the instrumented step (fr_profile_step) runs every
    # kernel on one stream, one after the other: both write disjoint elements,
    # so the states agree bit for bit
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_walls_p2")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=5)
    m, _ = _oracle(c, None)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as a, \
            F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as b:
        for ctx in (a, b):
            F.fr_set_element_order(ctx, caps)
            F.fr_state_set(ctx, u)
        F.fr_rk_step_graph(a, 3)
        ms, n = F.fr_profile_step(b, 3)
        assert n[5] > 0 and n[2] > 0
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))


def test_orders_on_one_candidate_and_removal():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_walls_p2")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=13)
    m, s = _oracle(c, caps)
    _, s0 = _oracle(c, None)
    u = c["state"](m.xsp)
    mesh = (c["nodes"], c["conn"])
    with F.fr_mesh_load([mesh, mesh], gpu_options(c)) as ctx:
        F.fr_set_element_order(ctx, caps, cand=1)
        ud = torch.tensor(np.concatenate([u, u]), device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.cpu().numpy()
        assert relerr(R[:E], s0.residual(u)) <= fp64_tol(s0.residual, u)
        assert relerr(R[E:], s.residual(u)) <= fp64_tol(s.residual, u)
        F.fr_set_element_order(ctx, None, cand=1)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.cpu().numpy()
        assert relerr(R[E:], s0.residual(u)) <= fp64_tol(s0.residual, u)
        with pytest.raises(F.FrError):
            F.fr_set_element_order(ctx, np.full(E, c["p"] + 1), cand=0)
        with pytest.raises(F.FrError):
            F.fr_set_element_order(ctx, np.full(E, -1), cand=0)


def test_all_degree_p_is_the_plain_path():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_p1")
    E = len(c["conn"])
    m, _ = _oracle(c, None)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as a, \
            F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as b:
        F.fr_set_element_order(b, np.full(E, c["p"], np.int32))
        for ctx in (a, b):
            F.fr_state_set(ctx, u)
            F.fr_rk_step(ctx, 2)
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))


def test_conservation_with_orders_on_periodic_box():
    # the projection keeps each element's mean: on a periodic affine box the
    # integrals of the conserved variables stay put
    from paper_2501_05709_gb300 import fr as F
    c = make_case("tgv3d_p3")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=17)
    m, _ = _oracle(c, None)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_set_element_order(ctx, caps)
        F.fr_state_set(ctx, u)
        i0 = F.fr_integrals(ctx, 0)
        F.fr_rk_step(ctx, 10)
        i1 = F.fr_integrals(ctx, 0)
    nv = m.dim + 2
    scale = np.abs(i0[:nv]).max()
    assert np.abs(i1[:nv] - i0[:nv]).max() <= 1e-12 * scale


def test_orders_fp32_bound():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=19)
    m, s = _oracle(c, caps)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision=1)) as ctx:
        F.fr_set_element_order(ctx, caps)
        ud = torch.tensor(u, dtype=torch.float32, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.double().cpu().numpy()
    assert relerr(R, s.residual(u)) <= 1e-5


def test_euler_with_orders_fp64():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("euler3d_ogrid_p2")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=23)
    m, s = _oracle(c, caps)
    u = c["state"](m.xsp)
    R_or = s.residual(u)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_set_element_order(ctx, caps)
        ud = torch.tensor(u, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.cpu().numpy()
    assert relerr(R, R_or) <= fp64_tol(s.residual, u)


def test_reduced_elements_run_their_own_kernels():
    # per RK stage one face and one residual launch per reduced degree present
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=29)
    m, _ = _oracle(c, None)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_state_set(ctx, u)
        _, n0 = F.fr_profile_step(ctx, 1)
        F.fr_set_element_order(ctx, caps)
        F.fr_state_set(ctx, u)
        _, n1 = F.fr_profile_step(ctx, 1)
    nq = len(set(int(q) for q in caps) - {c["p"]})
    assert n0[5] == 0 and n1[5] == 4 * 2 * nq
    assert n1[2] == n0[2] == 4


def test_source_needs_a_uniform_degree():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_p1")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=31)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_set_element_order(ctx, caps)
        with pytest.raises(F.FrError) as e:
            F.fr_set_source(ctx, 0, [(1.0, 10.0, (0.5, 0.5, 0.5), 2.0)])
        assert e.value.code == F.FR_EINVAL
        F.fr_set_element_order(ctx, None)
        F.fr_set_source(ctx, 0, [(1.0, 10.0, (0.5, 0.5, 0.5), 2.0)])
        with pytest.raises(F.FrError) as e:
            F.fr_set_element_order(ctx, caps)
        assert e.value.code == F.FR_EINVAL


def test_tensor_core_mode_with_orders():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    E = len(c["conn"])
    caps = _caps(E, c["p"], seed=37)
    m, s = _oracle(c, caps)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision=F.FR_BF16X3_TC)) as ctx:
        F.fr_set_element_order(ctx, caps)
        ud = torch.tensor(u, dtype=torch.float32, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.double().cpu().numpy()
    assert relerr(R, s.residual(u)) <= 1e-3
