"""GPU parity of the adaptive time step (Section 3.1) through the C-ABI:
the step each candidate takes, RK4 steps with it, batched candidates, graph
replay, switching off, FP32."""
import numpy as np
import pytest

from ._cases import gpu_options, make_case, oracle_for

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


@pytest.mark.parametrize("name", ["ns3d_curved_p3", "ns3d_ogrid_p3", "euler3d_ogrid_p2", "vortex2d_p2"])
def test_adaptive_step_matches_oracle(name):
    from oracle import timestep as T
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    cfl = 0.4
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_set_adaptive_dt(ctx, cfl)
        F.fr_rk_step(ctx, 1)
        dt = F.fr_cand_dt(ctx, 0)
    assert abs(dt - T.cfl_dt(m, s.ph, u, cfl)) <= 1e-13 * dt


def test_adaptive_rk4_steps_fp64():
    from oracle import timestep as T
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    cfl = 0.3
    ref = u.copy()
    for _ in range(3):
        dt = T.cfl_dt(m, s.ph, ref, cfl)
        ref = s.rk4_step(ref, dt)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_set_adaptive_dt(ctx, cfl)
        F.fr_rk_step(ctx, 3)
        out = F.fr_state_get(ctx)
    assert relerr(out - u, ref - u) <= 1e-11


def test_batched_candidates_get_their_own_steps():
    from oracle import timestep as T
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_p1")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    nodes2 = np.asarray(c["nodes"]) * 0.5          # same connectivity, half the size
    from oracle.mesh import Mesh
    from oracle.fr import FRSolver
    m2 = Mesh(nodes2, c["conn"], c["p"])
    with F.fr_mesh_load([(c["nodes"], c["conn"]), (nodes2, c["conn"])], gpu_options(c)) as ctx:
        F.fr_state_set(ctx, np.concatenate([u, u]))
        F.fr_set_adaptive_dt(ctx, 0.5)
        F.fr_rk_step(ctx, 1)
        d0, d1 = F.fr_cand_dt(ctx, 0), F.fr_cand_dt(ctx, 1)
    assert abs(d0 - T.cfl_dt(m, s.ph, u, 0.5)) <= 1e-13 * d0
    assert abs(d1 - T.cfl_dt(m2, FRSolver(m2, s.ph).ph, u, 0.5)) <= 1e-13 * d1
    assert d1 < d0


def test_adaptive_graph_replay_and_switch_off():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_ogrid_p3")
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    opts = gpu_options(c)
    with F.fr_mesh_load((c["nodes"], c["conn"]), opts) as a, F.fr_mesh_load((c["nodes"], c["conn"]), opts) as b:
        for ctx in (a, b):
            F.fr_state_set(ctx, u)
            F.fr_set_adaptive_dt(ctx, 0.4)
        F.fr_rk_step(a, 4)
        F.fr_rk_step_graph(b, 4)
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))
        assert F.fr_cand_dt(a, 0) == F.fr_cand_dt(b, 0) != opts.dt
        F.fr_set_adaptive_dt(a, 0.0)
        assert F.fr_cand_dt(a, 0) == opts.dt


def test_adaptive_step_fp32():
    from oracle import timestep as T
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_ogrid_p3")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision=1)) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_set_adaptive_dt(ctx, 0.4)
        F.fr_rk_step(ctx, 1)
        dt = F.fr_cand_dt(ctx, 0)
    assert abs(dt - T.cfl_dt(m, s.ph, u, 0.4)) <= 2e-6 * dt
