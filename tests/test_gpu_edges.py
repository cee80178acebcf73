"""Edge cases through the C-ABI: the shortest FW-H record, a full sampling
history, a source far from every solution point, zero-amplitude source, and a
single-element adaptive step."""
import numpy as np
import pytest

from ._cases import fp64_tol, gpu_options, make_case, oracle_for

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


def test_fwh_shortest_record_matches_oracle():
    # nt = 5, the least the 4th-order time derivative accepts, a compact surface
    # so that the observer window is not empty
    from oracle import fwh as O
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    y, n, dS = W.sphere_surface(0.01, 6, 2 * np.pi / 12)
    M = [0.2, 0.0, 0.1]
    dt = 0.004
    tau = dt * np.arange(5)
    fld = W.monopole_field(y[None], tau[:, None], M)
    hist = np.concatenate([fld["rho"][..., None], fld["vel"], fld["p"][..., None]], axis=-1)
    obs = np.array([[3.0, 1.0, 0.0]])
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    p_out, nt_out, t0 = F.fwh_integrate(dev(hist), dev(y), dev(n), dev(dS), dt, 0.0, obs, M, 340.75, 1.234, fld["p0"])
    ts, pp = O.fwh_integrate(hist, y, n, dS, dt, obs[0], M, 340.75, 1.234, fld["p0"])
    assert nt_out[0] == len(ts) and nt_out[0] >= 1
    assert relerr(p_out[0, :nt_out[0]].cpu().numpy(), pp) <= 1e-12


def test_sampling_history_overflow_is_reported():
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    c = make_case("ns3d_ogrid_p3")
    m, _ = oracle_for(c)
    y, _, _ = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.2, span=0.2)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_state_set(ctx, c["state"](m.xsp))
        h = F.fwh_register(ctx, 0, y, 2, 1)
        F.fr_rk_step(ctx, 3)                       # three samples into a history of two
        with pytest.raises(F.FrError):
            F.fwh_history(ctx, h, len(y))
        F.fwh_clear(ctx, h)
        F.fr_rk_step(ctx, 1)
        assert F.fwh_history(ctx, h, len(y)).shape[0] == 1


@pytest.mark.parametrize("src", [[(0.05, 100.0, (40.0, 40.0, 40.0), 0.5)], [(0.0, 10.0, (0.5, 0.5, 0.5), 0.5)]])
def test_inert_sources_leave_the_residual(src):
    # a source far from every solution point, or of zero amplitude, changes nothing
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_p1")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_set_source(ctx, 0, src, 0.3)
        ud = torch.tensor(u, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        assert relerr(Rd.cpu().numpy(), s.residual(u)) <= fp64_tol(s.residual, u)


def test_single_element_adaptive_step():
    from oracle import timestep as T
    from paper_2501_05709_gb300 import fr as F
    c = make_case("single_element")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c)) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_set_adaptive_dt(ctx, 0.3)
        F.fr_rk_step(ctx, 2)
        dt = F.fr_cand_dt(ctx, 0)
        out = F.fr_state_get(ctx)
    ref = u.copy()
    for _ in range(2):
        d = T.cfl_dt(m, s.ph, ref, 0.3)
        ref = s.rk4_step(ref, d)
    assert abs(dt - d) <= 1e-13 * d
    assert relerr(out - u, ref - u) <= 1e-11
