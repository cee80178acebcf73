"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle, element
by element on seeded inputs (FP64: relative L2 <= 1e-12)."""
import numpy as np
import pytest

from ._cases import CASES, fp64_tol, gpu_options, make_case, oracle_for

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


def _load(c, precision=0):
    from paper_2501_05709_gb300 import fr as F
    return F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision))


@pytest.mark.parametrize("name", CASES)
def test_residual_fp64(name):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    R_or = s.residual(u)
    with _load(c) as ctx:
        ud = torch.tensor(u, device="cuda")
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        R = Rd.cpu().numpy()
    assert relerr(R, R_or) <= fp64_tol(s.residual, u)


METRIC_PATH = {"vortex2d_p2": 2, "tgv3d_p3": 2, "single_element": 2, "rot3d_p3": 1, "walls3d_p2": 2,
               "rotwalls3d_p3": 1, "farfield3d_euler_p2": 2, "walls2d_p3": 2, "rot3d_euler_p2": 1,
               "turned3d_affine_p3": 1, "tgv3d_p4": 2, "rot3d_p4": 1, "turned3d_affine_p4": 1,
               "rotwalls3d_p4": 1}


@pytest.mark.parametrize("name", CASES)
def test_affine_detection(name):
    """Straight-sided meshes take the per-element metric path (round-off in
    analytically zero metric components is not variation), axis-aligned ones
    the diagonal-metric path; curved meshes keep per-point metrics."""
    c = make_case(name)
    with _load(c) as ctx:
        assert ctx.affine == METRIC_PATH.get(name, 0)


@pytest.mark.parametrize("name", ["vortex2d_p2", "tgv3d_p3", "ns3d_ogrid_p3", "ns3d_walls_p2", "rot3d_p3",
                                  "rotwalls3d_p3", "farfield3d_euler_p2", "turned3d_curved_p3", "turned_ogrid_p3",
                                  "turned2d_curved_p2_g2", "tgv3d_p4", "rot3d_p4", "turned3d_affine_p4",
                                  "turned3d_curved_p4", "rotwalls3d_p4", "ns3d_ogrid_p4"])
def test_rk4_steps_fp64(name):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    ref = u.copy()
    for _ in range(3):
        ref = s.rk4_step(ref, c["dt"])
    with _load(c) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_rk_step(ctx, 3)
        out = F.fr_state_get(ctx)

    def three_steps(v):
        for _ in range(3):
            v = s.rk4_step(v, c["dt"])
        return v - u

    assert relerr(out - u, ref - u) <= fp64_tol(three_steps, u, base=1e-11)
    assert relerr(out, ref) <= 1e-14


def test_graph_replay_matches_direct_stepping():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_ogrid_p3")
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    with _load(c) as a, _load(c) as b:
        F.fr_state_set(a, u)
        F.fr_state_set(b, u)
        F.fr_rk_step(a, 4)
        F.fr_rk_step_graph(b, 4)
        ua, ub = F.fr_state_get(a), F.fr_state_get(b)
        fa, fb = F.fr_forces(a, 0), F.fr_forces(b, 0)
    assert np.array_equal(ua, ub)
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("name", ["tgv3d_p3", "ns3d_curved_p3", "rot3d_p3"])
def test_conservation_on_gpu(name):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    with _load(c) as ctx:
        F.fr_state_set(ctx, u)
        before = F.fr_integrals(ctx)
        F.fr_rk_step(ctx, 5)
        after = F.fr_integrals(ctx)
    nv = m.dim + 2
    scale = np.abs(before[:nv]).max()
    assert np.all(np.abs(after[:nv] - before[:nv]) <= 1e-12 * scale)


@pytest.mark.parametrize("name", ["ns3d_ogrid_p3", "turned_ogrid_p3", "ns3d_ogrid_p4"])
def test_forces_match_oracle(name):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    Fo = s.wall_force(u)
    rho, vel, p = c["freestream"]
    a = np.deg2rad(3.0)
    opts = gpu_options(c)
    opts.lift_dir[0], opts.lift_dir[1] = -np.sin(a), np.cos(a)
    opts.drag_dir[0], opts.drag_dir[1] = np.cos(a), np.sin(a)
    opts.ref_area = 0.2
    with F.fr_mesh_load((c["nodes"], c["conn"]), opts) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_rk_step(ctx, 1)
        out = F.fr_forces(ctx, 0)
    q = 0.5 * rho * np.dot(vel, vel) * 0.2
    cl = (Fo[0] * -np.sin(a) + Fo[1] * np.cos(a)) / q
    cd = (Fo[0] * np.cos(a) + Fo[1] * np.sin(a)) / q
    assert abs(out[0] - cl) <= 1e-12 * max(1.0, abs(cl))
    assert abs(out[1] - cd) <= 1e-12 * max(1.0, abs(cd))
    assert out[4] == 1.0


@pytest.mark.parametrize("name", ["ns3d_ogrid_p3", "turned_ogrid_p3", "ns3d_ogrid_p4"])
def test_sampling_matches_oracle(name):
    from oracle.sampling import locate, sample
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    y, _, _ = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.05, span=0.2)
    el, xi = locate(m, y)
    ref = sample(m, s.ph, u, el, xi)
    with _load(c) as ctx:
        F.fr_state_set(ctx, u)
        h = F.fwh_register(ctx, 0, y, 4)
        F.fwh_sample(ctx, h)
        F.fwh_sample(ctx, h)
        hist = F.fwh_history(ctx, h, len(y))
    assert hist.shape == (2, len(y), 5)
    assert np.max(np.abs(hist[0] - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(hist[0], hist[1])


def test_fwh_integrate_matches_oracle():
    from oracle import fwh as O
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    y, n, dS = W.sphere_surface(1.0, 12, 2 * np.pi / 18)
    M = [0.5, 0.1, 0.5]
    dt = 0.004
    tau = dt * np.arange(150)
    fld = W.monopole_field(y[None], tau[:, None], M)
    hist = np.concatenate([fld["rho"][..., None], fld["vel"], fld["p"][..., None]], axis=-1)
    obs = np.array([[20.0, 0.0, 0.0], [0.0, -15.0, 3.0]])
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    for Lspan, nc in ((0.0, 1), (0.7, 5)):
        p_out, nt_out, t0 = F.fwh_integrate(dev(hist), dev(y), dev(n), dev(dS), dt, 0.0, obs, M, 340.75, 1.234,
                                            fld["p0"], Lspan=Lspan, ncopies=nc)
        p_out = p_out.cpu().numpy()
        for o in range(len(obs)):
            ts, pp = O.fwh_integrate(hist, y, n, dS, dt, obs[o], M, 340.75, 1.234, fld["p0"], Lspan=Lspan,
                                     ncopies=nc)
            assert nt_out[o] == len(ts)
            assert abs(t0[o] - ts[0]) <= 1e-12
            assert relerr(p_out[o, :nt_out[o]], pp) <= 1e-12


def test_fp32_residual_error_is_bounded():
    # stated FP32 bound: relative L2 of the residual against the FP64 oracle.
    # Rounding only the state to float moves the oracle's own residual by
    # 2.2e-6 .. 2.7e-6 on the curved and turned cases, but by 3.8e-4 (p = 3)
    # and 6.9e-4 (p = 4) on the low-Mach Taylor-Green box, whose residual is a
    # small difference of fluxes carrying p ~ 71; the bounds are 2.6 .. 4.4x
    # those floors there.
    from paper_2501_05709_gb300 import fr as F
    for name, tol in (("ns3d_curved_p3", 1e-5), ("ns3d_ogrid_p3", 1e-4), ("tgv3d_p3", 1e-3), ("rot3d_p3", 1e-5),
                      ("rot3d_p4", 1e-5), ("tgv3d_p4", 3e-3)):
        c = make_case(name)
        m, s = oracle_for(c)
        u = c["state"](m.xsp)
        R_or = s.residual(u)
        with _load(c, precision=1) as ctx:
            ud = torch.tensor(u, device="cuda", dtype=torch.float32)
            Rd = torch.empty_like(ud)
            F.fr_residual(ctx, ud, Rd)
            torch.cuda.synchronize()
            R = Rd.double().cpu().numpy()
        assert relerr(R, R_or) <= tol, name


def test_diagonal_metric_path_matches_the_full_one():
    # the axis-aligned path (metric path 2) skips the exact-zero metric terms
    # and agrees with the oracle in both precisions; the turned box of
    # rot3d_p3 covers the full affine path (1) in the tests above
    from paper_2501_05709_gb300 import fr as F
    c = make_case("tgv3d_p3")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    for prec, tol in ((0, fp64_tol(s.residual, u)), (1, 1e-3)):
        with _load(c, precision=prec) as ctx:
            assert ctx.affine == 2
            dt = torch.float64 if prec == 0 else torch.float32
            ud = torch.tensor(u, device="cuda", dtype=dt)
            Rd = torch.empty_like(ud)
            F.fr_residual(ctx, ud, Rd)
            torch.cuda.synchronize()
            assert relerr(Rd.double().cpu().numpy(), s.residual(u)) <= tol


def test_autotune_keeps_results():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("tgv3d_p3")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    R_or = s.residual(u)
    tol = fp64_tol(s.residual, u)
    with _load(c) as ctx:
        F.fr_state_set(ctx, u)
        F.fr_autotune(ctx)
        for epb in (1, 3, 7):
            F.fr_set_tile(ctx, epb)
            ud = torch.tensor(u, device="cuda")
            Rd = torch.empty_like(ud)
            F.fr_residual(ctx, ud, Rd)
            torch.cuda.synchronize()
            assert relerr(Rd.cpu().numpy(), R_or) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_accepts_unaligned_buffers(precision):
    # a caller's state may start at any element offset (e.g. a sliced tensor)
    from paper_2501_05709_gb300 import fr as F
    c = make_case("tgv3d_p3")
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    dt = torch.float64 if precision == 0 else torch.float32
    with _load(c, precision) as ctx:
        big = torch.zeros(u.size + 1, dtype=dt, device="cuda")
        big[1:] = torch.tensor(u.ravel(), dtype=dt, device="cuda")
        Rbig = torch.zeros(u.size + 3, dtype=dt, device="cuda")
        F.fr_residual(ctx, big[1:], Rbig[3:])
        ref = torch.empty(u.shape, dtype=dt, device="cuda")
        F.fr_residual(ctx, torch.tensor(u, dtype=dt, device="cuda"), ref)
        torch.cuda.synchronize()
    assert torch.equal(Rbig[3:].view(u.shape), ref)


def test_sampling_interval():
    # every=3 over 7 steps: records at steps 0, 3, 6 equal to every-step sampling
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    c = make_case("ns3d_ogrid_p3")
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    y, _, _ = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.1, span=0.2)
    with _load(c, 1) as a, _load(c, 1) as b:
        F.fr_state_set(a, u)
        F.fr_state_set(b, u)
        ha = F.fwh_register(a, 0, y, 3, 3)
        hb = F.fwh_register(b, 0, y, 7, 1)
        F.fr_rk_step_graph(a, 7)
        F.fr_rk_step(b, 7)
        ra = F.fwh_history(a, ha, len(y))
        rb = F.fwh_history(b, hb, len(y))
    assert ra.shape[0] == 3 and rb.shape[0] == 7
    assert np.array_equal(ra, rb[[0, 3, 6]])
