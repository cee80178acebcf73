"""GPU tests of the explicit integrator in coefficient form (fr_set_rk_scheme)
and of the device-side non-finite detection, through the C-ABI.

* RK4 entered as coefficients reproduces the built-in RK4 bit for bit (FP64
  and FP32, affine, curved and walled meshes, graph replay, forces, samples).
* Other schemes (forward Euler, Heun, Shu-Osher SSP RK3, Williamson's 2N RK3;
  odd stage counts use a third trace buffer) match the oracle's step in FP64,
  with and without the time-dependent energy source (stage times).
* A step that blows up sets the candidate's flag: fr_state_get and fr_forces
  return FR_ENONFINITE, only for the diverging candidate of a batch, and
  fr_state_set clears it.  NaNs produced by arithmetic do not fault the GPU.
"""
import math

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


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _load(c, precision=0):
    from paper_2501_05709_gb300 import fr as F
    return F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision))


@pytest.mark.parametrize("name", ["tgv3d_p3", "ns3d_curved_p3", "ns3d_ogrid_p3", "rot3d_euler_p2"])
@pytest.mark.parametrize("precision", [0, 1])
def test_rk4_coefficients_reproduce_the_builtin_step_bitwise(name, precision):
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import schemes as SC
    from paper_2501_05709_gb300 import workloads as W
    c = make_case(name)
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    y, _, _ = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.1, span=0.2)
    walls = name == "ns3d_ogrid_p3"
    with _load(c, precision) as a, _load(c, precision) as b:
        F.fr_set_rk_scheme(b, SC.RK4)
        for ctx in (a, b):
            F.fr_state_set(ctx, u)
        if walls:
            ha, hb = F.fwh_register(a, 0, y, 8), F.fwh_register(b, 0, y, 8)
        F.fr_rk_step(a, 2)
        F.fr_rk_step(b, 2)
        F.fr_rk_step_graph(a, 2)
        F.fr_rk_step_graph(b, 2)
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))
        if walls:
            assert np.array_equal(F.fr_forces(a, 0), F.fr_forces(b, 0))
            assert np.array_equal(F.fwh_history(a, ha, len(y)), F.fwh_history(b, hb, len(y)))
        F.fr_set_rk_scheme(b, None)          # back to the built-in RK4
        F.fr_rk_step(a, 1)
        F.fr_rk_step(b, 1)
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))


@pytest.mark.parametrize("scheme", ["euler", "heun2", "ssprk3", "williamson3"])
@pytest.mark.parametrize("name", ["ns3d_curved_p3", "ns3d_ogrid_p3"])
def test_coefficient_schemes_match_the_oracle(scheme, name):
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import schemes as SC
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    dt = c["dt"] if scheme != "euler" else 0.25 * c["dt"]
    coef = SC.SCHEMES[scheme]

    def two(v):
        for _ in range(2):
            v = s.coef_step(v, dt, coef)
        return v - u
    ref = two(u) + u
    opts = gpu_options(c)
    opts.dt = dt
    with F.fr_mesh_load((c["nodes"], c["conn"]), opts) as ctx:
        F.fr_set_rk_scheme(ctx, coef)
        F.fr_state_set(ctx, u)
        F.fr_rk_step_graph(ctx, 2)
        out = F.fr_state_get(ctx)
    assert _rel(out - u, ref - u) <= fp64_tol(two, u, base=1e-11)


@pytest.mark.parametrize("scheme", ["heun2", "ssprk3"])
def test_coefficient_schemes_with_source_stage_times(scheme):
    from oracle.fr import FRSolver
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import schemes as SC
    src = [(0.05, 100.0, (0.45, 0.52, 0.48), 0.5), (0.02, 40.0, (0.2, 0.7, 0.3), 1.3)]
    c = make_case("ns3d_curved_p3")
    m, s0 = oracle_for(c)
    s = FRSolver(m, s0.ph, source=src)
    u = c["state"](m.xsp)
    t0, dt = 0.37, c["dt"]
    coef = SC.SCHEMES[scheme]

    def two(v):
        for k in range(2):
            v = s.coef_step(v, dt, coef, t=t0 + k * dt)
        return v - u
    ref = two(u) + u
    with _load(c) as ctx:
        F.fr_set_rk_scheme(ctx, coef)
        F.fr_set_source(ctx, 0, src, t0)
        F.fr_state_set(ctx, u)
        F.fr_rk_step(ctx, 2)
        out = F.fr_state_get(ctx)
        assert abs(F.fr_source_time(ctx, 0) - (t0 + 2 * dt)) <= 1e-15
    assert _rel(out - u, ref - u) <= fp64_tol(two, u, base=1e-11)


def test_inconsistent_scheme_is_rejected():
    from paper_2501_05709_gb300 import fr as F
    c = make_case("tgv3d_p3")
    with _load(c) as ctx:
        with pytest.raises(F.FrError) as e:
            F.fr_set_rk_scheme(ctx, [(1.0, 0.0, 0.5, 0.0, 0.0, 0.0)])   # advances u by dt/2
        assert e.value.code == F.FR_EINVAL


@pytest.mark.parametrize("precision", [0, 1])
def test_blow_up_sets_the_nonfinite_flag(precision):
    from paper_2501_05709_gb300 import fr as F
    c = make_case("tgv3d_p3")
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    opts = gpu_options(c, precision)
    opts.dt = 5.0                       # far beyond the stable step
    with F.fr_mesh_load((c["nodes"], c["conn"]), opts) as ctx:
        F.fr_state_set(ctx, u)
        assert not F.fr_nonfinite(ctx)
        F.fr_rk_step_graph(ctx, 12)
        assert F.fr_nonfinite(ctx) and F.fr_nonfinite(ctx, 0)
        with pytest.raises(F.FrError) as e:
            F.fr_state_get(ctx)
        assert e.value.code == F.FR_ENONFINITE
        dev = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(F.FrError) as e:
            F.fr_state_get(ctx, out=dev)
        assert e.value.code == F.FR_ENONFINITE
        # a new state clears the flag; a stable step keeps it clear
        F.fr_state_set(ctx, u)
        assert not F.fr_nonfinite(ctx)
        F.fr_set_cand_dt(ctx, 0, c["dt"])
        F.fr_rk_step(ctx, 2)
        assert not F.fr_nonfinite(ctx)
        assert np.isfinite(F.fr_state_get(ctx)).all()


def test_only_the_diverging_candidate_is_flagged():
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    c = make_case("ns3d_ogrid_p3")
    rho, vel, p = c["freestream"]
    nsp = (c["p"] + 1) ** 3
    opts = gpu_options(c)
    opts.lift_dir[1], opts.drag_dir[0], opts.ref_area = 1.0, 1.0, 0.2
    E = len(c["nodes"])
    u = np.concatenate([W.perturbed_uniform(E, nsp, rho, vel, p, amplitude=0.02, seed=k) for k in range(2)])
    with F.fr_mesh_load([(c["nodes"], c["conn"])] * 2, opts) as ctx:
        F.fr_set_cand_dt(ctx, 1, 0.5)   # candidate 1 diverges
        F.fr_state_set(ctx, u)
        F.fr_rk_step(ctx, 12)
        assert not F.fr_nonfinite(ctx, 0) and F.fr_nonfinite(ctx, 1) and F.fr_nonfinite(ctx, -1)
        f0 = F.fr_forces(ctx, 0)
        assert np.isfinite(f0).all()
        with pytest.raises(F.FrError) as e:
            F.fr_forces(ctx, 1)
        assert e.value.code == F.FR_ENONFINITE
        assert np.isfinite(F.fr_state_get(ctx, cand=0)).all()
        with pytest.raises(F.FrError):
            F.fr_state_get(ctx, cand=1)
        F.fr_state_set(ctx, u[E:], cand=1)
        assert not F.fr_nonfinite(ctx)
