"""Tensor-core precision modes (FR_TF32_TC, FR_BF16X3_TC: FP32 state and
point-wise arithmetic, the residual's gradient and divergence line operators
as m16n8k8 MMAs with FP32 accumulation) against the FP64 oracle, through the
C-ABI.

Stated bounds (relative L2 of the residual against the oracle), about 3-4x
the measured errors: curved box TF32 5e-2 / BF16x3 1e-3 (measured 1.4e-2 /
2.5e-4; FP32 3.3e-6), O-grid with walls 2e-2 / 5e-4 (3.9e-3 / 1.0e-4), p = 4
curved box 5e-2 / 1e-3 (1.2e-2 / 2.2e-4).  BF16x3 is always closer to the
oracle than TF32 and FP32 closer than both.  The low-Mach Taylor-Green
residual, a small difference of fluxes carrying p ~ 71, loses most of its
digits in TF32 (measured 0.38) and 1.1e-2 in BF16x3."""
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


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _residual(c, u, precision):
    from paper_2501_05709_gb300 import fr as F
    with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision)) as ctx:
        ud = torch.tensor(u, device="cuda", dtype=torch.float32)
        Rd = torch.empty_like(ud)
        F.fr_residual(ctx, ud, Rd)
        torch.cuda.synchronize()
        return Rd.double().cpu().numpy()


@pytest.mark.parametrize("name,tf32,bf16x3", [("ns3d_curved_p3", 5e-2, 1e-3), ("turned3d_curved_p3", 5e-2, 1e-3),
                                              ("rot3d_p3", 5e-2, 1e-3), ("ns3d_ogrid_p3", 2e-2, 5e-4),
                                              ("ns3d_p4_g2", 5e-2, 1e-3), ("tgv3d_p3", 1.0, 5e-2)])
def test_tensor_core_residual_against_the_oracle(name, tf32, bf16x3):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    R_or = s.residual(u)
    e32 = _rel(_residual(c, u, F.FR_FP32), R_or)
    etf = _rel(_residual(c, u, F.FR_TF32_TC), R_or)
    ebf = _rel(_residual(c, u, F.FR_BF16X3_TC), R_or)
    assert etf <= tf32 and ebf <= bf16x3
    assert e32 < ebf < etf


def test_tensor_core_steps_track_fp32():
    # three RK4 steps: the tensor-core modes stay within their residual error
    # of the FP32 path (state increments, relative L2)
    from paper_2501_05709_gb300 import fr as F
    c = make_case("ns3d_curved_p3")
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    out = {}
    for prec in (F.FR_FP32, F.FR_TF32_TC, F.FR_BF16X3_TC):
        with F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, prec)) as ctx:
            F.fr_state_set(ctx, u)
            F.fr_rk_step_graph(ctx, 3)
            out[prec] = F.fr_state_get(ctx) - u
    assert _rel(out[F.FR_TF32_TC], out[F.FR_FP32]) <= 5e-2
    assert _rel(out[F.FR_BF16X3_TC], out[F.FR_FP32]) <= 1e-3


def test_tensor_core_modes_reject_unbuilt_configurations():
    from paper_2501_05709_gb300 import fr as F
    for name in ("walls2d_p3", "ns3d_walls_p2"):
        c = make_case(name)
        with pytest.raises(F.FrError) as e:
            F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, F.FR_TF32_TC))
        assert e.value.code == F.FR_EINVAL
