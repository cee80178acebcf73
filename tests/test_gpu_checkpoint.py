"""Checkpoint and resume through the C-ABI: a run interrupted after k steps,
its state read with fr_state_get, the context destroyed, and the run resumed
in a new context from fr_state_set (with the source time and per-candidate
steps restored) ends bit for bit where the uninterrupted run ends.  The traces
of a set state are recomputed by the same warp routine the stage epilogue
uses, and the float state survives the double round trip exactly, so this
holds in FP64 and FP32."""
import numpy as np
import pytest

from ._cases import gpu_options, make_case, oracle_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SRC = [(0.05, 100.0, (0.45, 0.52, 0.48), 0.5)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    B.build()


@pytest.mark.parametrize("name", ["ns3d_curved_p3", "ns3d_ogrid_p3", "turned_ogrid_p3"])
@pytest.mark.parametrize("precision", [0, 1])
def test_resume_from_checkpoint_is_bitwise(name, precision):
    from paper_2501_05709_gb300 import fr as F
    c = make_case(name)
    m, _ = oracle_for(c)
    u = c["state"](m.xsp)
    with_src = name == "ns3d_curved_p3"
    n, k = 6, 2

    def load():
        ctx = F.fr_mesh_load((c["nodes"], c["conn"]), gpu_options(c, precision))
        F.fr_set_cand_dt(ctx, 0, 0.9 * c["dt"])
        return ctx

    with load() as a:
        if with_src:
            F.fr_set_source(a, 0, SRC, 0.1)
        F.fr_state_set(a, u)
        F.fr_rk_step_graph(a, n)
        want = F.fr_state_get(a)
    with load() as b:
        if with_src:
            F.fr_set_source(b, 0, SRC, 0.1)
        F.fr_state_set(b, u)
        F.fr_rk_step_graph(b, k)
        ck = F.fr_state_get(b)
        t_ck = F.fr_source_time(b, 0) if with_src else None
    with load() as r:
        if with_src:
            F.fr_set_source(r, 0, SRC, t_ck)
        F.fr_state_set(r, ck)
        F.fr_rk_step(r, n - k)
        got = F.fr_state_get(r)
    assert np.array_equal(got, want)
