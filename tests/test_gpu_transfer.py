"""State transfers through the C-ABI.  From and to pinned host memory the
conversion kernel reads or writes the host array directly over the CPU-GPU
link; from and to pageable memory the library stages the doubles on the
device; from and to device memory it converts in place.  All three give the
same state bit for bit, in FP64 and FP32, for the whole state and for one
candidate of a batch."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    B.build()


def _pinned(shape):
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_pageable_and_device_transfers_agree(precision):
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    nodes, conn = W.box_mesh(3, 5, 0.0, 2 * math.pi, q=1)
    opts = F.options(order=3, precision=precision, viscous=True, mu=1e-3, p_inf=1 / (1.4 * 0.04), dt=1e-4)
    with F.fr_mesh_load((nodes, conn), opts) as a, F.fr_mesh_load((nodes, conn), opts) as b, \
            F.fr_mesh_load((nodes, conn), opts) as c:
        x = F.fr_sp_coords(a)
        u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(x, seed=3, periods=[2 * math.pi] * 3), 0, 1))
        hp = _pinned(u.shape)
        hp[...] = u
        F.fr_state_set(a, u)                                   # pageable: staged copy
        F.fr_state_set(b, hp)                                  # pinned: read over the link
        F.fr_state_set(c, torch.tensor(u, device="cuda"))      # device
        ga = F.fr_state_get(a)
        gb = F.fr_state_get(b, out=_pinned(u.shape))           # pinned: written over the link
        gc = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        F.fr_state_get(c, out=gc)
        torch.cuda.synchronize()
        assert np.array_equal(ga, gb) and np.array_equal(ga, gc.cpu().numpy())
        if precision == 0:
            assert np.array_equal(ga, u)
        else:
            assert np.array_equal(ga, u.astype(np.float32).astype(np.float64))
        # and the states step alike
        for ctx in (a, b, c):
            F.fr_rk_step_graph(ctx, 2)
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(b))
        assert np.array_equal(F.fr_state_get(a), F.fr_state_get(c))


def test_pinned_transfer_of_one_candidate():
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    meshes = [W.box_mesh(3, n, 0.0, 2 * math.pi, q=1) for n in (3, 4)]
    opts = F.options(order=2, precision=1, viscous=True, mu=1e-3, p_inf=1 / (1.4 * 0.04), dt=1e-4)
    with F.fr_mesh_load(meshes, opts) as ctx:
        x = F.fr_sp_coords(ctx)
        u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(x, seed=5, periods=[2 * math.pi] * 3), 0, 1))
        F.fr_state_set(ctx, u)
        first, n = F.fr_cand_range(ctx, 1)
        v = 1.0 + 0.5 * u[first:first + n]
        hp = _pinned(v.shape)
        hp[...] = v
        F.fr_state_set(ctx, hp, cand=1)
        out = F.fr_state_get(ctx, cand=1, out=_pinned(v.shape))
        assert np.array_equal(out, v.astype(np.float32).astype(np.float64))
        other = F.fr_state_get(ctx, cand=0)
        f0, n0 = F.fr_cand_range(ctx, 0)
        assert np.array_equal(other, u[f0:f0 + n0].astype(np.float32).astype(np.float64))
