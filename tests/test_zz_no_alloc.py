"""fwh_integrate_noalloc against fwh_integrate, through the C-ABI.

The no-allocation variant exists for callers whose device memory is owned by
their own pool allocator (or who cannot afford cudaFree's device-wide
synchronisation): it keeps its scratch in a fixed 32 MiB device array instead
of calling cudaMalloc.  Two calls in a row with different inputs must each
match the allocating entry point within the FP64 parity tolerance (1e-12
relative L2), so contents left in the shared array by one call cannot leak
into the next.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run(fn, hist, y, n, dS, dt, obs, M, c0, rho0, p0, Lspan, ncopies, cap):
    from paper_2501_05709_gb300 import fr as F
    nobs = obs.shape[0]
    p_out = torch.full((nobs, cap), float("nan"), dtype=torch.float64, device="cuda")
    nt_out = np.zeros(nobs, dtype=np.int32)
    t0_out = np.zeros(nobs)
    Mh = np.ascontiguousarray(M, dtype=np.float64)
    rc = fn(C.c_void_p(hist.data_ptr()), hist.shape[0], hist.shape[1], C.c_void_p(y.data_ptr()),
            C.c_void_p(n.data_ptr()), C.c_void_p(dS.data_ptr()), dt, 0.0, C.c_void_p(obs.ctypes.data), nobs,
            C.c_void_p(Mh.ctypes.data), c0, rho0, p0, Lspan, ncopies, C.c_void_p(p_out.data_ptr()), cap,
            C.c_void_p(nt_out.ctypes.data), C.c_void_p(t0_out.ctypes.data), None)
    assert rc == 0, F.lib().fr_last_error().decode()
    return p_out.cpu().numpy(), nt_out, t0_out


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    B.build()
    L = F.lib()
    y0, n0, dS0 = W.sphere_surface(1.0, 12, 2 * np.pi / 18)
    cases = [
        # (Mach vector, observers, span copies, source field)
        ([0.5, 0.1, 0.5], np.array([[20.0, 0.0, 0.0], [0.0, -15.0, 3.0]]), (0.0, 1), W.monopole_field),
        ([0.3, 0.0, 0.2], np.array([[0.0, 30.0, 1.0]]), (0.7, 5), W.dipole_field),
    ]
    dt = 0.004
    tau = dt * np.arange(160)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    for M, obs, (Lspan, nc), field in cases:
        fld = field(y0[None], tau[:, None], M)
        hist = np.concatenate([fld["rho"][..., None], fld["vel"], fld["p"][..., None]], axis=-1)
        args = (dev(hist), dev(y0), dev(n0), dev(dS0), dt, obs, M, 340.75, 1.234, fld["p0"], Lspan, nc, 400)
        ref, nt_ref, t0_ref = _run(L.fwh_integrate, *args)
        out, nt_out, t0_out = _run(L.fwh_integrate_noalloc, *args)
        assert np.array_equal(nt_out, nt_ref) and np.allclose(t0_out, t0_ref, rtol=0, atol=1e-15)
        for o in range(len(obs)):
            a, b = out[o, :nt_out[o]], ref[o, :nt_ref[o]]
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    from paper_2501_05709_gb300 import fr as F
    B.build()
    L = F.lib()
    nt, npts = 1000, 600  # 8 * 600 * 1000 = 4.8M doubles > 2^22
    hist = torch.zeros((nt, npts, 5), dtype=torch.float64, device="cuda")
    hist[..., 0] = 1.2
    hist[..., 4] = 1e5
    y = torch.zeros((npts, 3), dtype=torch.float64, device="cuda")
    y[:, 0] = torch.linspace(0, 1, npts, dtype=torch.float64)
    nrm = torch.zeros((npts, 3), dtype=torch.float64, device="cuda")
    nrm[:, 2] = 1.0
    dS = torch.ones(npts, dtype=torch.float64, device="cuda")
    obs = np.array([[0.0, 50.0, 0.0]])
    with pytest.raises(AssertionError) as ei:
        _run(L.fwh_integrate_noalloc, hist, y, nrm, dS, 1e-3, obs, [0.0, 0.0, 0.0], 340.0, 1.2, 1e5, 0.0, 1, nt)
    assert "fixed maximum" in str(ei.value)
