"""Thin ctypes binding of libfr (``include/fr.h``): the same call names, argument
marshalling only.  Every compute step runs in the CUDA library; there is no
Python or CPU fallback, and loading fails loudly when the library is missing.

Device buffers are passed as torch CUDA tensors (or raw integer device
pointers); host buffers as numpy arrays.  ``stream`` is an integer CUDA stream
handle (0 = legacy default stream), e.g. ``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfr.so")

FR_OK = 0
FR_EINVAL = -1
FR_ENOMEM = -2
FR_ECUDA = -3
FR_ENONFINITE = -4
FR_ETIMEOUT = -5
FR_EWINDOW = -6
FR_EMESH = -7
FR_FP64 = 0
FR_FP32 = 1
FR_TF32_TC = 2
FR_BF16X3_TC = 3
FR_CORR_DG = 0
FR_CORR_HUYNH_G2 = 1
FR_BC_WALL = 1
FR_BC_FARFIELD = 2

_NAMES = {0: "FR_OK", -1: "FR_EINVAL", -2: "FR_ENOMEM", -3: "FR_ECUDA", -4: "FR_ENONFINITE",
          -5: "FR_ETIMEOUT", -6: "FR_EWINDOW", -7: "FR_EMESH"}


class FrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class fr_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelem", C.c_int), ("geom_order", C.c_int),
                ("nodes", C.POINTER(C.c_double)), ("conn", C.POINTER(C.c_int32))]


class fr_options(C.Structure):
    _fields_ = [("order", C.c_int), ("correction", C.c_int), ("precision", C.c_int), ("viscous", C.c_int),
                ("gamma", C.c_double), ("prandtl", C.c_double), ("mu", C.c_double), ("br2_eta", C.c_double),
                ("rho_inf", C.c_double), ("p_inf", C.c_double), ("vel_inf", C.c_double * 3),
                ("dt", C.c_double), ("lift_dir", C.c_double * 3), ("drag_dir", C.c_double * 3),
                ("ref_area", C.c_double)]


_lib = None

_SIGS = {
    "fr_ctx_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "fr_mesh_load": (C.c_int, [C.POINTER(fr_mesh_desc), C.c_int, C.POINTER(fr_options), C.POINTER(C.c_void_p)]),
    "fr_destroy": (C.c_int, [C.c_void_p]),
    "fr_last_error": (C.c_char_p, []),
    "fr_sp_coords": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fr_cand_range": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "fr_state_set": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "fr_state_get": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "fr_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_rk_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fr_rk_step_graph": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fr_set_cand_dt": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "fr_forces": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fr_forces_reset": (C.c_int, [C.c_void_p]),
    "fr_nonfinite": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "fr_set_rk_scheme": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fr_integrals": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fwh_register": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "fwh_sample": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fwh_history": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]),
    "fwh_clear": (C.c_int, [C.c_void_p, C.c_int]),
    "fwh_integrate": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                C.c_double, C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fwh_integrate_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_double, C.c_double, C.c_void_p, C.c_int, C.c_void_p, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_int,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "fwh_psd": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_int,
                          C.POINTER(C.c_int), C.c_void_p]),
    "fr_set_source": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_double]),
    "fr_source_time": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "fr_set_adaptive_dt": (C.c_int, [C.c_void_p, C.c_double]),
    "fr_cand_dt": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "fr_set_element_order": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fr_set_tile": (C.c_int, [C.c_void_p, C.c_int]),
    "fr_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "fr_launch_count": (C.c_int64, [C.c_void_p]),
    "fr_profile_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_probe_fp64_peak": (C.c_int, [C.POINTER(C.c_double), C.c_void_p]),
}


def lib():
    """The loaded libfr (raises if the library has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfr is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != FR_OK:
        raise FrError(rc, lib().fr_last_error().decode())


def _ptr(x):
    """Device pointer of a torch tensor, or an int pointer, or a numpy host pointer."""
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(s.cuda_stream)


def options(order=3, correction=FR_CORR_DG, precision=FR_FP64, viscous=False, gamma=1.4, prandtl=0.71,
            mu=0.0, br2_eta=1.0, rho_inf=1.0, p_inf=1.0, vel_inf=(0.0, 0.0, 0.0), dt=1e-3,
            lift_dir=(0.0, 1.0, 0.0), drag_dir=(1.0, 0.0, 0.0), ref_area=1.0):
    o = fr_options()
    o.order, o.correction, o.precision, o.viscous = order, correction, precision, int(bool(viscous))
    o.gamma, o.prandtl, o.mu, o.br2_eta = gamma, prandtl, mu, br2_eta
    o.rho_inf, o.p_inf, o.dt, o.ref_area = rho_inf, p_inf, dt, ref_area
    for i in range(3):
        o.vel_inf[i] = vel_inf[i] if i < len(vel_inf) else 0.0
        o.lift_dir[i] = lift_dir[i] if i < len(lift_dir) else 0.0
        o.drag_dir[i] = drag_dir[i] if i < len(drag_dir) else 0.0
    return o


class Context:
    """Owns an ``fr_ctx*``; ``close()`` (or ``fr_destroy``) releases it."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep
        d = (C.c_int64 * 8)()
        _check(lib().fr_ctx_dims(handle, d))
        self.dim, self.order, self.nvar, self.nsp, self.nelem, self.ncand, self.precision, self.affine = \
            [int(v) for v in d]
        self.np_dtype = np.float64 if self.precision == FR_FP64 else np.float32

    def close(self):
        if self.handle:
            lib().fr_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def state_shape(self):
        return (self.nelem, self.nvar, self.nsp)


def fr_mesh_load(meshes, opts):
    """meshes: (nodes, conn) or a list of them (one per candidate)."""
    if isinstance(meshes, tuple) and len(meshes) == 2 and isinstance(meshes[0], np.ndarray):
        meshes = [meshes]
    descs = (fr_mesh_desc * len(meshes))()
    keep = []
    for k, (nodes, conn) in enumerate(meshes):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        E, nn, dim = nodes.shape
        q = int(round(nn ** (1.0 / dim))) - 1
        descs[k].dim, descs[k].nelem, descs[k].geom_order = dim, E, q
        descs[k].nodes = nodes.ctypes.data_as(C.POINTER(C.c_double))
        descs[k].conn = conn.ctypes.data_as(C.POINTER(C.c_int32))
        keep += [nodes, conn]
    h = C.c_void_p()
    _check(lib().fr_mesh_load(descs, len(meshes), C.byref(opts), C.byref(h)))
    return Context(h, None)


def fr_destroy(ctx):
    ctx.close()


def fr_ctx_dims(ctx):
    d = (C.c_int64 * 8)()
    _check(lib().fr_ctx_dims(ctx.handle, d))
    return [int(v) for v in d]


def fr_cand_range(ctx, cand=-1):
    a, b = C.c_int64(), C.c_int64()
    _check(lib().fr_cand_range(ctx.handle, cand, C.byref(a), C.byref(b)))
    return a.value, b.value


def fr_sp_coords(ctx, cand=-1):
    _, n = fr_cand_range(ctx, cand)
    out = np.empty((n, ctx.nsp, ctx.dim))
    _check(lib().fr_sp_coords(ctx.handle, cand, _ptr(out)))
    return out


def fr_state_set(ctx, u, cand=-1, stream=None):
    """u: host numpy float64 or device torch float64 tensor, canonical layout."""
    on_dev = 0 if isinstance(u, np.ndarray) else 1
    if on_dev == 0:
        u = np.ascontiguousarray(u, dtype=np.float64)
    _check(lib().fr_state_set(ctx.handle, cand, _ptr(u), on_dev, _stream(stream)))


def fr_state_get(ctx, cand=-1, out=None, stream=None):
    _, n = fr_cand_range(ctx, cand)
    host = out is None or isinstance(out, np.ndarray)
    if out is None:
        out = np.empty((n, ctx.nvar, ctx.nsp))
    _check(lib().fr_state_get(ctx.handle, cand, _ptr(out), 0 if host else 1, _stream(stream)))
    return out


def fr_residual(ctx, u, R, stream=None):
    _check(lib().fr_residual(ctx.handle, _ptr(u), _ptr(R), _stream(stream)))


def fr_rk_step(ctx, nsteps, stream=None):
    _check(lib().fr_rk_step(ctx.handle, int(nsteps), _stream(stream)))


def fr_set_cand_dt(ctx, cand, dt):
    _check(lib().fr_set_cand_dt(ctx.handle, int(cand), float(dt)))


def fr_rk_step_graph(ctx, nsteps, stream=None):
    _check(lib().fr_rk_step_graph(ctx.handle, int(nsteps), _stream(stream)))


def fr_forces(ctx, cand=0):
    out = np.zeros(5)
    _check(lib().fr_forces(ctx.handle, cand, _ptr(out)))
    return out


def fr_forces_reset(ctx):
    _check(lib().fr_forces_reset(ctx.handle))


def fr_nonfinite(ctx, cand=-1):
    """True when a step left NaN or Inf in candidate cand (-1: any)."""
    f = C.c_int(0)
    _check(lib().fr_nonfinite(ctx.handle, cand, C.byref(f)))
    return bool(f.value)


def fr_set_rk_scheme(ctx, coef=None):
    """Explicit scheme in coefficient form, coef [nstages][6] = (a, b, c, d, e,
    f) per stage (see include/fr.h); None returns to the built-in RK4."""
    if coef is None:
        _check(lib().fr_set_rk_scheme(ctx.handle, 0, None))
        return
    k = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1, 6)
    _check(lib().fr_set_rk_scheme(ctx.handle, len(k), _ptr(k)))


def fr_integrals(ctx, cand=-1):
    out = np.zeros(ctx.nvar + 1)
    _check(lib().fr_integrals(ctx.handle, cand, _ptr(out)))
    return out


def fwh_register(ctx, cand, xyz, capacity, every=1):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    h = C.c_int()
    _check(lib().fwh_register(ctx.handle, cand, xyz.shape[0], _ptr(xyz), int(capacity), int(every), C.byref(h)))
    return h.value


def fwh_sample(ctx, handle, stream=None):
    _check(lib().fwh_sample(ctx.handle, handle, _stream(stream)))


def fwh_history(ctx, handle, npts):
    n = C.c_int()
    _check(lib().fwh_history(ctx.handle, handle, None, C.byref(n)))
    out = np.empty((n.value, npts, 5))
    _check(lib().fwh_history(ctx.handle, handle, _ptr(out), C.byref(n)))
    return out


def fwh_clear(ctx, handle):
    _check(lib().fwh_clear(ctx.handle, handle))


def fwh_integrate(hist, y, n, dS, dtau, tau0, obs, Minf, c0, rho0, p0, Lspan=0.0, ncopies=1, p_out=None,
                  cap=None, stream=None):
    """hist, y, n, dS: device float64 tensors; obs: host [nobs, 3].  Returns
    (p_out device tensor [nobs, cap], nt_out [nobs], t0_out [nobs])."""
    obs = np.ascontiguousarray(np.atleast_2d(obs), dtype=np.float64)
    nobs = obs.shape[0]
    nt, npts = int(hist.shape[0]), int(hist.shape[1])
    if cap is None:
        cap = nt
    if p_out is None:
        import torch
        p_out = torch.zeros((nobs, cap), dtype=torch.float64, device=hist.device)
    M = np.ascontiguousarray(Minf, dtype=np.float64)
    nt_out = np.zeros(nobs, dtype=np.int32)
    t0_out = np.zeros(nobs)
    _check(lib().fwh_integrate(_ptr(hist), nt, npts, _ptr(y), _ptr(n), _ptr(dS), float(dtau), float(tau0),
                               _ptr(obs), nobs, _ptr(M), float(c0), float(rho0), float(p0), float(Lspan),
                               int(ncopies), _ptr(p_out), int(cap), _ptr(nt_out), _ptr(t0_out), _stream(stream)))
    return p_out, nt_out, t0_out


def fwh_psd(p, dt, nseg=3, nt=None, psd=None, stream=None):
    """Welch PSD (nseg Hann windows, 50% overlap) of device float64 series
    p [nobs, ld] (first nt entries of each row).  Returns (psd device tensor
    [nobs, nfreq], frequencies as a numpy array)."""
    nobs, ld = int(p.shape[0]), int(p.shape[1])
    nt = ld if nt is None else int(nt)
    cap = 2 * (nt // (nseg + 1)) // 2 + 1
    if psd is None:
        import torch
        psd = torch.zeros((nobs, max(cap, 1)), dtype=torch.float64, device=p.device)
    nf = C.c_int()
    _check(lib().fwh_psd(_ptr(p), nobs, nt, ld, float(dt), int(nseg), _ptr(psd), int(psd.shape[1]), C.byref(nf),
                         _stream(stream)))
    L = 2 * (nf.value - 1)
    return psd[:, :nf.value], np.arange(nf.value) / (L * dt)


def fr_set_source(ctx, cand, sources, t0=0.0):
    """Energy sources of Eq. D.1 for candidate cand: sources = [(A, k, (x, y, z), f), ...]
    (at most 4); the candidate's time becomes t0."""
    arr = np.ascontiguousarray([[A, k, *list(xs)[:3], *([0.0] * (3 - len(xs))), f] for A, k, xs, f in sources],
                               dtype=np.float64).reshape(-1, 6)
    _check(lib().fr_set_source(ctx.handle, int(cand), int(arr.shape[0]), _ptr(arr) if arr.size else None,
                               float(t0)))


def fr_source_time(ctx, cand=0):
    t = C.c_double()
    _check(lib().fr_source_time(ctx.handle, int(cand), C.byref(t)))
    return t.value


def fr_set_adaptive_dt(ctx, cfl):
    """Adaptive RK4 step, dt = cfl / max spectral rate per candidate (cfl <= 0: fixed steps)."""
    _check(lib().fr_set_adaptive_dt(ctx.handle, float(cfl)))


def fr_cand_dt(ctx, cand=0):
    t = C.c_double()
    _check(lib().fr_cand_dt(ctx.handle, int(cand), C.byref(t)))
    return t.value


def fr_set_element_order(ctx, order, cand=-1):
    """Per-element polynomial degree (0..p) of candidate cand (cand = -1: the whole
    batch); None gives every element of it the context's p again."""
    if order is None:
        _check(lib().fr_set_element_order(ctx.handle, int(cand), None))
        return
    arr = np.ascontiguousarray(order, dtype=np.int32)
    _, n = fr_cand_range(ctx, cand)
    if arr.shape != (n,):
        raise ValueError(f"order needs {n} entries")
    _check(lib().fr_set_element_order(ctx.handle, int(cand), _ptr(arr)))


def fr_set_tile(ctx, epb):
    _check(lib().fr_set_tile(ctx.handle, int(epb)))


def fr_autotune(ctx):
    b = C.c_int()
    _check(lib().fr_autotune(ctx.handle, C.byref(b)))
    return b.value


def fr_launch_count(ctx):
    return int(lib().fr_launch_count(ctx.handle))


def fr_probe_fp64_peak(stream=None):
    """Measured FP64 FMA throughput of the current GPU, GFLOP/s."""
    g = C.c_double()
    _check(lib().fr_probe_fp64_peak(C.byref(g), _stream(stream)))
    return g.value


def fr_profile_step(ctx, nsteps, stream=None):
    """(ms [6], launches [6]) per kernel kind: traces, viscous faces, residual+RK, forces/sampling,
    energy source, reduced-degree elements (their face and residual kernels)."""
    ms = np.zeros(6)
    n = np.zeros(6, dtype=np.int64)
    _check(lib().fr_profile_step(ctx.handle, int(nsteps), _stream(stream), _ptr(ms), _ptr(n)))
    return ms, n
