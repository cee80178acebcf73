"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point that include/fr.h declares, and rejects bad input on the host
(no compute call: there is no GPU here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2501_05709_gb300 import build as B
from paper_2501_05709_gb300 import fr as F

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fr.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z0-9_]+\s*\*?\s*((?:fr|fwh)_[a-z0-9_]+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fr_mesh_load", "fr_residual", "fr_rk_step", "fr_forces", "fwh_sample", "fwh_integrate"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(declared_functions()) <= set(F._SIGS)


def test_build_targets_sm103a_only():
    assert B.ARCH == "-gencode=arch=compute_103a,code=sm_103a"


def _desc(nodes, conn):
    d = F.fr_mesh_desc()
    d.dim, d.nelem, d.geom_order = nodes.shape[2], nodes.shape[0], 1
    d.nodes = nodes.ctypes.data_as(C.POINTER(C.c_double))
    d.conn = conn.ctypes.data_as(C.POINTER(C.c_int32))
    return d


def test_mesh_load_rejects_bad_input_on_host(lib):
    from paper_2501_05709_gb300 import workloads as W
    nodes, conn = W.box_mesh(3, 2, 0.0, 1.0)
    conn = conn.astype(np.int32)
    out = C.c_void_p()
    d = _desc(nodes, conn)
    d.nelem = 0
    assert lib.fr_mesh_load(C.byref(d), 1, C.byref(F.options()), C.byref(out)) == F.FR_EINVAL
    assert out.value is None
    d = _desc(nodes, conn)
    assert lib.fr_mesh_load(C.byref(d), 1, C.byref(F.options(order=7)), C.byref(out)) == F.FR_EINVAL
    assert b"order" in lib.fr_last_error()
    assert lib.fr_mesh_load(C.byref(d), 1, C.byref(F.options(viscous=True, mu=0.0)), C.byref(out)) == F.FR_EINVAL
    assert lib.fr_mesh_load(None, 1, C.byref(F.options()), C.byref(out)) == F.FR_EINVAL


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2501_05709_gb300 import workloads as W
    nodes, conn = W.box_mesh(3, 2, 0.0, 1.0)
    with pytest.raises(F.FrError) as ei:
        F.fr_mesh_load((nodes, conn), F.options())
    assert ei.value.code == F.FR_ECUDA


def test_fwh_integrate_rejects_bad_sizes_on_host(lib):
    z = np.zeros(16)
    M = np.zeros(3)
    nt_out = np.zeros(1, np.int32)
    t0 = np.zeros(1)
    p = C.c_void_p(z.ctypes.data)
    rc = lib.fwh_integrate(p, 3, 1, p, p, p, 0.1, 0.0, p, 1, C.c_void_p(M.ctypes.data), 340.0, 1.2, 1e5, 0.0,
                           1, p, 4, C.c_void_p(nt_out.ctypes.data), C.c_void_p(t0.ctypes.data), None)
    assert rc == F.FR_EINVAL
    rc = lib.fwh_integrate(p, 8, 1, p, p, p, 0.1, 0.0, p, 1, C.c_void_p(M.ctypes.data), 340.0, 1.2, 1e5, 0.0,
                           2, p, 4, C.c_void_p(nt_out.ctypes.data), C.c_void_p(t0.ctypes.data), None)
    assert rc == F.FR_EINVAL
    M2 = np.array([0.8, 0.7, 0.0])
    rc = lib.fwh_integrate(p, 8, 1, p, p, p, 0.1, 0.0, p, 1, C.c_void_p(M2.ctypes.data), 340.0, 1.2, 1e5, 0.0,
                           1, p, 4, C.c_void_p(nt_out.ctypes.data), C.c_void_p(t0.ctypes.data), None)
    assert rc == F.FR_EINVAL


def test_new_entry_points_reject_bad_input_on_host(lib):
    # argument checks that run before any device work
    z = np.zeros(64)
    p = C.c_void_p(z.ctypes.data)
    nf = C.c_int()
    assert lib.fwh_psd(None, 1, 16, 16, 0.1, 3, p, 16, C.byref(nf), None) == F.FR_EINVAL
    assert lib.fwh_psd(p, 1, 3, 3, 0.1, 3, p, 16, C.byref(nf), None) == F.FR_EINVAL      # record too short
    assert lib.fwh_psd(p, 1, 16, 8, 0.1, 3, p, 16, C.byref(nf), None) == F.FR_EINVAL     # ld < nt
    assert lib.fwh_psd(p, 1, 16, 16, 0.0, 3, p, 16, C.byref(nf), None) == F.FR_EINVAL    # dt <= 0
    assert lib.fwh_psd(p, 1, 16, 16, 0.1, 3, p, 2, C.byref(nf), None) == F.FR_EINVAL     # cap < L/2 + 1
    t = C.c_double()
    assert lib.fr_set_source(None, 0, 0, None, 0.0) == F.FR_EINVAL
    assert lib.fr_source_time(None, 0, C.byref(t)) == F.FR_EINVAL
    assert lib.fr_set_adaptive_dt(None, 0.5) == F.FR_EINVAL
    assert lib.fr_cand_dt(None, 0, C.byref(t)) == F.FR_EINVAL
    assert lib.fr_set_element_order(None, -1, None) == F.FR_EINVAL
    flag = C.c_int()
    assert lib.fr_nonfinite(None, -1, C.byref(flag)) == F.FR_EINVAL
    assert lib.fr_set_rk_scheme(None, 0, None) == F.FR_EINVAL


def test_tensor_core_modes_are_validated_on_host(lib):
    # the tensor-core precision modes exist in 3D at p = 3 and 4 only; other
    # requests fail before any device work
    from paper_2501_05709_gb300 import workloads as W
    out = C.c_void_p()
    nodes, conn = W.box_mesh(2, 2, 0.0, 1.0)
    d = _desc(nodes, conn.astype(np.int32))
    assert lib.fr_mesh_load(C.byref(d), 1, C.byref(F.options(order=3, precision=F.FR_TF32_TC)),
                            C.byref(out)) == F.FR_EINVAL
    nodes, conn = W.box_mesh(3, 2, 0.0, 1.0)
    d = _desc(nodes, conn.astype(np.int32))
    assert lib.fr_mesh_load(C.byref(d), 1, C.byref(F.options(order=2, precision=F.FR_BF16X3_TC)),
                            C.byref(out)) == F.FR_EINVAL
    assert b"tensor-core" in lib.fr_last_error()
    assert lib.fr_mesh_load(C.byref(d), 1, C.byref(F.options(order=3, precision=7)), C.byref(out)) == F.FR_EINVAL


def _function_body(src, name):
    """Source text of the first definition of function `name` (brace matched)."""
    import re
    m = re.search(r"\b%s\s*\([^;{]*\)\s*\{" % re.escape(name), src)
    assert m, name
    i, depth = m.end() - 1, 0
    for j in range(i, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[i:j + 1]
    raise AssertionError(name)


def test_noalloc_fwh_path_names_no_device_allocation():
    # fwh_integrate_noalloc and every helper it calls use no allocating
    # runtime routine; fwh_integrate, which shares the helpers, does
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2501_05709_gb300", "csrc", "fwh.cu")).read()
    body = _function_body(src, "fwh_integrate_noalloc")
    called = {"fwh_plan", "fwh_run", "noalloc_scratch", "fwh_series_doubles", "fwh_partial_doubles"}
    assert called <= set(re.findall(r"\b(\w+)\s*\(", body))
    alloc = re.compile(r"\b(cudaMalloc\w*|cudaFree\w*|cudaMallocAsync|cudaFreeAsync|cuMem\w*Alloc\w*|malloc|new)\b")
    for name in ["fwh_integrate_noalloc"] + sorted(called):
        assert not alloc.search(_function_body(src, name)), name
    assert re.search(r"\bcudaMalloc\b", _function_body(src, "fwh_integrate"))
