"""Byte accounting behind the roofline figures of bench.py (per element and
RK stage, p = 3, FP32 unless stated) and the far-field sponge degrees of the
O-grid workload (host only)."""
import sys

import numpy as np
import pytest


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = argv[:1]
    try:
        import bench as B
    finally:
        sys.argv = argv
    return B


def test_algorithmic_bytes_per_element(bench):
    a = bench.algorithmic_bytes(1, 3, 4, viscous=True, curved=False)
    assert a["visc"] == 5256 and a["resid"] == 11336
    c = bench.algorithmic_bytes(1, 3, 4, viscous=True, curved=True)
    assert c["visc"] == 8856 and c["resid"] == 14936
    d = bench.algorithmic_bytes(1, 3, 8, viscous=True, curved=False)
    assert d["visc"] == 10488 and d["resid"] == 22648
    # Euler: no viscous-flux array, no viscous kernel
    e = bench.algorithmic_bytes(1, 3, 4, viscous=False, curved=False)
    assert e["visc"] == 0 and e["resid"] == 9416
    # linear in the element count
    assert bench.algorithmic_bytes(7, 3, 4)["resid"] == 7 * bench.algorithmic_bytes(1, 3, 4)["resid"]


def test_sponge_degrees_of_the_ogrid():
    from paper_2501_05709_gb300 import workloads as W
    nodes, _ = W.ogrid_mesh(40, 20, 1, 0.2, r_outer=10.0, first_cell=2e-2)
    q = W.sponge_orders(nodes, 3)
    X = np.asarray(nodes)
    r = np.hypot(X[:, :, 0].mean(axis=1) - 0.5, X[:, :, 1].mean(axis=1))
    assert q.dtype == np.int32 and q.min() >= 0 and q.max() == 3
    assert np.all(q[r < 4.0] == 3) and np.all(q[r >= 8.0] == 0)
    assert np.all(q[(r >= 6.0) & (r < 8.0)] == 1)
    # never rises with the distance from the body
    order = np.argsort(r)
    assert np.all(np.diff(q[order]) <= 0)


def test_reduced_bytes_per_element(bench):
    # a reduced element moves a degree-p element's arrays (state, traces,
    # viscous fluxes, RK arrays at the degree-p points) with the metric terms
    # (S and 1/|J|, 10 values per point in 3D) at its (q+1)^3 points, in each
    # of its two kernels
    full = bench.algorithmic_bytes(1, 3, 4, viscous=True, curved=True)
    for q in range(3):
        r = bench.reduced_bytes([q], 3, 4, viscous=True, curved=True)
        assert r == full["visc"] + full["resid"] - 2 * 10 * (64 - (q + 1) ** 3) * 4
    # Euler on an affine mesh: no face kernel, no viscous-flux array; a
    # degree-p element holds one metric set, a reduced one a set per q point
    e = bench.algorithmic_bytes(1, 3, 4, viscous=False, curved=False)
    assert bench.reduced_bytes([1], 3, 4, viscous=False) == e["resid"] + 10 * (8 - 1) * 4
    # degree-p elements are not counted; additive over elements
    assert bench.reduced_bytes([3, 3], 3, 4) == 0
    assert bench.reduced_bytes([0, 1, 1, 3], 3, 4) == (bench.reduced_bytes([0], 3, 4)
                                                       + 2 * bench.reduced_bytes([1], 3, 4))
