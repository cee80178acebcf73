"""What rounding the metric terms to float costs, measured in the FP64 oracle.

The FP32 mode stores S = |J| dxi/dx, |J| and the face normals in float
(computed in double, rounded once).  Evaluating the FP64 residual with only
those metric arrays rounded to float changes it by at most ~3.4e-7 (relative
L2) on the curved meshes of the parity cases, several times less than rounding
the state itself to float (1e-6 .. 3e-6), which every FP32 mode must do; so
keeping the metrics in double would not make the FP32 path noticeably more
accurate (it would move ~33% more bytes per curved DOF and put the metric
contractions on the FP64 pipe)."""
import copy

import numpy as np
import pytest

from oracle.fr import FRSolver

from ._cases import make_case, oracle_for


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("name", ["ns3d_curved_p3", "ns3d_ogrid_p3", "turned3d_curved_p3", "ns3d_p4_g2",
                                  "ns2d_curved_p3_g2"])
def test_float_metrics_cost_less_than_a_float_state(name):
    c = make_case(name)
    m, s = oracle_for(c)
    u = c["state"](m.xsp)
    R = s.residual(u)
    mf = copy.copy(m)
    for k in ("S", "J", "N"):
        setattr(mf, k, getattr(m, k).astype(np.float32).astype(np.float64))
    e_metric = _rel(FRSolver(mf, s.ph).residual(u), R)
    e_state = _rel(s.residual(u.astype(np.float32).astype(np.float64)), R)
    assert e_metric <= 1e-6
    assert e_metric <= e_state / 3.0
