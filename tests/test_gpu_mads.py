"""The optimisation loop on the GPU path (Section 3.4, Appendix E): the
baseline design and one complete OrthoMADS poll, every poll point a candidate
of one batched context, scored by Eq. 8 from the mean forces and the FW-H
OASPL at the observer 10c below each trailing edge.  Coarse O-grids and one
convective time: a check of the machinery, not of the paper's optimum."""
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


def test_one_poll_of_the_naca_optimisation():
    from paper_2501_05709_gb300 import cases as C
    from paper_2501_05709_gb300 import mads as M
    polls = []
    r = C.optimize_naca(max_iter=1, log=polls.append)
    base = r["baseline"]
    assert base["oaspl_db"] is not None and math.isfinite(base["oaspl_db"])
    assert abs(base["cl_mean"]) < 2.0 and 0.0 < base["cd_mean"] < 1.0
    # NACA 0012 at 6 degrees: positive lift
    assert base["cl_mean"] > 0.1
    res = r["result"]
    assert res.iterations == 1 and len(polls) == 1
    h = res.history[0]
    assert h["points"] + h["infeasible"] == 8 and len(polls[0]) == h["points"]
    # every evaluated candidate scored by Eq. 8 against the baseline
    for c in polls[0]:
        assert np.all(c["design"] >= M.NACA_BOUNDS[:, 0] - 1e-9) and np.all(c["design"] <= M.NACA_BOUNDS[:, 1] + 1e-9)
    finite = [c for c in polls[0] if c.get("oaspl_db") is not None and math.isfinite(c["oaspl_db"])]
    assert len(finite) >= h["points"] // 2
    f_base = M.objective(base["oaspl_db"], base["cl_mean"], base["cd_mean"], base["cl_mean"], base["cd_mean"])
    assert res.f <= f_base
