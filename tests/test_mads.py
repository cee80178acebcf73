"""Host logic of the optimisation loop (Section 3.4, Appendix E): the Eq. 8
objective, the OrthoMADS poll directions and mesh rules, and the loop on
closed-form functions (no GPU)."""
import math

import numpy as np
import pytest

from paper_2501_05709_gb300 import mads as M


def test_objective_branches():
    # drag at or below the baseline: only the lift penalty (Eq. 8, second case)
    assert M.objective(80.0, 0.5, 0.03, 0.6, 0.04) == pytest.approx(80.0 + 8000.0 * 0.01)
    assert M.objective(80.0, 0.6, 0.04, 0.6, 0.04) == 80.0
    # drag above the baseline: both penalties (first case)
    assert M.objective(80.0, 0.6, 0.05, 0.6, 0.04) == pytest.approx(80.0 + 400000.0 * 1e-4)
    # continuous where the cases meet
    a = M.objective(80.0, 0.55, 0.04 + 1e-12, 0.6, 0.04)
    b = M.objective(80.0, 0.55, 0.04, 0.6, 0.04)
    assert abs(a - b) < 1e-9


def test_halton_points():
    # radical inverses in bases 2 and 3 (textbook values)
    assert [M.radical_inverse(t, 2) for t in range(1, 8)] == [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875]
    assert M.radical_inverse(1, 3) == pytest.approx(1 / 3)
    assert M.radical_inverse(5, 3) == pytest.approx(2 / 3 + 1 / 9)
    u = M.halton(7, 4)
    assert u.shape == (4,) and np.all((u >= 0) & (u < 1))


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 6, 8])
def test_poll_set_is_orthogonal_maximal_positive_basis(l):
    n = 4
    D = M.poll_directions(l, n)
    assert D.shape == (n, 2 * n) and D.dtype.kind == "i"
    H = D[:, :n]
    q2 = H[0] @ H[0]
    # mutually orthogonal columns of equal length |q|^2
    assert np.array_equal(H.T @ H, q2 * np.eye(n, dtype=np.int64))
    q = M.adjusted_direction(M.PRIMES[n - 1] + l, l, n)
    assert int(q @ q) ** 2 == q2
    assert np.linalg.norm(q) <= 2 ** (l / 2) + 1e-12
    # [H, -H] positively spans R^n: every direction has a poll direction at
    # an acute angle
    rng = np.random.default_rng(l)
    for w in rng.normal(size=(200, n)):
        assert np.max(w @ D) > 0
    # the poll step length Delta^m |q|^2 stays within a factor 4 of the poll size 2^-l
    step = 4.0 ** -l * math.sqrt(q2)
    assert 2.0 ** -l / 4 <= step <= 2.0 ** -l + 1e-12


def test_mesh_size_rules():
    # Delta^m = 4^-l: a success multiplies it by 4 up to 1, a failure divides by 4
    assert M.next_mesh_index(3, True) == 2
    assert M.next_mesh_index(0, True) == 0
    assert M.next_mesh_index(2, False) == 3
    l = 2
    for s in (True, True, True, False, False, True):
        l = M.next_mesh_index(l, s)
        assert 4.0 ** -l <= 1.0


def test_scaling_round_trip():
    X = np.array([0.0, 4.0, 12.0, 6.0])
    x = M.to_scaled(X)
    assert np.allclose(x, [0.5, 0.0, 0.5, 0.5])
    assert np.allclose(M.to_design(x), X)


def test_complete_poll_in_one_batch_and_feasibility():
    calls = []

    def f(points):
        points = np.asarray(points)
        calls.append(points.copy())
        assert np.all((points >= 0) & (points <= 1))        # infeasible points are never evaluated
        return np.sum((points - 0.3) ** 2, axis=1)

    r = M.orthomads(f, np.array([0.0, 0.0, 1.0, 0.5]), l0=1, max_iter=4)
    assert len(calls) == 1 + r.iterations                     # one call per iteration: the whole poll
    for c, h in zip(calls[1:], r.history):
        assert len(c) == h["points"] and h["points"] + h["infeasible"] == 8
    assert r.evaluations == sum(len(c) for c in calls)


def test_converges_on_a_quadratic_and_keeps_the_mesh():
    target = np.array([0.3, 0.7, 0.45, 0.2])
    f = lambda P: np.sum((np.asarray(P) - target) ** 2, axis=1)
    x0 = np.array([0.9, 0.1, 0.5, 0.8])
    r = M.orthomads(f, x0, l0=1, max_iter=200, min_poll=1e-4)
    assert r.f < 1e-5 and np.linalg.norm(r.x - target) < 5e-3
    # the incumbent only improves, and the mesh index follows the rules
    fs = [h["f"] for h in r.history]
    assert all(b <= a for a, b in zip(fs, fs[1:]))
    for a, b in zip(r.history, r.history[1:]):
        assert b["mesh_index"] == M.next_mesh_index(a["mesh_index"], a["success"])


def test_piecewise_objective_drives_the_search():
    # a toy landscape with the Eq. 8 shape: an "OASPL" falling with x0, a lift
    # that must stay at its baseline, a drag that must not rise above it
    def evaluate(P):
        out = []
        for x in np.asarray(P):
            oaspl = 90.0 - 5.0 * x[0]
            cl = 0.6 + 0.2 * (x[1] - 0.5)
            cd = 0.04 + 0.02 * max(x[0] - 0.6, 0.0)
            out.append(M.objective(oaspl, cl, cd, 0.6, 0.04))
        return out

    r = M.orthomads(evaluate, np.array([0.2, 0.5, 0.5, 0.5]), l0=1, max_iter=60, min_poll=1e-3)
    assert r.f < evaluate([[0.2, 0.5, 0.5, 0.5]])[0]
    # the optimum trades the OASPL gain against the drag penalty past x0 = 0.6
    # and keeps the lift near its baseline
    assert 0.6 < r.x[0] <= 1.0 and abs(r.x[1] - 0.5) < 0.05


def test_bad_start_is_rejected():
    with pytest.raises(ValueError):
        M.orthomads(lambda P: np.zeros(len(P)), np.array([1.2, 0.0, 0.0, 0.0]))
