"""OrthoMADS poll loop on the host and the shape-optimisation objective.

The objective is Eq. 8 (Section 3.4): the OASPL at the observer plus a
quadratic penalty on the mean-lift deviation from the baseline design, and a
second one on the mean drag where it exceeds the baseline's.  The optimiser
is the mesh adaptive direct search of Appendix E (OrthoMADS): design
variables scaled to [0, 1], mesh size Delta^m = 4^-l (never above 1), poll
size Delta^p = sqrt(Delta^m) for the maximal positive basis of 2n
directions, every poll point evaluated before the iteration ends (the
paper's choice), Delta^m divided by 4 after a failed iteration and
multiplied by 4 (up to 1) after a successful one.  Points outside the design
box are infeasible and discarded (never evaluated).

The poll directions follow the published OrthoMADS construction (cited by the
paper, not printed in it): the Halton point u_t of the mesh index, turned
into the integer direction q closest in length to (not longer than)
2^(l/2) along 2u_t - 1, and the Householder matrix H = |q|^2 I - 2 q q^T,
whose columns and their negatives form the poll set [H, -H].  H has
mutually orthogonal columns of length |q|^2, so a poll point lies
Delta^m |q|^2 ~ Delta^p from the incumbent.  No search step is run (the
step is optional in MADS and the paper gives no rule for it).

The batch evaluator receives every feasible poll point of one iteration at
once: with the FR library those become the candidates of one context,
advanced together (the batched poll of the GPU path).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PRIMES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)

# Section 3.4: penalty weights of Eq. 8
EPS_LIFT = 8000.0
EPS_DRAG = 400000.0

# Section 3.4: design variables and their ranges, X = [c_max (% chord),
# position of c_max (tenths of chord), t_max (% chord), angle of attack (deg)]
NACA_BOUNDS = np.array([[-10.0, 10.0], [4.0, 9.0], [6.0, 18.0], [0.0, 12.0]])


def objective(oaspl, cl_mean, cd_mean, cl_base, cd_base, eps_lift=EPS_LIFT, eps_drag=EPS_DRAG):
    """Eq. 8: OASPL + eps1 (C_L - C_L,base)^2, plus eps2 (C_D - C_D,base)^2
    when the mean drag exceeds the baseline's."""
    f = oaspl + eps_lift * (cl_mean - cl_base) ** 2
    if cd_mean > cd_base:
        f += eps_drag * (cd_mean - cd_base) ** 2
    return f


def radical_inverse(t, base):
    """Van der Corput radical inverse of the integer t >= 0 in `base`."""
    r, f = 0.0, 1.0 / base
    while t > 0:
        t, d = divmod(t, base)
        r += d * f
        f /= base
    return r


def halton(t, n):
    """The t-th Halton point in [0, 1)^n (bases: the first n primes)."""
    if n > len(PRIMES):
        raise ValueError(f"at most {len(PRIMES)} design variables")
    return np.array([radical_inverse(t, PRIMES[i]) for i in range(n)])


def adjusted_direction(t, l, n):
    """Integer vector q along 2 u_t - 1 (u_t the Halton point) with the
    largest scale a such that q = round(a v), v the unit direction, has
    |q| <= 2^(l/2); never zero (falls back to the axis of the largest |v_i|)."""
    v = 2.0 * halton(t, n) - 1.0
    nv = np.linalg.norm(v)
    v = v / nv if nv > 0 else np.eye(n)[0]
    target = 2.0 ** (0.5 * l)
    best = None
    for a in np.linspace(target * math.sqrt(n) + 1.0, 0.0, 4001):
        q = np.rint(a * v)
        if np.linalg.norm(q) <= target + 1e-12 and np.any(q != 0):
            best = q
            break
    if best is None:
        best = np.zeros(n)
        i = int(np.argmax(np.abs(v)))
        best[i] = 1.0 if v[i] >= 0 else -1.0
    return best.astype(np.int64)


def householder(q):
    """H = |q|^2 I - 2 q q^T (integer, mutually orthogonal columns of length |q|^2)."""
    q = np.asarray(q, np.int64)
    return int(q @ q) * np.eye(len(q), dtype=np.int64) - 2 * np.outer(q, q)


def poll_directions(l, n, t0=None):
    """The maximal positive basis [H, -H] (n x 2n, integer) of mesh index l;
    Halton index t = t0 + l, t0 the n-th prime by default."""
    t0 = PRIMES[n - 1] if t0 is None else t0
    H = householder(adjusted_direction(t0 + l, l, n))
    return np.concatenate([H, -H], axis=1)


def next_mesh_index(l, success):
    """Delta^m = 4^-l: divided by 4 after a failure, multiplied by 4 (never
    above 1) after a success."""
    return max(l - 1, 0) if success else l + 1


@dataclass
class MadsResult:
    x: np.ndarray                 # scaled incumbent in [0, 1]^n
    f: float
    iterations: int
    evaluations: int
    history: list = field(default_factory=list)   # per iteration: dict


def orthomads(evaluate, x0, l0=2, max_iter=20, min_poll=1e-3, max_evals=None):
    """Minimise over [0, 1]^n.  `evaluate(points)` takes an array [m, n] of
    scaled points and returns m objective values (one call per iteration:
    the whole poll).  Stops after max_iter iterations, when the poll size
    2^-l drops below min_poll, or when max_evals would be exceeded."""
    x = np.asarray(x0, float).copy()
    n = x.size
    if np.any(x < 0.0) or np.any(x > 1.0):
        raise ValueError("the initial point must lie in [0, 1]^n")
    fx = float(np.asarray(evaluate(x[None, :]), float)[0])
    evals, l = 1, int(l0)
    hist = []
    for it in range(1, max_iter + 1):
        if 2.0 ** (-l) < min_poll:
            break
        D = poll_directions(l, n)
        dm = 4.0 ** (-l)
        pts = x[None, :] + dm * D.T.astype(float)
        feas = np.all((pts >= 0.0) & (pts <= 1.0), axis=1)
        cand = pts[feas]
        if max_evals is not None and evals + len(cand) > max_evals:
            break
        fv = np.asarray(evaluate(cand), float) if len(cand) else np.zeros(0)
        evals += len(cand)
        success = False
        if len(cand) and np.min(fv) < fx:
            j = int(np.argmin(fv))
            x, fx, success = cand[j].copy(), float(fv[j]), True
        hist.append({"iteration": it, "mesh_index": l, "mesh_size": dm, "poll_size": 2.0 ** (-l),
                     "points": len(cand), "infeasible": int((~feas).sum()), "success": success, "f": fx,
                     "x": x.copy()})
        l = next_mesh_index(l, success)
    return MadsResult(x=x, f=fx, iterations=len(hist), evaluations=evals, history=hist)


def to_design(x, bounds=NACA_BOUNDS):
    """Scaled point in [0, 1]^n -> physical design variables."""
    b = np.asarray(bounds, float)
    return b[:, 0] + np.asarray(x, float) * (b[:, 1] - b[:, 0])


def to_scaled(X, bounds=NACA_BOUNDS):
    b = np.asarray(bounds, float)
    return (np.asarray(X, float) - b[:, 0]) / (b[:, 1] - b[:, 0])
