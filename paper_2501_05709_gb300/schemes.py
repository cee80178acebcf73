"""Coefficient tables of explicit Runge-Kutta schemes for ``fr_set_rk_scheme``.

Each scheme is a list of stages (a, b, c, d, e, f) of the coefficient form
declared in include/fr.h: with k = R(v) at stage i,
    acc <- e acc + f dt k        (acc = f dt k at the first stage)
    v   <- a u0 + b v + c dt k + d acc
starting from v = u0, the last v being the new state.  The tables restate
published schemes in that form; Section 3.1's own optimal scheme takes its
coefficients from the work it cites and can be entered the same way.
"""
from __future__ import annotations

# classic four-stage RK4: u1 = u0 + dt/6 (k1 + 2 k2 + 2 k3 + k4), stage inputs
# u0, u0 + dt/2 k1, u0 + dt/2 k2, u0 + dt k3 (acc carries dt/6 k1 + dt/3 k2 + dt/3 k3)
RK4 = [(1.0, 0.0, 0.5, 0.0, 0.0, 1.0 / 6.0),
       (1.0, 0.0, 0.5, 0.0, 1.0, 1.0 / 3.0),
       (1.0, 0.0, 1.0, 0.0, 1.0, 1.0 / 3.0),
       (1.0, 0.0, 1.0 / 6.0, 1.0, 1.0, 0.0)]

# forward Euler
EULER = [(1.0, 0.0, 1.0, 0.0, 0.0, 0.0)]

# Heun's second-order method: u1 = u0 + dt/2 (k1 + k2), k2 at u0 + dt k1
HEUN2 = [(1.0, 0.0, 1.0, 0.0, 0.0, 0.5),
         (1.0, 0.0, 0.5, 1.0, 1.0, 0.0)]

# Shu-Osher three-stage third-order strong-stability-preserving scheme:
# v1 = u0 + dt k(u0); v2 = 3/4 u0 + 1/4 (v1 + dt k(v1)); u1 = 1/3 u0 + 2/3 (v2 + dt k(v2))
SSPRK3 = [(1.0, 0.0, 1.0, 0.0, 0.0, 0.0),
          (0.75, 0.25, 0.25, 0.0, 0.0, 0.0),
          (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0.0, 0.0, 0.0)]

# Williamson's two-register (2N) third-order scheme: dU <- A_i dU + dt k,
# u <- u + B_i dU with A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15)
WILLIAMSON3 = [(0.0, 1.0, 0.0, 1.0 / 3.0, 0.0, 1.0),
               (0.0, 1.0, 0.0, 15.0 / 16.0, -5.0 / 9.0, 1.0),
               (0.0, 1.0, 0.0, 8.0 / 15.0, -153.0 / 128.0, 1.0)]

SCHEMES = {"rk4": RK4, "euler": EULER, "heun2": HEUN2, "ssprk3": SSPRK3, "williamson3": WILLIAMSON3}
