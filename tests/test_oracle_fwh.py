"""Pins of the oracle's FW-H integration (Appendix B) against the closed-form
moving-medium monopole and dipole of Appendix C, and of its numerical
ingredients against closed forms."""
import json
import os

import numpy as np
import pytest

from oracle import fwh
from paper_2501_05709_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fwh_verification.json")))


def _history(field, y, tau, M, A=1.0):
    f = field(y[None, :, :], tau[:, None], M, A=A)
    return np.concatenate([f["rho"][..., None], f["vel"], f["p"][..., None]], axis=-1), f["p0"]


def _relerr(field, dist, M, plane, A=1.0, nobs=6):
    g = GOLD["monopole"]
    y, n, dS = W.sphere_surface(g["sphere_radius_m"], g["polar_sections"], g["azimuthal_spacing_rad"])
    T = 2 * np.pi / g["omega_rad_per_s"]
    dt = g["dt_over_T"] * T
    tau = dt * np.arange(int(g["periods"] / g["dt_over_T"]) + 40)
    hist, p0 = _history(field, y, tau, M, A)
    errs, rms = [], []
    for ang in np.linspace(0.0, 2 * np.pi, nobs, endpoint=False):
        obs = dist * (np.array([np.cos(ang), 0, np.sin(ang)]) if plane == "x1x3"
                      else np.array([np.cos(ang), np.sin(ang), 0]))
        ts, pp = fwh.fwh_integrate(hist, y, n, dS, dt, obs, M, g["c0_m_per_s"], g["rho0_kg_per_m3"], p0)
        ex = field(obs[None, :], ts, M, A=A)["pprime"]
        errs.append(np.sqrt(np.mean((pp - ex) ** 2)))
        rms.append(np.sqrt(np.mean(ex ** 2)))
    return max(errs) / max(rms)


@pytest.mark.parametrize("M", GOLD["monopole"]["mach_vectors"])
def test_monopole_moving_medium(M):
    assert _relerr(W.monopole_field, GOLD["monopole"]["observer_distance_m"], M, "x1x3") < 1e-3


@pytest.mark.parametrize("M", GOLD["dipole"]["mach_vectors"])
def test_dipole_moving_medium(M):
    # linear-acoustics amplitude, so the quadratic terms of Q and L_i stay negligible
    assert _relerr(W.dipole_field, GOLD["dipole"]["observer_distance_m"], M, "x1x2", A=1e-3) < 1e-3


def test_dipole_full_amplitude():
    # A = 1 as printed: nonlinear source terms add a small, Mach-dependent error
    assert _relerr(W.dipole_field, 100.0, [0.8, 0.0, 0.4], "x1x2") < 5e-3


def test_moving_medium_field_solves_convective_wave_equation():
    # guard for the closed form itself: (1/c^2)(d/dt + U.grad)^2 phi = lap phi
    M = np.array([0.5, 0.1, 0.5])
    c0, om = 340.75, 10 * np.pi
    x0 = np.array([3.0, -2.0, 1.5])
    h, ht = 1e-3, 1e-5

    def phi(x, t):
        b2 = 1.0 / (1.0 - M @ M)
        Mr = x @ M
        Rs = np.sqrt(x @ x + b2 * Mr ** 2) / np.sqrt(b2)
        R = b2 * (Rs - Mr)
        return np.exp(1j * om * (t - R / c0)) / (4 * np.pi * Rs)

    def Dt(f):
        return lambda x, t: (f(x, t + ht) - f(x, t - ht)) / (2 * ht)

    def Dx(f, k):
        e = np.zeros(3)
        e[k] = h
        return lambda x, t: (f(x + e, t) - f(x - e, t)) / (2 * h)

    def conv(f):
        return lambda x, t: Dt(f)(x, t) + c0 * sum(M[k] * Dx(f, k)(x, t) for k in range(3))

    lhs = conv(conv(phi))(x0, 0.1) / c0 ** 2
    lap = sum((phi(x0 + h * e, 0.1) - 2 * phi(x0, 0.1) + phi(x0 - h * e, 0.1)) / h ** 2 for e in np.eye(3))
    assert abs(lhs - lap) < 1e-4 * abs(lap)


def test_zero_disturbance_gives_zero_sources():
    # reading of u_i as the disturbance velocity: uniform free stream -> Q = L = 0
    y, n, dS = W.sphere_surface()
    M = np.array([0.3, 0.1, 0.2])
    c0, rho0 = 340.0, 1.2
    p0 = rho0 * c0 ** 2 / 1.4
    hist = np.zeros((6, len(y), 5))
    hist[..., 0] = rho0
    hist[..., 1:4] = c0 * M
    hist[..., 4] = p0
    Q, L = fwh.source_terms(hist, n, M, c0, rho0, p0)
    assert np.max(np.abs(Q)) < 1e-12 and np.max(np.abs(L)) < 1e-9


def test_ddt4_and_cubic_interp_exact_on_polynomials():
    t = 0.1 * np.arange(12)
    f = 2.0 - t + 0.5 * t ** 2 - 0.3 * t ** 3 + 0.2 * t ** 4
    df = -1.0 + t - 0.9 * t ** 2 + 0.8 * t ** 3
    assert np.max(np.abs(fwh.ddt4(f, 0.1) - df)) < 1e-10
    g = (1.0 + t - 2 * t ** 2 + t ** 3)[:, None]
    s = np.array([[0.3], [4.7], [10.6], [0.0], [11.0]])
    tt = 0.1 * s
    assert np.allclose(fwh.cubic_interp(g, s), 1.0 + tt - 2 * tt ** 2 + tt ** 3, atol=1e-12)


def test_copies_with_zero_shift_are_additive():
    y, n, dS = W.sphere_surface(1.0, 10, 2 * np.pi / 15)
    M = [0.2, 0.0, 0.1]
    dt = 0.004
    tau = dt * np.arange(120)
    hist, p0 = _history(W.monopole_field, y, tau, M)
    obs = np.array([0.0, -20.0, 0.0])
    t1, p1 = fwh.fwh_integrate(hist, y, n, dS, dt, obs, M, 340.75, 1.234, p0)
    t3, p3 = fwh.fwh_integrate(hist, y, n, dS, dt, obs, M, 340.75, 1.234, p0, Lspan=0.0, ncopies=3)
    assert np.allclose(t1, t3) and np.allclose(p3, 3 * p1, rtol=1e-12, atol=1e-15)


def test_empty_window_raises():
    y, n, dS = W.sphere_surface(1.0, 6, 2 * np.pi / 8)
    hist, p0 = _history(W.monopole_field, y, 0.004 * np.arange(8), [0, 0, 0])
    with pytest.raises(ValueError):
        fwh.fwh_integrate(hist, y, n, dS, 0.004, np.array([0, 30.0, 0]), [0, 0, 0], 340.75, 1.234, p0,
                          Lspan=50.0, ncopies=5)


def test_oaspl_reference():
    assert abs(fwh.oaspl(2e-5, p_inf=1.0, p_inf_dim=1.0)) < 1e-12
    assert abs(fwh.oaspl(2e-4, 1.0, 1.0) - 20.0) < 1e-12
    assert abs(fwh.prms([1.0, -1.0, 1.0, -1.0]) - 1.0) < 1e-15
