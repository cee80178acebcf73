"""FW-H acoustic integration on a stationary permeable surface in a uniformly
moving medium (Appendices A and B), advanced-time form.

Steps, in the order of Appendix B:

F1. Per panel (one point at its centre, Appendix B): centre y, outward unit
    normal n, area dS; samples rho, p and the total velocity.  Reading: the
    u_i of Eqs. A.5/A.7 is the disturbance velocity V - U_inf (with zero
    disturbance and a moving medium Q must vanish), surface velocity v = 0.
F2. Q = rho (u_n + U_inf,n) - rho0 U_inf,n (Eq. A.5) and
    L_i = (p - p0) n_i + rho u_i (u_n + U_inf,n) (Eqs. A.7-A.8, sigma_ij
    omitted: only rho, p and velocity are sampled, Section 3.4).
F3. dQ/dtau, dL_i/dtau by 4th-order central differences, one-sided 4th order
    at the two ends of the record (the paper does not give the operator).
F4. Per (panel, observer): r = x - y, gamma_PG^2 = 1/(1 - |M|^2) (the gamma of
    Eqs. B.8-B.12 is this Prandtl-Glauert factor, not the gas constant),
    R* (Eq. B.8), R (Eq. B.9), dR*/dx_i (Eq. B.11), dR/dx_i (Eq. B.12).
F5. Integrands of Eqs. B.2-B.3 with M_R = M.dR/dx, M_R* = M.dR*/dx,
    Ldot_R = Ldot.dR/dx, L_R* = L.dR*/dx (Eqs. B.4-B.7), times dS.
F6. Advanced (observer) time t = tau + R/c0 per panel (Eq. B.13); the unified
    observer window starts when the last panel's first signal arrives and
    ends when the first panel's last signal arrives; step = source step.
F7. Each panel's integrand is interpolated onto the unified times with a
    4-point cubic Lagrange stencil (the paper leaves the operator open) and
    summed (Eq. B.14); the surface is repeated along z at k*Lspan,
    k = -K..K, total length (2K+1) Lspan (Section 3.3.1, Fig. 6 caption).
F8. p'_rms about the window mean; OASPL in dB re 20 uPa.

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def ddt4(f, dt):
    """4th-order finite-difference time derivative along axis 0 (needs >= 5 samples)."""
    f = np.asarray(f, float)
    n = f.shape[0]
    if n < 5:
        raise ValueError("need at least 5 samples")
    d = np.empty_like(f)
    d[2:-2] = (f[:-4] - 8.0 * f[1:-3] + 8.0 * f[3:-1] - f[4:]) / (12.0 * dt)
    d[0] = (-25.0 * f[0] + 48.0 * f[1] - 36.0 * f[2] + 16.0 * f[3] - 3.0 * f[4]) / (12.0 * dt)
    d[1] = (-3.0 * f[0] - 10.0 * f[1] + 18.0 * f[2] - 6.0 * f[3] + f[4]) / (12.0 * dt)
    d[-1] = (25.0 * f[-1] - 48.0 * f[-2] + 36.0 * f[-3] - 16.0 * f[-4] + 3.0 * f[-5]) / (12.0 * dt)
    d[-2] = (3.0 * f[-1] + 10.0 * f[-2] - 18.0 * f[-3] + 6.0 * f[-4] - f[-5]) / (12.0 * dt)
    return d


def cubic_interp(series, s):
    """Interpolate series [Nt, P] at fractional indices s [T, P] with the 4-point
    Lagrange stencil j0..j0+3, j0 = floor(s) - 1 clamped to [0, Nt-4]."""
    Nt = series.shape[0]
    j0 = np.clip(np.floor(s).astype(np.int64) - 1, 0, Nt - 4)
    x = s - j0
    out = np.zeros(s.shape)
    cols = np.arange(s.shape[1])[None, :]
    for m in range(4):
        w = np.ones(s.shape)
        for k in range(4):
            if k != m:
                w *= (x - k) / (m - k)
        out += w * series[j0 + m, cols]
    return out


def source_terms(hist, n, M, c0, rho0, p0):
    """F1-F2: Q [Nt, P] and L [Nt, P, 3] from samples hist [Nt, P, 5]."""
    U = c0 * np.asarray(M, float)
    rho = hist[..., 0]
    u = hist[..., 1:4] - U
    p = hist[..., 4]
    un = np.sum(u * n, axis=-1)
    Un = n @ U
    Q = rho * (un + Un) - rho0 * Un
    L = (p - p0)[..., None] * n + rho[..., None] * u * (un + Un)[..., None]
    return Q, L


def fwh_integrate(hist, y, n, dS, dtau, obs, M, c0, rho0, p0, Lspan=0.0, ncopies=1, tau0=0.0):
    """Acoustic pressure p'(t*) at observer obs [3].

    hist [Nt, P, 5] = (rho, V1, V2, V3, p) per source time tau0 + k dtau.
    Returns (t* [T], p' [T]).  Raises ValueError if the window is empty.
    """
    hist = np.asarray(hist, float)
    Nt = hist.shape[0]
    M = np.asarray(M, float)
    Q, L = source_terms(hist, n, M, c0, rho0, p0)
    Qd = ddt4(Q, dtau)
    Ld = ddt4(L, dtau)
    b2 = 1.0 / (1.0 - M @ M)
    if ncopies < 1 or ncopies % 2 == 0:
        raise ValueError("ncopies must be odd")
    K = (ncopies - 1) // 2
    ez = np.array([0.0, 0.0, 1.0])
    parts = []
    for k in range(-K, K + 1):
        r = np.asarray(obs, float)[None, :] - (y + k * Lspan * ez)
        Mr = r @ M
        Rs = np.sqrt(np.sum(r * r, axis=1) + b2 * Mr ** 2) / np.sqrt(b2)
        R = b2 * (Rs - Mr)
        Rts = (r + b2 * Mr[:, None] * M) / (b2 * Rs[:, None])
        Rt = b2 * (Rts - M)
        MR = Rt @ M
        MRs = Rts @ M
        IT = ((1.0 - MR) * Qd / Rs - Q * c0 * MRs / Rs ** 2) * dS
        IL = ((np.einsum("tpi,pi->tp", Ld, Rt) / c0) / Rs
              + np.einsum("tpi,pi->tp", L, Rts) / Rs ** 2) * dS
        parts.append((IT + IL, R / c0))
    delays = np.concatenate([d for _, d in parts])
    start = tau0 + delays.max()
    end = tau0 + (Nt - 1) * dtau + delays.min()
    if end < start:
        raise ValueError("empty observer window")
    T = int(np.floor((end - start) / dtau + 1e-9)) + 1
    tstar = start + dtau * np.arange(T)
    acc = np.zeros(T)
    for I, delay in parts:
        s = (tstar[:, None] - tau0 - delay[None, :]) / dtau
        acc += cubic_interp(I, s).sum(axis=1)
    return tstar, acc / (4.0 * np.pi)


def prms(pp):
    """Root mean square of p' about its mean over the window."""
    pp = np.asarray(pp, float)
    return float(np.sqrt(np.mean((pp - pp.mean()) ** 2)))


def oaspl(p_rms, p_inf=1.0, p_inf_dim=101325.0, p_ref=2e-5):
    """OASPL in dB re 20 uPa; a nondimensional p_rms is scaled by p_inf_dim/p_inf."""
    return 20.0 * np.log10(p_rms * (p_inf_dim / p_inf) / p_ref)
