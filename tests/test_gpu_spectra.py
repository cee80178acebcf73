"""GPU side of the acoustic post-processing rows: Welch PSD (three Hann
windows, 50% overlap, Section 3.3) against the oracle, the FW-H -> PSD chain
at many observers (a directivity circle), and the Appendix C dipole closed form
through the GPU FW-H integration."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fwh_verification.json")))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_05709_gb300 import build as B
    B.build()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("nobs,nt,nseg", [(1, 64, 3), (3, 1001, 3), (2, 4332, 3), (4, 5000, 2), (1, 3, 1)])
def test_psd_matches_oracle(nobs, nt, nseg):
    from oracle import spectra as S
    from paper_2501_05709_gb300 import fr as F
    rng = np.random.default_rng(nt + nobs)
    x = rng.standard_normal((nobs, nt)) * 1e-3 + 0.5
    ld = nt + 7                                     # padded rows, as fwh_integrate's output
    xp = np.zeros((nobs, ld))
    xp[:, :nt] = x
    P, f = F.fwh_psd(dev(xp), 0.01, nseg=nseg, nt=nt)
    fo, Po = S.welch_psd(x, 0.01, nseg=nseg)
    assert np.allclose(f, fo, rtol=1e-14, atol=0)
    P = P.cpu().numpy()
    assert P.shape == Po.shape
    assert np.max(np.abs(P - Po)) <= 1e-12 * np.max(np.abs(Po))


def test_psd_rejects_short_records():
    from paper_2501_05709_gb300 import fr as F
    with pytest.raises(F.FrError):
        F.fwh_psd(dev(np.zeros((1, 3))), 0.1, nseg=3)


def test_directivity_circle_and_psd_chain():
    # 36 observers on a circle, FW-H then PSD on the GPU, against the oracle chain
    from oracle import fwh as O
    from oracle import spectra as S
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    y, n, dS = W.sphere_surface(1.0, 12, 2 * np.pi / 18)
    M = [0.3, 0.0, 0.0]
    dt = 0.004
    tau = dt * np.arange(400)
    fld = W.monopole_field(y[None], tau[:, None], M)
    hist = np.concatenate([fld["rho"][..., None], fld["vel"], fld["p"][..., None]], axis=-1)
    ang = np.radians(np.arange(0, 360, 10))
    obs = 10.0 * np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
    p_out, nt_out, t0 = F.fwh_integrate(dev(hist), dev(y), dev(n), dev(dS), dt, 0.0, obs, M, 340.75, 1.234,
                                        fld["p0"])
    nmin = int(nt_out.min())
    P, f = F.fwh_psd(p_out, dt, nseg=3, nt=nmin)
    P = P.cpu().numpy()
    pp = p_out.cpu().numpy()
    for o in (0, 9, 17, 30):
        ts, po = O.fwh_integrate(hist, y, n, dS, dt, obs[o], M, 340.75, 1.234, fld["p0"])
        assert np.max(np.abs(pp[o, :nt_out[o]] - po)) <= 1e-12 * np.max(np.abs(po))
        _, Po = S.welch_psd(po[:nmin], dt)
        assert np.max(np.abs(P[o] - Po)) <= 1e-10 * np.max(np.abs(Po))
    # the source frequency (5 Hz) carries the peak at every angle
    k = np.argmax(P, axis=1)
    assert np.all(np.abs(f[k] - GOLD["monopole"]["omega_rad_per_s"] / (2 * np.pi)) <= 1.5 * (f[1] - f[0]))


@pytest.mark.parametrize("M", GOLD["dipole"]["mach_vectors"])
def test_dipole_closed_form_on_gpu(M):
    # Appendix C.2: the GPU FW-H reproduces the moving-medium dipole at 100 m
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    g = GOLD["monopole"]
    y, n, dS = W.sphere_surface(g["sphere_radius_m"], g["polar_sections"], g["azimuthal_spacing_rad"])
    T = 2 * np.pi / g["omega_rad_per_s"]
    dt = g["dt_over_T"] * T
    tau = dt * np.arange(int(g["periods"] / g["dt_over_T"]) + 40)
    f = W.dipole_field(y[None], tau[:, None], M, A=1e-3)
    hist = np.concatenate([f["rho"][..., None], f["vel"], f["p"][..., None]], axis=-1)
    ang = np.linspace(0.0, 2 * np.pi, 6, endpoint=False)
    dist = GOLD["dipole"]["observer_distance_m"]
    obs = dist * np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
    p_out, nt_out, t0 = F.fwh_integrate(dev(hist), dev(y), dev(n), dev(dS), dt, 0.0, obs, M, g["c0_m_per_s"],
                                        g["rho0_kg_per_m3"], f["p0"])
    pp = p_out.cpu().numpy()
    errs, rms = [], []
    for o in range(len(obs)):
        ts = t0[o] + dt * np.arange(nt_out[o])
        ex = W.dipole_field(obs[o][None, :], ts, M, A=1e-3)["pprime"]
        errs.append(np.sqrt(np.mean((pp[o, :nt_out[o]] - ex) ** 2)))
        rms.append(np.sqrt(np.mean(ex ** 2)))
    assert max(errs) / max(rms) < 1e-3
