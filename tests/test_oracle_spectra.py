"""Pins of the Welch PSD oracle (three Hann windows, 50% overlap; Section 3.3)
against the library routine it must reduce to and against Parseval's identity."""
import numpy as np
import pytest

from oracle import spectra


@pytest.mark.parametrize("nt", [64, 1001, 4332])
def test_equals_scipy_welch(nt):
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(nt)
    x = rng.standard_normal((3, nt)) + 0.3
    dt = 0.009233
    f, P = spectra.welch_psd(x, dt)
    L = spectra.segment_length(nt)
    f2, P2 = sig.welch(x, fs=1 / dt, window="hann", nperseg=L, noverlap=L // 2, detrend="constant",
                       scaling="density", return_onesided=True, axis=-1)
    assert np.allclose(f, f2, rtol=1e-14, atol=0)
    assert np.max(np.abs(P - P2)) <= 1e-12 * np.max(np.abs(P2))


def test_parseval():
    # sum_k P_k df equals the segment-averaged windowed variance sum w^2 y^2 / sum w^2
    rng = np.random.default_rng(3)
    nt, dt = 2000, 0.01
    x = rng.standard_normal(nt)
    f, P = spectra.welch_psd(x, dt)
    L = spectra.segment_length(nt)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(L) / L)
    ref = np.mean([np.sum(w ** 2 * (x[s * L // 2:s * L // 2 + L] - x[s * L // 2:s * L // 2 + L].mean()) ** 2)
                   for s in range(3)]) / np.sum(w ** 2)
    assert abs(np.sum(P) * (f[1] - f[0]) - ref) <= 1e-12 * ref


def test_sinusoid_power_and_peak():
    # a bin-centred sine of amplitude a carries a^2/2, all within the Hann main lobe
    nt, dt = 4096, 1e-3
    L = spectra.segment_length(nt)
    k0 = 37
    a = 0.7
    t = dt * np.arange(nt)
    x = a * np.sin(2 * np.pi * k0 / (L * dt) * t)
    f, P = spectra.welch_psd(x, dt)
    df = f[1] - f[0]
    assert int(np.argmax(P)) == k0
    assert abs(np.sum(P[k0 - 1:k0 + 2]) * df - a * a / 2) <= 1e-12
    assert np.sum(P) * df == pytest.approx(a * a / 2, rel=1e-12)


def test_too_short():
    with pytest.raises(ValueError):
        spectra.welch_psd(np.zeros(3), 0.1)
