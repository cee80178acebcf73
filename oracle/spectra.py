"""Power spectral density of the acoustic pressure at an observer by Welch's
method, as the paper states it (Section 3.3, FW-H validation): three Hann
("Hanning") windows with 50% overlap.

Readings (the paper gives only the method, the window and the overlap):

* Segment length L = 2 floor(nt / (nseg + 1)) (even), step L/2: nseg
  half-overlapping segments cover the first (nseg + 1) L / 2 samples.
* Periodic Hann window w_n = (1 - cos(2 pi n / L)) / 2, n = 0..L-1.
* Each segment loses its mean before windowing.
* One-sided density: P_k = c_k |sum_n w_n y_n exp(-2 pi i k n / L)|^2 /
  (f_s sum_n w_n^2), f_s = 1 / dt, c_k = 2 except c_0 = c_{L/2} = 1,
  averaged over the segments; f_k = k f_s / L, k = 0..L/2.

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def segment_length(nt, nseg=3):
    """Even segment length of nseg half-overlapping segments within nt samples."""
    return 2 * (int(nt) // (nseg + 1))


def welch_psd(p, dt, nseg=3):
    """(f [L/2+1], PSD [..., L/2+1]) of the series p [..., nt] sampled every dt."""
    p = np.asarray(p, float)
    nt = p.shape[-1]
    L = segment_length(nt, nseg)
    if L < 2:
        raise ValueError("record too short for the segments")
    step = L // 2
    n = np.arange(L)
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * n / L)
    fs = 1.0 / dt
    scale = 1.0 / (fs * np.sum(w * w))
    acc = 0.0
    for s in range(nseg):
        y = p[..., s * step:s * step + L]
        y = y - y.mean(axis=-1, keepdims=True)
        X = np.fft.rfft(w * y, axis=-1)          # library FFT as one step
        P = scale * np.abs(X) ** 2
        P[..., 1:L // 2] *= 2.0
        acc = acc + P
    return np.arange(L // 2 + 1) * fs / L, acc / nseg
