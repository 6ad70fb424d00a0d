"""Phase and gain continuity of a received tone (the measures behind the
paper's first experiment, Sec. III: a moving 1 kHz source simulated by the
method vs by static-response splicing, compared for phase discontinuities
and gain sawtooth).

The received signal y is brought to baseband around the tone frequency f0:
z(n) = analytic(y)(n) e^{-j 2 pi f0 n / fs}, whose magnitude is the gain
envelope and whose unwrapped angle is the phase. Both vary smoothly for a
continuously moving source; splicing adds steps at the frame boundaries.
"""
from __future__ import annotations

import numpy as np


def baseband(y: np.ndarray, fs: float, f0: float) -> np.ndarray:
    """Complex envelope of a narrow-band signal around f0 (FFT analytic signal,
    demodulated, then averaged over one period of f0 to remove the residue of
    other components)."""
    y = np.asarray(y, np.float64)
    n = y.size
    Y = np.fft.fft(y)
    h = np.zeros(n)
    h[0] = 1.0
    if n % 2 == 0:
        h[n // 2] = 1.0
        h[1:n // 2] = 2.0
    else:
        h[1:(n + 1) // 2] = 2.0
    a = np.fft.ifft(Y * h)
    z = a * np.exp(-2j * np.pi * f0 * np.arange(n) / fs)
    per = max(1, int(round(fs / f0)))
    k = np.ones(per) / per
    return np.convolve(z, k, mode="same")


def continuity(y: np.ndarray, fs: float, f0: float, frame_len: int, skip: int = 0) -> dict:
    """Largest phase step (radians) and relative gain step at the frame
    boundaries, compared with the largest per-sample change elsewhere, and the
    gain sawtooth (RMS of the gain minus its three-frame moving average,
    relative to the mean gain). `skip` samples at each end are ignored."""
    z = baseband(y, fs, f0)
    ph = np.unwrap(np.angle(z))
    g = np.abs(z)
    lo, hi = skip, z.size - skip
    dph = np.diff(ph)[lo:hi - 1]
    dg = np.diff(g)[lo:hi - 1] / max(np.mean(g[lo:hi]), 1e-300)
    idx = np.arange(lo, hi - 1)
    at = (idx + 1) % frame_len == 0                      # step from the last sample of a frame
    # local trend of the per-sample changes (Doppler drift, distance decay):
    # their average over a frame; steps are smeared over one period of f0 by
    # the envelope average, so the excess is summed over one period
    per = max(1, int(round(fs / f0)))
    trend = np.ones(frame_len) / frame_len
    kern = np.ones(per)
    sph = np.convolve(dph - np.convolve(dph, trend, mode="same"), kern, mode="same")
    sg = np.convolve(dg - np.convolve(dg, trend, mode="same"), kern, mode="same")
    # "elsewhere": samples at least one period away from every boundary; both
    # sets keep clear of the ends, where the moving averages are truncated
    pos = (idx + 1) % frame_len
    inner = (idx >= lo + frame_len + per) & (idx < hi - 1 - frame_len - per)
    at &= inner
    far = (np.minimum(pos, frame_len - pos) > per) & inner
    w = 3 * frame_len
    mov = np.convolve(g, np.ones(w) / w, mode="same")
    saw = np.sqrt(np.mean((g[lo + w:hi - w] - mov[lo + w:hi - w]) ** 2)) / np.mean(g[lo + w:hi - w])
    return {
        "phase_step_rad": float(np.max(np.abs(sph[at]))) if np.any(at) else 0.0,
        "phase_step_elsewhere_rad": float(np.max(np.abs(sph[far]))),
        "gain_step": float(np.max(np.abs(sg[at]))) if np.any(at) else 0.0,
        "gain_step_elsewhere": float(np.max(np.abs(sg[far]))),
        "gain_sawtooth": float(saw),
    }
