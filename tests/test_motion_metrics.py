"""The phase and gain continuity measures (motion_metrics) on tones with known
steps (no GPU): a smooth Doppler chirp with decaying gain shows no step; a
0.3 rad phase step and a 10 % gain step at one frame boundary are found there
and not elsewhere."""
import numpy as np

from paper_2508_03065_gb300 import motion_metrics as M

FS, F0, N, FRAME = 16000.0, 1000.0, 32000, 640


def _tone(phase_step=0.0, gain_step=0.0):
    t = np.arange(N) / FS
    ph = 2 * np.pi * F0 * t - 2 * np.pi * F0 * 0.005 * t ** 2     # slow Doppler drift
    a = 1.0 - 0.2 * t
    ph[20 * FRAME:] += phase_step
    a[25 * FRAME:] *= 1.0 + gain_step
    return a * np.sin(ph)


def test_smooth_tone_has_no_steps():
    m = M.continuity(_tone(), FS, F0, FRAME, skip=2000)
    assert m["phase_step_rad"] < 1e-4 and m["gain_step"] < 1e-5 and m["gain_sawtooth"] < 1e-4


def test_phase_step_is_found_at_its_boundary():
    m = M.continuity(_tone(phase_step=0.3), FS, F0, FRAME, skip=2000)
    assert abs(m["phase_step_rad"] - 0.3) < 0.03
    assert m["phase_step_elsewhere_rad"] < 0.05


def test_gain_step_is_found_at_its_boundary():
    m = M.continuity(_tone(gain_step=0.1), FS, F0, FRAME, skip=2000)
    assert 0.07 < m["gain_step"] < 0.11
    assert m["gain_step_elsewhere"] < 0.01
