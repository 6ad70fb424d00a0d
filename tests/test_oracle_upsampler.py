"""Pins of the oracle's band-limited knot upsampler (Sec. II-C: the distance of
an image is a band-limited signal sampled at the tier's knots and recovered by
an upsampler), no GPU:
- at a virtual knot that is a knot, the distance is the exact distance there;
- a still source keeps its distance exactly (the weights sum to one);
- on a smooth path sampled at 5 Hz (the ratio 3200 at 16 kHz), the upsampled
  distance follows the exact distance far more closely than linear
  interpolation of the same knots does, within a bound set by the band-limited
  kernel's truncation.
"""
import numpy as np

from oracle import api as oracle


def _scene(traj_kind, traj, up, step=3200, K=1, duration=2.0):
    return oracle.Scene(dims=(6.0, 5.0, 3.0), beta=(0.7,) * 6, mic=(2.0, 2.5, 1.2), K=K, fs=16000.0,
                        tiers=((10**9, step, up),), taps=32, window=0, traj_kind=traj_kind, traj=traj,
                        duration=duration)


def _direct(sc):
    tab = oracle.enumerate_images(sc)
    return [i for i in range(tab["tier"].size) if np.all(tab["n"][i] == 0) and np.all(tab["p"][i] == 0)][0]


def test_knots_are_exact():
    sc = _scene(1, [3.0, 2.5, 1.5, 1.2, 1.0, 0.3], up=100)
    i = _direct(sc)
    n = np.array([0, 3200, 6400, 9600])
    _, _, d = oracle.delay_gain(sc, i, n)
    assert np.max(np.abs(d - oracle.image_distance(sc, i, n / 16000.0))) < 1e-13


def test_still_source_is_constant():
    sc = _scene(0, [3.0, 2.5, 1.5, 1.0, 0.0, 0.0, 0.0], up=64, K=2)
    tab = oracle.enumerate_images(sc)
    n = np.arange(0, 20000, 37)
    for i in range(0, tab["tier"].size, 7):
        _, _, d = oracle.delay_gain(sc, i, n)
        assert np.max(np.abs(d - d[0])) < 1e-12 * d[0]


def test_smooth_path_is_recovered():
    # circle of radius 1.2 m at 1 m/s (0.13 Hz) around (3, 2.5) seen from (2, 2.5): the
    # distance varies by about 2.4 m over the 2 s
    traj = [3.0, 2.5, 1.5, 1.2, 1.0, 0.3]
    bl, lin = _scene(1, traj, up=100), _scene(1, traj, up=1)
    i = _direct(bl)
    n = np.arange(16000, 24000, 13)                      # away from the path's ends
    exact = oracle.image_distance(bl, i, n / 16000.0)
    _, _, d_bl = oracle.delay_gain(bl, i, n)
    _, _, d_lin = oracle.delay_gain(lin, i, n)
    e_bl, e_lin = np.max(np.abs(d_bl - exact)), np.max(np.abs(d_lin - exact))
    assert e_lin > 1e-3                                 # linear interpolation between 5 Hz knots
    assert e_bl < 1e-4 and e_bl < e_lin / 10


def test_brute_force_with_upsampled_tier():
    from paper_2508_03065_gb300 import workloads as W
    from oracle import brute
    from tests.scenes import oracle_scene, rel_l2
    spec = W.small_scene(seed=13, K=2, seconds=128 / 16000.0, window=W.HANN, taps=8, traj_kind=W.CIRCLE,
                         tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)])
    x = spec.x.astype(np.float64)
    y = oracle.synthesize(oracle_scene(spec), x)
    yb = np.array(brute.synthesize(spec, list(x), x.size))
    assert rel_l2(y, yb) < 1e-12
