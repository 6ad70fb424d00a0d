"""Pins of the oracle with a moving microphone array (no GPU).

The microphones move rigidly, m(t) = m + a(t) - a(0), a(t) a trajectory of the
source's kinds. Pinned by:
- comoving source and array on the same line: every unmirrored image (p = 0)
  keeps its distance; mirrored ones do not;
- relative motion on the direct path: a still source with the array displaced
  by w(t) equals a source displaced by -w(t) with a still array;
- free field, microphone receding radially from a still source at v: the
  received 1 kHz sine is x(t - r(t)/c) / (4 pi r(t)) within the fractional-delay
  response error, with apparent frequency f0 (1 - v/c);
- the pure-Python brute force (mirroring, de Boor) on a tiny room with a
  circling array;
- derivatives with respect to the array trajectory: the complex step of a knot
  delay against that of the explicit distance (a line array), and the
  complex-step loss gradient against Richardson-extrapolated central
  differences (circle and spline arrays, both delay models).
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import api as oracle
from oracle import brute
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2


def _scene(**kw):
    base = dict(dims=(6.0, 5.0, 3.0), beta=(0.7, 0.8, 0.6, 0.9, 0.75, 0.65), mic=(2.5, 2.0, 1.2),
                K=2, fs=16000.0, tiers=((1, 1), (10**9, 16)), taps=32, window=0,
                traj_kind=0, traj=[1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 1.0], duration=1.0)
    base.update(kw)
    return oracle.Scene(**base)


def test_comoving_source_and_array_keep_unmirrored_distances():
    line = [3.0, 2.0, 0.5, 1.0]          # direction and speed shared by both
    sc = _scene(traj=[1.5, 1.2, 1.4] + line, arr_kind=0, arr_traj=[0.0, 0.0, 0.0] + line)
    tab = oracle.enumerate_images(sc)
    t = np.linspace(0.0, 1.0, 9)
    moved = 0
    for i in range(tab["tier"].size):
        d = oracle.image_distance(sc, i, t)
        if np.all(tab["p"][i] == 0):
            assert np.max(np.abs(d - d[0])) < 1e-12
        else:
            moved += np.max(np.abs(d - d[0])) > 1e-3
    assert moved > 0


def test_relative_motion_on_the_direct_path():
    w = [0.6, -0.3, 0.2, 0.8]            # direction and speed of the displacement
    s0 = [2.0, 2.5, 1.5]
    a = _scene(traj=s0 + [1.0, 0.0, 0.0, 0.0], arr_kind=0, arr_traj=[0.0, 0.0, 0.0] + w)
    b = _scene(traj=s0 + [-v for v in w[:3]] + [w[3]])
    ta, tb = oracle.enumerate_images(a), oracle.enumerate_images(b)
    ia = [i for i in range(ta["tier"].size) if np.all(ta["n"][i] == 0) and np.all(ta["p"][i] == 0)][0]
    ib = [i for i in range(tb["tier"].size) if np.all(tb["n"][i] == 0) and np.all(tb["p"][i] == 0)][0]
    t = np.linspace(0.0, 1.0, 11)
    assert np.max(np.abs(oracle.image_distance(a, ia, t) - oracle.image_distance(b, ib, t))) < 1e-12


def test_free_field_receding_microphone_doppler():
    fs, f0, v, c = 16000.0, 1000.0, 2.0, 343.0
    src = np.array([2.0, 2.0, 1.5])
    m0 = np.array([2.6, 2.8, 1.5])
    u = (m0 - src) / np.linalg.norm(m0 - src)
    sc = _scene(dims=(8.0, 8.0, 3.0), beta=(0.0,) * 6, mic=tuple(m0), K=0, fs=fs, c=c,
                traj_kind=0, traj=list(src) + [1.0, 0.0, 0.0, 0.0], taps=32, window=0,
                arr_kind=0, arr_traj=[0.0, 0.0, 0.0] + list(u) + [v])
    n_s = int(2 * fs)
    x = np.sin(2 * np.pi * f0 * np.arange(n_s) / fs)
    y = oracle.synthesize(sc, x)
    n = np.arange(n_s)
    r = np.linalg.norm(m0 - src) + v * n / fs
    exact = np.sin(2 * np.pi * f0 * (n / fs - r / c)) / (4 * np.pi * r)
    alpha = np.linspace(0, 1, 201)
    taps = oracle.tap_weights(sc, alpha)
    k = np.arange(-16, 16)
    wn = 2 * np.pi * f0 / fs
    eps = np.max(np.abs((taps * np.exp(-1j * wn * (alpha[:, None] + k[None, :]))).sum(1) - 1.0))
    tau = r * fs / c
    valid = (n - tau > 16) & (n - tau < n_s - 17)
    assert eps < 1e-2
    assert np.max(np.abs(y - exact)[valid] * 4 * np.pi * r[valid]) <= eps * 1.01 + 1e-12
    yy = y[valid]
    zc = np.nonzero(np.diff(np.signbit(yy)))[0]
    tz = (zc + yy[zc] / (yy[zc] - yy[zc + 1])) / fs
    f_est = (len(tz) - 1) / (2 * (tz[-1] - tz[0]))
    assert abs(f_est - f0 * (1 - v / c)) < 1e-3 * f0 * v / c + 1e-6 * f0


@pytest.mark.parametrize("arr_kind,arr_traj", [
    (W.CIRCLE, [0.0, 0.0, 0.0, 0.3, 1.5, 0.0]),
    (W.LINE, [0.0, 0.0, 0.0, 1.0, -1.0, 0.3, 1.2]),
])
def test_brute_force_tiny_room_moving_array(arr_kind, arr_traj):
    spec = W.small_scene(seed=12, K=2, seconds=128 / 16000.0, window=W.HANN, taps=8,
                         traj_kind=W.SPLINE, tiers=[(1, 16000.0), (W.RHO_INF, 2000.0)])
    spec = replace(spec, arr_kind=arr_kind, arr_traj=arr_traj, arr_duration=spec.duration)
    x = spec.x.astype(np.float64)
    y = oracle.synthesize(oracle_scene(spec), x)
    yb = np.array(brute.synthesize(spec, list(x), x.size))
    assert rel_l2(y, yb) < 1e-12


@pytest.mark.parametrize("param", [54, 56, 57, 58, 60])
def test_array_derivative_matches_closed_form(param):
    """Complex-step derivative of a knot delay with respect to the array's line
    parameters (ids 54.., arr_traj[]) against the complex-step derivative of the
    explicit distance |r_i - (m + v t u)|, u = dir / |dir|, for the direct path
    and mirrored images (reception-time delays; the array's offset a(0) cancels)."""
    h = 1e-20
    arr = [0.3, -0.2, 0.1, 0.6, 0.8, 0.1, 0.9]
    sc = _scene(traj_kind=0, traj=[1.2, 1.1, 1.4, 1.0, 0.5, 0.0, 0.0], arr_kind=0, arr_traj=arr, arr_duration=1.0)
    tab = oracle.enumerate_images(sc)
    t = np.array([0.0, 0.2, 0.7])
    src = np.array(sc.traj[:3])
    for i in range(0, tab["tier"].size, 9):
        got = oracle.knot_delay_cs(sc, i, t, param)
        sg = np.array([1 - 2 * int(p) for p in tab["p"][i]])
        r = sg * src + 2.0 * np.array([int(n) for n in tab["n"][i]]) * np.array(sc.dims)
        q = np.array(arr, dtype=complex)
        q[param - 54] += 1j * h
        u = q[3:6] / np.sqrt(np.sum(q[3:6] ** 2))
        want = []
        for tk in t:
            m = np.array(sc.mic) + q[6] * tk * u          # a(t) - a(0) = v t u (the p0 terms cancel)
            want.append((np.sqrt(np.sum((r - m) ** 2)) / sc.c).imag / h)
        want = np.array(want)
        assert np.max(np.abs(got - want)) <= 1e-10 * max(np.max(np.abs(want)), 1e-12), (i, got, want)


@pytest.mark.parametrize("delay_model,arr_kind,ids", [(0, W.CIRCLE, [54, 55, 57, 58, 59]),
                                                      (0, W.SPLINE, [54, 58, 62, 65]),
                                                      (1, W.LINE, [54, 57, 58, 60])])
def test_array_loss_gradient_matches_richardson(delay_model, arr_kind, ids):
    """Complex-step loss gradient with respect to the array trajectory's
    parameters against central differences of the real loss with Richardson
    extrapolation."""
    spec = W.small_scene(seed=46, K=1, seconds=0.02, window=W.HANN, taps=16, traj_kind=W.SPLINE,
                         tiers=[(0, 16000.0), (W.RHO_INF, 2000.0)])
    arr = {W.LINE: [0.0, 0.0, 0.0, 0.3, 0.9, 0.2, 0.8],
           W.CIRCLE: [0.0, 0.0, 0.0, 0.12, 0.6, 0.4],
           W.SPLINE: [0.0, 0.0, 0.0, 0.05, 0.02, 0.0, 0.08, 0.07, 0.01, 0.1, 0.12, 0.03]}[arr_kind]
    spec = replace(spec, delay_model=delay_model, arr_kind=arr_kind, arr_traj=arr, arr_duration=spec.duration,
                   arr_n_ctrl=4 if arr_kind == W.SPLINE else 0)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    target = np.random.default_rng(6).standard_normal(spec.n_in) * 0.01
    g_cs = oracle.loss_grad_cs(sc, x, target, ids)

    def loss_at(pid, dv):
        a = list(sc.arr_traj)
        a[pid - 54] += dv
        return oracle.loss(replace(sc, arr_traj=a), x, target)

    for q, pid in enumerate(ids):
        hh = 1e-4
        d1 = (loss_at(pid, hh) - loss_at(pid, -hh)) / (2 * hh)
        d2 = (loss_at(pid, hh / 2) - loss_at(pid, -hh / 2)) / hh
        fd = (4 * d2 - d1) / 3
        assert abs(fd - g_cs[q]) <= 1e-6 * np.max(np.abs(g_cs)) + 1e-6 * abs(g_cs[q]), (pid, fd, g_cs[q])
