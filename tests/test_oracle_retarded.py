"""Pins of the oracle's emission-time (retarded) delay model (no GPU).

Delay model 1 takes, at every knot time t, the path length c tau of the sound
that reaches the microphone at t: c tau = |r_i(t - tau) - m(t)| (the Green's
function of Sec. II-A integrated along the image's path). Pinned by:
- a still source: both delay models coincide;
- free field, a source receding radially at v: tau(t) = (r0 + v t) / (c + v)
  exactly, so y = x(t_e) / (4 pi R(t_e)) within the fractional-delay response
  error, with the moving-source Doppler frequency f0 / (1 + v/c) (the
  reception-time model gives f0 (1 - v/c));
- source and microphone moving together: the direct path's delay is constant,
  the root of a quadratic;
- the defining equation at knots, checked with the brute force's own path and
  mirroring (spline source, circling array);
- the pure-Python brute force (bisection) on a tiny room;
- derivatives: the complex-step derivative of the delay against the
  derivative of the closed-form root for uniform linear motion, and the
  complex-step loss gradient against Richardson-extrapolated central
  differences of the real-valued loss.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import api as oracle
from oracle import brute
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2


def test_still_source_models_coincide():
    spec = W.small_scene(seed=41, K=3, traj_kind=W.LINE, seconds=0.05)
    spec = replace(spec, traj=list(spec.traj[:6]) + [0.0])
    x = spec.x.astype(np.float64)
    a = oracle.synthesize(oracle_scene(spec), x)
    b = oracle.synthesize(oracle_scene(replace(spec, delay_model=1)), x)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("step", [1, 16, 800])
def test_receding_source_closed_form_and_doppler(step):
    fs, f0, v, c, r0 = 16000.0, 1000.0, 20.0, 343.0, 0.7
    m = np.array([50.0, 50.0, 50.0])
    u = np.array([2.0, -1.0, 0.5]) / np.linalg.norm([2.0, -1.0, 0.5])
    p0 = m + r0 * u
    sc = oracle.Scene(dims=(100.0, 100.0, 100.0), beta=(0.0,) * 6, mic=tuple(m), K=0, fs=fs, c=c,
                      tiers=((10**9, step),), taps=32, window=0, traj_kind=0,
                      traj=list(p0) + list(u) + [v], delay_model=1)
    n_s = int(2 * fs)
    x = np.sin(2 * np.pi * f0 * np.arange(n_s) / fs)
    y = oracle.synthesize(sc, x)
    t = np.arange(n_s) / fs
    te = (t - r0 / c) / (1.0 + v / c)
    R = r0 + v * te
    exact = np.sin(2 * np.pi * f0 * te) / (4 * np.pi * R)
    alpha = np.linspace(0, 1, 201)
    taps = oracle.tap_weights(sc, alpha)
    k = np.arange(-16, 16)
    wn = 2 * np.pi * f0 / fs
    eps = np.max(np.abs((taps * np.exp(-1j * wn * (alpha[:, None] + k[None, :]))).sum(1) - 1.0))
    valid = (te * fs > 16) & (te * fs < n_s - 17)
    assert eps < 1e-2
    assert np.max(np.abs(y - exact)[valid] * 4 * np.pi * R[valid]) <= eps * 1.01 + 1e-12
    yy = y[valid]
    zc = np.nonzero(np.diff(np.signbit(yy)))[0]
    tz = (zc + yy[zc] / (yy[zc] - yy[zc + 1])) / fs
    f_est = (len(tz) - 1) / (2 * (tz[-1] - tz[0]))
    assert abs(f_est - f0 / (1 + v / c)) < 2e-3
    assert abs(f_est - f0 * (1 - v / c)) > 2.0   # not the reception-time model


def test_comoving_direct_path_has_constant_delay():
    c, v = 343.0, 1.5
    w = np.array([0.6, 0.8, 0.0])
    s0 = np.array([2.0, 1.5, 1.4])
    m0 = np.array([3.1, 2.7, 1.2])
    sc = oracle.Scene(dims=(8.0, 7.0, 3.0), beta=(0.7,) * 6, mic=tuple(m0), K=1, fs=16000.0, c=c,
                      traj_kind=0, traj=list(s0) + list(w) + [v], arr_kind=0,
                      arr_traj=[0.0, 0.0, 0.0] + list(w) + [v], delay_model=1)
    tab = oracle.enumerate_images(sc)
    i = [i for i in range(tab["tier"].size) if np.all(tab["n"][i] == 0) and np.all(tab["p"][i] == 0)][0]
    D = s0 - m0
    vel = v * w
    a, b, cc = c * c - vel @ vel, 2 * (D @ vel), -(D @ D)   # |D - vel tau|^2 = (c tau)^2
    tau = (-b + math.sqrt(b * b - 4 * a * cc)) / (2 * a)
    t = np.linspace(0.0, 1.0, 9)
    assert np.max(np.abs(oracle.knot_delay(sc, i, t) - tau)) < 1e-14
    assert abs(oracle.knot_delay(replace(sc, delay_model=0), i, [0.5])[0] - np.linalg.norm(D) / c) < 1e-14


def test_knot_delays_solve_the_retarded_equation():
    spec = W.small_scene(seed=42, K=2, traj_kind=W.SPLINE, seconds=0.5, vmax=3.0)
    spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=[0.0, 0.0, 0.0, 0.2, 0.5, 0.3],
                   arr_duration=spec.duration, delay_model=1)
    sc = oracle_scene(spec)
    tab = oracle.enumerate_images(sc)
    mic = [float(v) for v in spec.mics[0]]
    t = np.array([0.0, 0.013, 0.2, 0.49])
    for i in range(0, tab["tier"].size, 7):
        sign = [1 - 2 * int(p) for p in tab["p"][i]]
        off = [2.0 * int(n) * L for n, L in zip(tab["n"][i], spec.dims)]
        tau = oracle.knot_delay(sc, i, t)
        for tk, tk_tau in zip(t, tau):
            q = brute.source(spec, tk - tk_tau)
            m = brute.mic_at(spec, mic, tk)
            d = math.sqrt(sum((sign[d] * q[d] + off[d] - m[d]) ** 2 for d in range(3)))
            assert abs(spec.c * tk_tau - d) < 1e-11


@pytest.mark.parametrize("traj_kind,arr", [(W.SPLINE, None), (W.CIRCLE, [0.0, 0.0, 0.0, 0.3, 1.5, 0.0])])
def test_brute_force_tiny_room_retarded(traj_kind, arr):
    spec = W.small_scene(seed=43, K=2, seconds=128 / 16000.0, window=W.HANN, taps=8,
                         traj_kind=traj_kind, tiers=[(1, 16000.0), (W.RHO_INF, 2000.0)])
    spec = replace(spec, delay_model=1)
    if arr is not None:
        spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=arr, arr_duration=spec.duration)
    x = spec.x.astype(np.float64)
    y = oracle.synthesize(oracle_scene(spec), x)
    yb = np.array(brute.synthesize(spec, list(x), x.size))
    assert rel_l2(y, yb) < 1e-12
    y0 = oracle.synthesize(oracle_scene(replace(spec, delay_model=0)), x)
    assert rel_l2(y, y0) > 1e-6   # the models differ on a moving source


def _closed_form_delay(p0, vel, m, c, t):
    # uniform motion r(t) = p0 + vel t, still microphone m: c tau = |A - vel tau|
    # with A = r(t) - m, the positive root of a quadratic (complex-safe)
    A = [p0[d] + vel[d] * t - m[d] for d in range(3)]
    vv = sum(v * v for v in vel)
    av = sum(a * v for a, v in zip(A, vel))
    aa = sum(a * a for a in A)
    a2 = c * c - vv
    return (-av + np.sqrt(av * av + a2 * aa)) / a2


@pytest.mark.parametrize("param", [0, 2, 3, 4, 6])
def test_delay_derivative_matches_closed_form_uniform_motion(param):
    """Complex-step derivative of the emission-time delay against the
    derivative of the closed-form root for uniform linear motion, for the
    direct path and mirrored images (each image moves uniformly too)."""
    c, h = 343.0, 1e-20
    base = [1.7, 2.2, 1.3, 0.6, -0.7, 0.2, 9.0]
    m = (4.1, 3.3, 1.6)
    dims = (6.0, 5.0, 3.0)
    sc = oracle.Scene(dims=dims, beta=(0.8,) * 6, mic=m, K=1, fs=16000.0, c=c,
                      traj_kind=0, traj=list(base), delay_model=1)
    tab = oracle.enumerate_images(sc)
    t = np.array([0.0, 0.011, 0.37])
    for i in range(0, tab["tier"].size, 5):
        got = oracle.knot_delay_cs(sc, i, t, param)
        sg = [1 - 2 * int(p) for p in tab["p"][i]]
        off = [2.0 * int(n) * L for n, L in zip(tab["n"][i], dims)]
        q = [complex(v) for v in base]
        q[param] += 1j * h
        nrm = np.sqrt(q[3] ** 2 + q[4] ** 2 + q[5] ** 2)
        p0 = [sg[d] * q[d] + off[d] for d in range(3)]
        vel = [sg[d] * q[6] * q[3 + d] / nrm for d in range(3)]
        want = np.array([_closed_form_delay(p0, vel, m, c, tk).imag / h for tk in t])
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want)), (i, got, want)


@pytest.mark.parametrize("traj_kind,ids", [(W.SPLINE, [0, 4, 8, 10]), (W.CIRCLE, [0, 1, 3, 4, 5])])
def test_loss_gradient_emission_time_matches_richardson(traj_kind, ids):
    """Complex-step loss gradient under emission-time delays against central
    differences of the real-valued loss with Richardson extrapolation."""
    spec = W.small_scene(seed=44, K=1, seconds=0.02, window=W.HANN, taps=16, traj_kind=traj_kind,
                         tiers=[(0, 16000.0), (W.RHO_INF, 2000.0)])
    spec = replace(spec, delay_model=1)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    target = np.random.default_rng(5).standard_normal(spec.n_in) * 0.01
    g_cs = oracle.loss_grad_cs(sc, x, target, ids + [48, 51])

    def loss_at(pid, dv):
        if pid < 48:
            tr = list(sc.traj)
            tr[pid] += dv
            return oracle.loss(replace(sc, traj=tr), x, target)
        be = list(sc.beta)
        be[pid - 48] += dv
        return oracle.loss(replace(sc, beta=tuple(be)), x, target)

    for q, pid in enumerate(ids + [48, 51]):
        hh = 1e-4
        d1 = (loss_at(pid, hh) - loss_at(pid, -hh)) / (2 * hh)
        d2 = (loss_at(pid, hh / 2) - loss_at(pid, -hh / 2)) / hh
        fd = (4 * d2 - d1) / 3
        assert abs(fd - g_cs[q]) <= 1e-6 * np.max(np.abs(g_cs)) + 1e-6 * abs(g_cs[q]), (pid, fd, g_cs[q])
    # the emission-time gradient is not the reception-time one
    g0 = oracle.loss_grad_cs(oracle_scene(replace(spec, delay_model=0)), x, target, ids)
    assert np.linalg.norm(g0 - g_cs[:len(ids)]) > 1e-4 * np.linalg.norm(g_cs[:len(ids)])
