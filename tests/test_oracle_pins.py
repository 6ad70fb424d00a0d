"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test fixes a part of the oracle with a closed form, a library routine, a
brute-force reading or an invariant, chosen so that a plausible mistake (a
dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import i0 as scipy_i0

from oracle import api as oracle
from oracle import brute
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(**kw):
    base = dict(dims=(5.0, 4.0, 3.0), beta=(0.7, 0.8, 0.6, 0.9, 0.75, 0.65), mic=(2.5, 2.0, 1.2),
                K=3, fs=16000.0, tiers=((1, 1), (10**9, 16)), taps=32, window=0,
                traj_kind=0, traj=[1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 1.0], duration=1.0)
    base.update(kw)
    return oracle.Scene(**base)


# ----------------------------------------------------------------- image set
def test_image_count_closed_form():
    # |n|_1 <= K lattice triples times 8 parities: 8 (2K+1)(2K^2+2K+3)/3
    for K in range(0, 9):
        assert oracle.image_count(K) == W.image_count(K)
    with open(os.path.join(GOLDEN, "image_counts.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for K, cnt in rows:
        assert oracle.image_count(int(K)) == int(cnt)


def test_reflection_shells_complete():
    # Images with exactly rho reflections form the surface of an L1 ball of
    # radius rho in reflection-count space: 1 image for rho=0, 4 rho^2 + 2 else.
    # Every such image lies in |n|_1 <= K when rho <= 2K-3.
    K = 6
    tab = oracle.enumerate_images(_scene(K=K))
    for rho in range(0, 2 * K - 2):
        expect = 1 if rho == 0 else 4 * rho * rho + 2
        assert int(np.sum(tab["rho"] == rho)) == expect, rho


def test_enumeration_matches_mirroring():
    # Brute-force mirroring of the source across the six walls must produce
    # exactly the images of the lattice set with rho <= 2K-3, with the same
    # per-wall reflection counts and the same distance to the microphone.
    K = 3
    sc = _scene(K=K, traj=[1.3, 0.7, 1.1, 1.0, 0.0, 0.0, 0.0])  # static source
    tab = oracle.enumerate_images(sc)
    src = np.array([1.3, 0.7, 1.1])
    mic = np.array(sc.mic)
    max_rho = 2 * K - 3
    bfs = brute.mirror_images(sc.dims, max_rho)
    assert len(bfs) == 1 + sum(4 * r * r + 2 for r in range(1, max_rho + 1))
    lookup = {}
    for i in range(len(tab["rho"])):
        key = (tuple(tab["n"][i]), tuple(tab["p"][i]))
        lookup[key] = i
    seen = set()
    for sign, off, hits in bfs:
        n, p = brute.lattice_of(sign, off, sc.dims)
        i = lookup[(tuple(n), tuple(p))]
        seen.add(i)
        assert tuple(tab["e"][i]) == tuple(hits)
        assert tab["rho"][i] == sum(hits)
        pos = np.array(sign) * src + np.array(off)
        d_bfs = np.linalg.norm(pos - mic)
        d_orc = oracle.image_distance(sc, i, [0.0])[0]
        assert abs(d_bfs - d_orc) < 1e-12
        beta = np.prod([sc.beta[w] ** hits[w] for w in range(6)])
        assert abs(tab["beta"][i] - beta) < 1e-15
    expect = {i for i in range(len(tab["rho"])) if tab["rho"][i] <= max_rho}
    assert seen == expect


def test_tier_assignment():
    sc = _scene(K=4, tiers=((0, 1), (3, 4), (10**9, 16)))
    tab = oracle.enumerate_images(sc)
    rho, tier = tab["rho"], tab["tier"]
    assert np.all(tier[rho == 0] == 0)
    assert np.all(tier[(rho >= 1) & (rho <= 3)] == 1)
    assert np.all(tier[rho >= 4] == 2)


# ----------------------------------------------------------------- kernel
@pytest.mark.parametrize("L", [8, 32, 64])
def test_hann_window_matches_numpy(L):
    sc = _scene(taps=L, window=0)
    u = np.arange(L + 1) - L / 2
    assert np.max(np.abs(oracle.window(sc, u) - np.hanning(L + 1))) < 1e-15


@pytest.mark.parametrize("L", [32, 64])
def test_kaiser_window_matches_library(L):
    beta = 8.0
    sc = _scene(taps=L, window=1, kaiser_beta=beta)
    u = np.arange(L + 1) - L / 2
    assert np.max(np.abs(oracle.window(sc, u) - np.kaiser(L + 1, beta))) < 1e-13
    rng = np.random.default_rng(0)
    v = rng.uniform(-L / 2, L / 2, 200)
    ref = scipy_i0(beta * np.sqrt(1 - (2 * v / L) ** 2)) / scipy_i0(beta)
    assert np.max(np.abs(oracle.window(sc, v) - ref)) < 1e-14


@pytest.mark.parametrize("window", [0, 1])
def test_taps_are_windowed_sinc(window):
    sc = _scene(taps=32, window=window)
    alpha = np.random.default_rng(1).uniform(0, 1, 50)
    taps = oracle.tap_weights(sc, alpha)
    k = np.arange(-16, 16)
    for a, row in zip(alpha, taps):
        u = a + k
        assert np.max(np.abs(row - oracle.window(sc, u) * np.sinc(u))) < 1e-15
    # alpha = 0: a pure integer shift (unit impulse at k = 0)
    imp = oracle.tap_weights(sc, [0.0])[0]
    assert imp[16] == 1.0 and np.max(np.abs(np.delete(imp, 16))) < 1e-16


# ----------------------------------------------------------------- trajectories
def test_spline_with_four_points_is_bezier():
    ctrl = np.array([[1.0, 1.0, 1.0], [2.5, 0.5, 1.5], [3.0, 3.0, 2.0], [4.0, 2.0, 1.2]])
    sc = _scene(traj_kind=2, traj=list(ctrl.ravel()), n_ctrl=4, duration=2.0)
    t = np.linspace(0, 2.0, 41)
    u = t / 2.0
    bern = np.stack([(1 - u) ** 3, 3 * u * (1 - u) ** 2, 3 * u * u * (1 - u), u ** 3], 1)
    assert np.max(np.abs(oracle.source_position(sc, t) - bern @ ctrl)) < 1e-14
    # clamped: the parameter stops at u = 1 past the duration
    assert np.max(np.abs(oracle.source_position(sc, [3.0])[0] - ctrl[-1])) < 1e-14


def test_spline_matches_de_boor():
    rng = np.random.default_rng(3)
    ctrl = rng.uniform(1, 3, (7, 3))
    sc = _scene(traj_kind=2, traj=list(ctrl.ravel()), n_ctrl=7, duration=1.5)
    sp = W.SceneSpec(dims=sc.dims, beta=sc.beta, mics=np.array([sc.mic]), K=1, fs=16000.0,
                     tiers=[(1, 16000.0)], traj_kind=2, traj=list(ctrl.ravel()), n_ctrl=7,
                     duration=1.5)
    for t in np.linspace(0, 1.5, 37):
        assert np.max(np.abs(oracle.source_position(sc, [t])[0] - np.array(brute.source(sp, t)))) < 1e-13


def test_line_and_circle_closed_forms():
    sc = _scene(traj_kind=0, traj=[1.0, 1.0, 1.5, 3.0, 4.0, 0.0, 2.0])
    p = oracle.source_position(sc, [0.5])[0]
    assert np.allclose(p, [1.0 + 2.0 * 0.5 * 0.6, 1.0 + 2.0 * 0.5 * 0.8, 1.5], atol=1e-15)
    sc = _scene(traj_kind=1, traj=[2.0, 2.0, 1.5, 1.0, 0.5, 0.0])
    t = np.linspace(0, 4 * np.pi, 9)  # angular speed 0.5 rad/s: one turn in 4 pi s
    p = oracle.source_position(sc, t)
    assert np.allclose(np.hypot(p[:, 0] - 2.0, p[:, 1] - 2.0), 1.0, atol=1e-14)
    assert np.allclose(p[0], [3.0, 2.0, 1.5], atol=1e-15)
    assert np.allclose(p[-1], p[0], atol=1e-13)
    assert np.allclose(p[4], [1.0, 2.0, 1.5], atol=1e-13)   # half a turn
    assert np.allclose(p[2], [2.0, 3.0, 1.5], atol=1e-13)   # a quarter turn, counter-clockwise


# ----------------------------------------------------------------- knots
def test_knots_reproduce_exact_distances_and_interpolate_linearly():
    sc = _scene(K=2, tiers=((1, 1), (10**9, 16)), traj_kind=1, traj=[2.5, 2.0, 1.5, 1.0, 1.5, 0.2])
    tab = oracle.enumerate_images(sc)
    i = int(np.nonzero(tab["tier"] == 1)[0][5])
    n = np.arange(0, 160)
    tau, g, d = oracle.delay_gain(sc, i, n)
    exact = oracle.image_distance(sc, i, n / sc.fs)
    knots = n % 16 == 0
    assert np.max(np.abs(d[knots] - exact[knots])) < 1e-13
    # in between, the distance is the chord between neighbouring knots
    j = n // 16
    d0 = oracle.image_distance(sc, i, j * 16 / sc.fs)
    d1 = oracle.image_distance(sc, i, (j + 1) * 16 / sc.fs)
    s = (n - 16 * j) / 16.0
    assert np.max(np.abs(d - ((1 - s) * d0 + s * d1))) < 1e-13
    assert np.max(np.abs(tau - d * sc.fs / sc.c)) < 1e-9
    assert np.max(np.abs(g - tab["beta"][i] / (4 * np.pi * d))) < 1e-15
    # chord error of a curve is bounded by (h^2/8) max|d''|; for a circle of
    # radius R at speed v, |d''| <= v^2/d + v^2/R
    v, R = 1.5, 1.0
    h = 16 / sc.fs
    bound = h * h / 8 * (v * v / np.min(exact) + v * v / R)
    assert np.max(np.abs(d - exact)) <= bound * 1.0001


def test_dense_tiers_are_exact():
    sc = _scene(K=2, tiers=((10**9, 1),), traj_kind=1, traj=[2.5, 2.0, 1.5, 1.0, 1.5, 0.2])
    n = np.arange(0, 50)
    for i in (0, 17, 93):
        _, _, d = oracle.delay_gain(sc, i, n)
        assert np.max(np.abs(d - oracle.image_distance(sc, i, n / sc.fs))) < 1e-13


# ----------------------------------------------------------------- closed forms
def test_free_field_doppler():
    # All walls absorbing: only the direct image remains. A 1 kHz sine (the
    # excitation of the paper's Sec. III experiment) from a source receding
    # radially at v must arrive as x(t - r(t)/c) / (4 pi r(t)): a Doppler-shifted
    # sine at f0 (1 - v/c), up to the windowed-sinc response error at f0.
    fs, f0, v, c = 16000.0, 1000.0, 2.0, 343.0
    mic = np.array([2.0, 2.0, 1.5])
    p0 = np.array([2.6, 2.8, 1.5])
    u = (p0 - mic) / np.linalg.norm(p0 - mic)
    sc = _scene(dims=(8.0, 8.0, 3.0), beta=(0.0,) * 6, mic=tuple(mic), K=0, fs=fs, c=c,
                traj_kind=0, traj=list(p0) + list(u) + [v], taps=32, window=0)
    n_s = int(2 * fs)
    x = np.sin(2 * np.pi * f0 * np.arange(n_s) / fs)
    y = oracle.synthesize(sc, x)
    n = np.arange(n_s)
    r = np.linalg.norm(p0 - mic) + v * n / fs
    exact = np.sin(2 * np.pi * f0 * (n / fs - r / c)) / (4 * np.pi * r)
    # response error of the fractional-delay filter at f0
    alpha = np.linspace(0, 1, 201)
    taps = oracle.tap_weights(sc, alpha)
    k = np.arange(-16, 16)
    w = 2 * np.pi * f0 / fs
    H = (taps * np.exp(-1j * w * (alpha[:, None] + k[None, :]))).sum(1)
    eps = np.max(np.abs(H - 1.0))
    tau = r * fs / c
    valid = (n - tau > 16) & (n - tau < n_s - 17)
    err = np.abs(y - exact)[valid] * 4 * np.pi * r[valid]
    assert eps < 1e-2
    assert np.max(err) <= eps * 1.01 + 1e-12
    # apparent frequency from the zero crossings of the received sine
    yy = y[valid]
    zc = np.nonzero(np.diff(np.signbit(yy)))[0]
    frac = yy[zc] / (yy[zc] - yy[zc + 1])
    tz = (zc + frac) / fs
    f_est = (len(tz) - 1) / (2 * (tz[-1] - tz[0]))
    assert abs(f_est - f0 * (1 - v / c)) < 1e-3 * f0 * v / c + 1e-6 * f0


@pytest.mark.parametrize("window", [0, 1])
def test_static_source_is_lti_convolution(window):
    # With a motionless source the moving-image sum must reduce to the static
    # image-source RIR of Eq. 1 (each image a windowed-sinc fractional delay
    # with gain beta_i / (4 pi d_i)) convolved with the signal. The RIR is
    # built here from brute-force mirrored images, numpy's sinc, numpy/scipy
    # windows and numpy's convolution.
    L, fs, c = 32, 16000.0, 343.0
    src = np.array([1.3, 1.1, 1.4])
    sc = _scene(K=3, window=window, taps=L, kaiser_beta=8.0,
                traj_kind=0, traj=list(src) + [1.0, 0.5, 0.2, 0.0])
    x = np.random.default_rng(7).standard_normal(3000)
    y = oracle.synthesize(sc, x)
    dims, mic = sc.dims, np.array(sc.mic)
    h = np.zeros(2000)
    for sign, off, hits in brute.mirror_images(dims, 2 * sc.K + 3):
        n_lat, _ = brute.lattice_of(sign, off, dims)
        if sum(abs(v) for v in n_lat) > sc.K:
            continue
        d = np.linalg.norm(np.array(sign) * src + np.array(off) - mic)
        tau = d * fs / c
        gain = np.prod([sc.beta[w] ** hits[w] for w in range(6)]) / (4 * np.pi * d)
        p = np.arange(int(np.floor(tau - L / 2)) - 1, int(np.ceil(tau + L / 2)) + 2)
        u = p - tau
        inside = (u >= -L / 2) & (u < L / 2)
        if window == 0:
            wv = 0.5 * (1 + np.cos(2 * np.pi * u / L))
        else:
            wv = scipy_i0(8.0 * np.sqrt(np.clip(1 - (2 * u / L) ** 2, 0, None))) / scipy_i0(8.0)
        h[p[inside]] += gain * wv[inside] * np.sinc(u[inside])
    ref = np.convolve(x, h)[: x.size]
    assert rel_l2(y, ref) < 1e-12


# ----------------------------------------------------------------- invariants
def _moving_small(window=0, taps=32, K=2):
    spec = W.small_scene(seed=3, K=K, seconds=0.02, window=window, taps=taps)
    return spec, oracle_scene(spec)


def test_image_order_and_subsets():
    spec, sc = _moving_small()
    x = spec.x.astype(np.float64)
    idx = np.arange(0, x.size, 7)
    n_img = oracle.image_count(sc.K)
    all_imgs = np.arange(n_img)
    y = oracle.y_at(sc, x, idx)
    y_rev = oracle.y_at(sc, x, idx, images=all_imgs[::-1])
    assert rel_l2(y_rev, y) < 1e-13
    perm = np.random.default_rng(0).permutation(n_img)
    a, b = perm[: n_img // 3], perm[n_img // 3:]
    assert rel_l2(oracle.y_at(sc, x, idx, images=a) + oracle.y_at(sc, x, idx, images=b), y) < 1e-13
    assert rel_l2(oracle.synthesize(sc, x)[idx], y) < 1e-15


def test_linearity_in_signal():
    spec, sc = _moving_small()
    rng = np.random.default_rng(5)
    x1, x2 = rng.standard_normal(spec.n_in), rng.standard_normal(spec.n_in)
    y = oracle.synthesize(sc, 0.3 * x1 - 2.0 * x2)
    assert rel_l2(y, 0.3 * oracle.synthesize(sc, x1) - 2.0 * oracle.synthesize(sc, x2)) < 1e-13


@pytest.mark.parametrize("window,taps,traj", [(0, 8, W.SPLINE), (1, 8, W.CIRCLE), (0, 32, W.LINE)])
def test_brute_force_tiny_room(window, taps, traj):
    spec = W.small_scene(seed=11, K=2, seconds=128 / 16000.0, window=window, taps=taps,
                         traj_kind=traj, tiers=[(1, 16000.0), (W.RHO_INF, 2000.0)])
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    y = oracle.synthesize(sc, x)
    yb = np.array(brute.synthesize(spec, list(x), x.size))
    assert rel_l2(y, yb) < 1e-12


# ----------------------------------------------------------------- gradients
def test_adjoint_x_is_transpose():
    spec, sc = _moving_small()
    rng = np.random.default_rng(9)
    x = rng.standard_normal(spec.n_in)
    v = rng.standard_normal(spec.n_in)
    lhs = np.dot(oracle.synthesize(sc, x), v)
    rhs = np.dot(x, oracle.adjoint_x(sc, v, spec.n_in))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    dx = oracle.adjoint_x(sc, v, spec.n_in)
    for m in (0, 57, spec.n_in - 1):
        e = np.zeros(spec.n_in)
        e[m] = 1.0
        assert abs(dx[m] - np.dot(v, oracle.synthesize(sc, e))) < 1e-13


def test_complex_step_matches_richardson_fd():
    spec = W.small_scene(seed=4, K=2, seconds=0.03, window=0, taps=32)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    target = np.random.default_rng(1).standard_normal(spec.n_in) * 0.01
    ids = [0, 4, 8, 11, 48, 51]   # three control-point coordinates and two walls
    g_cs = oracle.loss_grad_cs(sc, x, target, ids)

    def loss_at(pid, delta):
        tr = list(sc.traj)
        bt = list(sc.beta)
        if pid < 48:
            tr[pid] += delta
        else:
            bt[pid - 48] += delta
        s2 = oracle.Scene(**{**sc.__dict__, "traj": tr, "beta": bt})
        return oracle.loss(s2, x, target)

    for q, pid in enumerate(ids):
        h = 1e-3 if pid < 48 else 1e-4
        d1 = (loss_at(pid, h) - loss_at(pid, -h)) / (2 * h)
        d2 = (loss_at(pid, h / 2) - loss_at(pid, -h / 2)) / h
        rich = (4 * d2 - d1) / 3
        assert abs(g_cs[q] - rich) <= 1e-5 * max(abs(g_cs[q]), 1e-12), (pid, g_cs[q], rich)
