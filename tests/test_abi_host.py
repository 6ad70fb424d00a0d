"""The C ABI library without a GPU: it loads, exports every symbol declared in
include/msrc.h, and its host-side logic (validation, Farrow fit, image counts,
tier plan) behaves. No call here touches a device."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import api as oracle
from paper_2508_03065_gb300 import _lib
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "msrc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msrc_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def _desc(**kw):
    d = _lib.RoomDesc()
    d.dims[:] = kw.get("dims", [5.0, 4.0, 3.0])
    d.beta[:] = kw.get("beta", [0.7] * 6)
    d.c = kw.get("c", 343.0)
    d.fs = kw.get("fs", 16000.0)
    d.max_order = kw.get("K", 3)
    tiers = kw.get("tiers", [(1, 16000.0), (2**31 - 1, 1000.0)])
    d.n_tiers = len(tiers)
    rho = [0] * 4
    rate = [1.0] * 4
    up = [0] * 4
    for t, tier in enumerate(tiers):
        rho[t], rate[t] = tier[0], tier[1]
        up[t] = tier[2] if len(tier) > 2 else 0
    d.tier_max_rho[:] = rho
    d.tier_rate_hz[:] = rate
    d.tier_upsample[:] = up
    d.upsample_halfwidth = kw.get("upsample_halfwidth", 0)
    d.delay_model = kw.get("delay_model", 0)
    d.taps = kw.get("taps", 32)
    d.window = kw.get("window", 0)
    d.kaiser_beta = kw.get("kaiser_beta", 8.0)
    d.farrow_order = kw.get("farrow_order", 4)
    d.passband = kw.get("passband", 0.9)
    return d


def _create(**kw):
    lib = _lib.load()
    h = ctypes.c_void_p()
    st = lib.msrc_create_room(ctypes.byref(_desc(**kw)), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("bad", [
    dict(dims=[0.0, 4.0, 3.0]), dict(beta=[1.2] + [0.7] * 5), dict(c=-1.0), dict(fs=0.0),
    dict(K=61), dict(K=-1), dict(taps=31), dict(taps=4), dict(taps=66), dict(window=3),
    dict(tiers=[(1, 16000.0), (2**31 - 1, 700.0)]), dict(tiers=[]),
    dict(window=1, kaiser_beta=-1.0), dict(window=2, farrow_order=0), dict(window=2, farrow_order=5),
    dict(window=2, passband=0.01), dict(window=2, passband=0.99),
    dict(tiers=[(1, 16000.0), (2**31 - 1, 1000.0, 7)]), dict(tiers=[(2**31 - 1, 25.0, 1280)]),
    dict(tiers=[(2**31 - 1, 1000.0, -1)]), dict(upsample_halfwidth=9), dict(upsample_halfwidth=-1),
    dict(delay_model=2), dict(delay_model=-1)])
def test_create_room_rejects_bad_descriptions(bad):
    st, h = _create(**bad)
    assert st == _lib.ERR_INVALID_ARG
    assert not h.value
    assert len(_lib.load().msrc_last_error()) > 0


def test_null_arguments_are_errors_not_crashes():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.msrc_create_room(None, ctypes.byref(h)) == _lib.ERR_INVALID_ARG
    assert lib.msrc_set_trajectory(None, None, None, 1) == _lib.ERR_INVALID_ARG
    assert lib.msrc_workspace_size(None, 1, None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.msrc_synthesize(None, 1, None, None, None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.msrc_destroy_room(None) == _lib.OK
    assert lib.msrc_status_string(_lib.ERR_WORKSPACE) == b"workspace too small or misaligned"


def _traj(kind=0, params=(1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 1.0), duration=1.0, n_ctrl=0):
    t = _lib.TrajDesc()
    t.kind, t.n_ctrl, t.duration_s = kind, n_ctrl, duration
    p = [0.0] * 48
    p[: len(params)] = params
    t.params[:] = p
    return t


def _mics(*pts):
    a = np.ascontiguousarray(np.array(pts, np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("traj,mic,why", [
    (_traj(params=(1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 5.0)), (2.5, 2.0, 1.2), "leaves the room"),
    (_traj(params=(1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 1.0)), (6.0, 2.0, 1.2), "mic outside"),
    (_traj(params=(1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 1.0)), (1.5, 1.3, 1.5), "passes the mic"),
    (_traj(kind=1, params=(2.5, 2.0, 1.5, 1.0, 400.0, 0.0)), (2.5, 2.0, 1.2), "faster than c"),
    (_traj(kind=2, params=(1,) * 9, n_ctrl=3), (2.5, 2.0, 1.2), "too few control points"),
    (_traj(kind=7), (2.5, 2.0, 1.2), "unknown kind"),
    (_traj(duration=0.0), (2.5, 2.0, 1.2), "zero duration"),
])
def test_set_trajectory_rejects_invalid_geometry(traj, mic, why):
    lib = _lib.load()
    st, h = _create()
    assert st == _lib.OK
    arr, p = _mics(mic)
    assert lib.msrc_set_trajectory(h, ctypes.byref(traj), p, 1) == _lib.ERR_INVALID_ARG, why
    # a failed call leaves the room without a trajectory
    sz = ctypes.c_size_t()
    n = _lib.i64_array([16000])
    assert lib.msrc_workspace_size(_lib.ptr_array([h.value]), 1, n, n, ctypes.byref(sz), None) == _lib.ERR_STATE
    lib.msrc_destroy_room(h)


def test_workspace_and_signal_checks_without_device():
    lib = _lib.load()
    st, h = _create()
    arr, p = _mics((2.5, 2.0, 1.2))
    assert lib.msrc_set_trajectory(h, ctypes.byref(_traj()), p, 1) == _lib.OK
    hs = _lib.ptr_array([h.value])
    n = _lib.i64_array([16000])
    fwd = ctypes.c_size_t()
    assert lib.msrc_workspace_size(hs, 1, n, n, ctypes.byref(fwd), None) == _lib.OK
    assert fwd.value > 16000 * 4
    # too-small or misaligned workspace, bad lengths: rejected before any device call
    xs = _lib.ptr_array([1024])
    ys = _lib.ptr_array([4096])
    assert lib.msrc_synthesize(hs, 1, xs, n, ys, n, ctypes.c_void_p(256), 1024, None) == _lib.ERR_WORKSPACE
    assert lib.msrc_synthesize(hs, 1, xs, n, ys, n, ctypes.c_void_p(257), fwd.value, None) == _lib.ERR_WORKSPACE
    zero = _lib.i64_array([0])
    assert lib.msrc_synthesize(hs, 1, xs, zero, ys, n, ctypes.c_void_p(256), fwd.value, None) == _lib.ERR_INVALID_ARG
    # per-call tile configurations: the default's size, each configuration's
    # own size, and ids out of range refused
    fcfg = ctypes.c_size_t()
    assert lib.msrc_workspace_size_cfg(hs, 1, n, n, _lib.TILE_DEFAULT, ctypes.byref(fcfg), None) == _lib.OK
    assert fcfg.value == fwd.value
    sizes = []
    for c in range(lib.msrc_tile_configs()):
        assert lib.msrc_workspace_size_cfg(hs, 1, n, n, c, ctypes.byref(fcfg), None) == _lib.OK
        sizes.append(fcfg.value)
    assert fwd.value in sizes and len(set(sizes)) > 1  # the default is one of them (chosen automatically)
    assert lib.msrc_workspace_size_cfg(hs, 1, n, n, _lib.TILE_AUTO, ctypes.byref(fcfg), None) == _lib.OK
    assert fcfg.value == fwd.value
    for bad in (lib.msrc_tile_configs(), 99):
        assert lib.msrc_workspace_size_cfg(hs, 1, n, n, bad, ctypes.byref(fcfg), None) == _lib.ERR_INVALID_ARG
        assert lib.msrc_synthesize_cfg(hs, 1, xs, n, ys, n, bad, ctypes.c_void_p(256), 1 << 30,
                                       None) == _lib.ERR_INVALID_ARG
    lib.msrc_destroy_room(h)


@pytest.mark.parametrize("K,tiers", [(3, [(1, 16000.0), (2**31 - 1, 1000.0)]),
                                     (6, [(2, 16000.0), (8, 4000.0), (2**31 - 1, 500.0)])])
def test_image_counts_per_tier_match_oracle(K, tiers):
    lib = _lib.load()
    st, h = _create(K=K, tiers=tiers)
    assert st == _lib.OK
    cnt = ctypes.c_int64()
    per = (ctypes.c_int64 * 4)()
    assert lib.msrc_room_image_count(h, ctypes.byref(cnt), per) == _lib.OK
    sc = oracle.Scene(dims=(5.0, 4.0, 3.0), beta=(0.7,) * 6, mic=(2.5, 2.0, 1.2), K=K, fs=16000.0,
                      tiers=[(r, 1) for r, _ in tiers])
    tab = oracle.enumerate_images(sc)
    assert cnt.value == W.image_count(K) == tab["tier"].size
    for t in range(len(tiers)):
        assert per[t] == int(np.sum(tab["tier"] == t))
    lib.msrc_destroy_room(h)


@pytest.mark.parametrize("taps,window", [(8, 0), (32, 0), (32, 1), (64, 1), (24, 1)])
def test_farrow_fit_is_accurate(taps, window):
    lib = _lib.load()
    st, h = _create(taps=taps, window=window)
    assert st == _lib.OK
    e = ctypes.c_double()
    assert lib.msrc_room_fit_error(h, ctypes.byref(e)) == _lib.OK
    # worst polynomial error per tap (4 segments x degree 4, Chebyshev nodes,
    # float coefficients): 0.8e-6 for L >= 16, up to 1.4e-6 for L = 8. The
    # output error is ~3e-7 relative (errors of different taps do not align),
    # well inside the 1e-5 budget
    assert e.value < (2e-6 if taps < 16 else 1e-6)
    lib.msrc_destroy_room(h)


@pytest.mark.parametrize("taps,order,passband", [(8, 1, 0.5), (16, 3, 0.8), (32, 4, 0.9), (64, 2, 0.95)])
def test_least_squares_design_is_held_exactly(taps, order, passband):
    # a least-squares Farrow design of order <= 4 is itself a polynomial of
    # degree <= 4 on every segment: the device table holds it up to float
    # rounding
    lib = _lib.load()
    st, h = _create(taps=taps, window=2, farrow_order=order, passband=passband)
    assert st == _lib.OK
    e = ctypes.c_double()
    assert lib.msrc_room_fit_error(h, ctypes.byref(e)) == _lib.OK
    assert e.value < 1e-7
    lib.msrc_destroy_room(h)


def test_knot_spacing_from_paper_rates():
    # Sec. III: spatio-temporal rate equal to the 16 kHz audio rate, downsampled
    # by 3200 (a 5 Hz knot rate); tiers/rates must divide the audio rate.
    with open(os.path.join(ROOT, "tests", "golden", "paper_rates.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for fs, ratio in rows:
        fs, ratio = float(fs), int(ratio)
        st, h = _create(fs=fs, tiers=[(1, fs), (2**31 - 1, fs / ratio)])
        assert st == _lib.OK
        _lib.load().msrc_destroy_room(h)
    st, _ = _create(fs=16000.0, tiers=[(1, 16000.0), (2**31 - 1, 16000.0 / 3200.5)])
    assert st == _lib.ERR_INVALID_ARG


def test_array_trajectory_validation():
    # microphones carried out of the room, onto the source, or faster than
    # sound are refused and leave the room unchanged; None makes it static
    from paper_2508_03065_gb300 import api
    spec = W.small_scene(seed=5, K=2, seconds=0.25)
    room = api.Room.from_spec(spec)
    with pytest.raises(RuntimeError):
        room.set_array_trajectory(W.LINE, [0, 0, 0, 1.0, 0.0, 0.0, 40.0], spec.duration)
    with pytest.raises(RuntimeError):
        room.set_array_trajectory(W.LINE, [0, 0, 0, 1.0, 0.0, 0.0, 400.0], spec.duration)
    room.set_array_trajectory(W.CIRCLE, [0, 0, 0, 0.1, 0.3, 0.0], spec.duration)
    room.set_array_trajectory(None)



def test_band_limited_upsampling_planning():
    """Band-limited tiers plan forward and reverse-mode calls (the reverse
    mode adds the per-(mic, image, record knot) delay and gradient tables), and
    check the path's extension before t = 0 that their knots reach."""
    lib = _lib.load()
    n = _lib.i64_array([16000])
    arr, p = _mics((2.5, 2.0, 1.2))
    sizes, bsizes = [], []
    for tiers in ([(1, 16000.0), (2**31 - 1, 5.0)], [(1, 16000.0), (2**31 - 1, 5.0, 100)]):
        st, h = _create(tiers=tiers)
        assert st == _lib.OK
        assert lib.msrc_set_trajectory(h, ctypes.byref(_traj()), p, 1) == _lib.OK
        hs = _lib.ptr_array([h.value])
        fwd, bwd = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.msrc_workspace_size(hs, 1, n, n, ctypes.byref(fwd), None) == _lib.OK
        sizes.append(fwd.value)
        assert lib.msrc_workspace_size(hs, 1, n, n, None, ctypes.byref(bwd)) == _lib.OK
        bsizes.append(bwd.value)
        lib.msrc_destroy_room(h)
    assert sizes[1] > sizes[0]
    # reverse mode: the upsampled tier's images x 1601 record knots x 2 doubles more
    assert bsizes[1] > bsizes[0]
    # 2 m/s along (3, 2, 0) from x = 1 m: inside the room on [0, 1] s, but the
    # 5 Hz tier's kernel reaches 4 knots (0.8 s) before t = 0, where x < 0
    fast = _traj(params=(1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 2.0))
    for U, want in ((0, _lib.OK), (100, _lib.ERR_INVALID_ARG)):
        st, h = _create(tiers=[(1, 16000.0), (2**31 - 1, 5.0, U)])
        assert lib.msrc_set_trajectory(h, ctypes.byref(fast), p, 1) == _lib.OK
        fwd = ctypes.c_size_t()
        assert lib.msrc_workspace_size(_lib.ptr_array([h.value]), 1, n, n, ctypes.byref(fwd), None) == want
        lib.msrc_destroy_room(h)


def test_host_only_hooks_validate_arguments():
    # the bounded-wait test hook takes multiples of 16 bytes and 0 (off); the
    # peak measurement refuses null pointers before touching a device
    lib = _lib.load()
    assert lib.msrc_test_stall_window_copies(3) == _lib.ERR_INVALID_ARG
    assert lib.msrc_test_stall_window_copies(0) == _lib.OK
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    assert lib.msrc_measure_alu_peaks(None, None, ctypes.byref(f32), ctypes.byref(f64)) == _lib.ERR_INVALID_ARG


# Largest per-tap error of the device's Farrow table against the exact windowed
# sinc (the oracle's tap weights) on a 1e5-point grid of fractional delays.
# The synthesis table (4 segments x degree 4, Chebyshev nodes, float
# coefficients) measures 0.80-0.91e-6 for L >= 16 and 1.1-1.4e-6 for L = 8;
# the gradient kernel's degree-5 table 3e-8 to 7.4e-8. For one image and a
# white signal the tap errors move the output by sqrt(sum_k dh_k^2) relative to
# sqrt(sum_k h_k^2): at most 1.8e-6 (L >= 16) and 2.5e-6 (L = 8) at the worst
# delay, and they oscillate in alpha and differ per tap, so summed over images
# they stay near 3e-7 of the output: inside the 1e-5 parity bar.
FARROW_PIN = {0: {8: 1.5e-6, "other": 1.0e-6}, 1: {8: 1e-7, "other": 1e-7}}


@pytest.mark.parametrize("taps,window,beta", [(8, 0, 8.0), (16, 1, 8.0), (24, 1, 8.0), (32, 0, 8.0), (32, 1, 8.0),
                                              (64, 1, 8.0), (32, 1, 4.0)])
def test_device_farrow_table_against_oracle_taps(taps, window, beta):
    lib = _lib.load()
    st, h = _create(taps=taps, window=window, kaiser_beta=beta)
    assert st == _lib.OK
    alpha = (np.arange(100000) + 0.5) / 100000.0
    sc = oracle.Scene(dims=(5.0, 4.0, 3.0), beta=(0.7,) * 6, mic=(2.5, 2.0, 1.2), K=0, fs=16000.0,
                      tiers=[(2**31 - 1, 1)], taps=taps, window=window, kaiser_beta=beta)
    exact = oracle.tap_weights(sc, alpha)  # (alpha, k + L/2)
    seg = np.floor(4.0 * alpha).astype(int)
    w = 4.0 * alpha - seg - 0.5
    for which in (0, 1):
        out = np.zeros(4 * 6 * taps, np.float32)
        P = ctypes.c_int32()
        assert lib.msrc_room_farrow_table(h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          ctypes.byref(P)) == _lib.OK
        assert P.value == (5 if which == 0 else 6)
        tab = out[:4 * P.value * taps].reshape(4, P.value, taps).astype(np.float64)
        approx = np.zeros_like(exact)
        for q in range(P.value - 1, -1, -1):  # Horner in w, per alpha's segment
            approx = approx * w[:, None] + tab[seg, q, :]
        err = float(np.max(np.abs(approx - exact)))
        pin = FARROW_PIN[which][8 if taps == 8 else "other"]
        assert err < pin, (which, err)
        # the table is the fit of this room's kernel: a plausible mistake (a
        # segment or a tap shifted by one) is far outside the pin
        assert np.max(np.abs(approx[:, :-1] - exact[:, 1:])) > 100 * pin
    lib.msrc_destroy_room(h)


@pytest.mark.parametrize("tiers,expect", [([(1, 16000.0), (2**31 - 1, 1000.0)], 14),   # most images on 16-sample knots
                                          ([(1, 16000.0), (2**31 - 1, 250.0)], 11)])   # sparse knots
def test_automatic_tile_configuration(tiers, expect):
    # the default configuration follows the knot layout of the call's images
    lib = _lib.load()
    st, h = _create(K=6, tiers=tiers)
    assert st == _lib.OK
    arr, p = _mics((2.5, 2.0, 1.2))
    assert lib.msrc_set_trajectory(h, ctypes.byref(_traj()), p, 1) == _lib.OK
    hs = _lib.ptr_array([h.value])
    n = _lib.i64_array([16000])
    auto, want = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.msrc_workspace_size(hs, 1, n, n, ctypes.byref(auto), None) == _lib.OK
    assert lib.msrc_workspace_size_cfg(hs, 1, n, n, expect, ctypes.byref(want), None) == _lib.OK
    assert auto.value == want.value
    lib.msrc_destroy_room(h)
