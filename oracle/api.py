"""ctypes front end of the FP64 CPU oracle (oracle/oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path. It shares no code with
the CUDA library; scenes reach it as plain numbers (see ``Scene``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into oracle/_build/liboracle.so (g++, OpenMP, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = f"{_LIB}.{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_double * 3),
        ("beta", ctypes.c_double * 6),
        ("c", ctypes.c_double),
        ("fs", ctypes.c_double),
        ("kaiser_beta", ctypes.c_double),
        ("traj", ctypes.c_double * 48),
        ("duration", ctypes.c_double),
        ("mic", ctypes.c_double * 3),
        ("K", ctypes.c_int32),
        ("n_tiers", ctypes.c_int32),
        ("tier_max_rho", ctypes.c_int32 * 4),
        ("tier_step", ctypes.c_int32 * 4),
        ("taps", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("traj_kind", ctypes.c_int32),
        ("n_ctrl", ctypes.c_int32),
        ("farrow_order", ctypes.c_int32),
        ("farrow", ctypes.POINTER(ctypes.c_double)),
        ("arr_kind", ctypes.c_int32),
        ("arr_n_ctrl", ctypes.c_int32),
        ("arr_traj", ctypes.c_double * 48),
        ("arr_duration", ctypes.c_double),
        ("tier_up", ctypes.c_int32 * 4),
        ("up_halfwidth", ctypes.c_int32),
        ("delay_model", ctypes.c_int32),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_S = ctypes.POINTER(_Scene)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            L = ctypes.c_long
            lib.oracle_image_count.argtypes = [ctypes.c_int32]
            lib.oracle_image_count.restype = L
            lib.oracle_enumerate.argtypes = [_S, _I32, _I32, _I32, _I32, _I32, _D]
            lib.oracle_source_position.argtypes = [_S, _D, L, _D]
            lib.oracle_image_distance.argtypes = [_S, L, _D, L, _D]
            lib.oracle_knot_delay.argtypes = [_S, L, _D, L, _D]
            lib.oracle_knot_delay_cs.argtypes = [_S, L, _D, L, ctypes.c_int32, ctypes.c_double, _D]
            lib.oracle_delay_gain.argtypes = [_S, L, _I64, L, _D, _D, _D]
            lib.oracle_tap_weights.argtypes = [_S, _D, L, _D]
            lib.oracle_window.argtypes = [_S, _D, L, _D]
            lib.oracle_y_at.argtypes = [_S, _D, L, _I64, L, _I32, L, _D]
            lib.oracle_synthesize.argtypes = [_S, _D, L, L, _D]
            lib.oracle_adjoint_x.argtypes = [_S, _D, L, L, _D]
            lib.oracle_synthesize_envelope.argtypes = [_S, _D, L, L, ctypes.c_double, _D, _D]
            lib.oracle_adjoint_x_envelope.argtypes = [_S, _D, L, L, ctypes.c_double, _D, _D]
            lib.oracle_loss.argtypes = [_S, _D, L, L, _D]
            lib.oracle_loss.restype = ctypes.c_double
            lib.oracle_loss_grad_cs.argtypes = [_S, _D, L, L, _D, _I32, L, ctypes.c_double, _D]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Scene:
    """One scene and one microphone, as plain numbers.

    traj_kind: 0 line (traj = p0[3], direction[3], speed), 1 circle
    (traj = centre[3], radius, speed, start angle), 2 clamped cubic B-spline
    (traj = control points, 3 per point; n_ctrl points; u = clamp(t/duration)).
    window: 0 Hann, 1 Kaiser(kaiser_beta), 2 a Farrow polynomial per tap with
    coefficients `farrow` (taps x (order + 1), e.g. from oracle.gls.design).
    arr_kind: -1 static microphone; else the microphone moves as
    mic + a(t) - a(0) with a(t) a trajectory of that kind (arr_traj,
    arr_n_ctrl, arr_duration as for the source).
    tiers: list of (max_rho, knot_step_samples[, upsample]); an image goes to
    the first tier whose max_rho >= its reflection count, else to the last
    tier. upsample U > 1 (dividing the step) interpolates the knots' distances
    band-limited to U virtual knots per interval (Kaiser(8)-windowed sinc over
    2 up_halfwidth knots, normalised), then linearly.
    delay_model: 0 the knot distance is taken at the reception time; 1 it is
    the emission-time (retarded) path length c tau, c tau = |r_i(t - tau) - m(t)|.
    """

    dims: Sequence[float]
    beta: Sequence[float]
    mic: Sequence[float]
    K: int
    fs: float
    c: float = 343.0
    tiers: Sequence[tuple] = ((1, 1), (10**9, 16))
    taps: int = 32
    window: int = 0
    kaiser_beta: float = 8.0
    traj_kind: int = 0
    traj: Sequence[float] = field(default_factory=list)
    n_ctrl: int = 0
    duration: float = 1.0
    farrow: Optional[np.ndarray] = None
    arr_kind: int = -1
    arr_traj: Sequence[float] = field(default_factory=list)
    arr_n_ctrl: int = 0
    arr_duration: float = 1.0
    up_halfwidth: int = 4
    delay_model: int = 0

    def to_c(self) -> _Scene:
        s = _Scene()
        s.dims[:] = [float(v) for v in self.dims]
        s.beta[:] = [float(v) for v in self.beta]
        s.c = float(self.c)
        s.fs = float(self.fs)
        s.kaiser_beta = float(self.kaiser_beta)
        tr = [0.0] * 48
        tr[: len(self.traj)] = [float(v) for v in self.traj]
        s.traj[:] = tr
        s.duration = float(self.duration)
        s.mic[:] = [float(v) for v in self.mic]
        s.K = int(self.K)
        s.n_tiers = len(self.tiers)
        rho = [0] * 4
        step = [1] * 4
        up = [1] * 4
        for t, tier in enumerate(self.tiers):
            rho[t] = int(min(tier[0], 2**31 - 1))
            step[t] = int(tier[1])
            up[t] = int(tier[2]) if len(tier) > 2 else 1
            if up[t] > 1 and step[t] % up[t]:
                raise ValueError("upsampling factor must divide the knot step")
        s.tier_max_rho[:] = rho
        s.tier_step[:] = step
        s.tier_up[:] = up
        s.up_halfwidth = int(self.up_halfwidth)
        s.delay_model = int(self.delay_model)
        s.taps = int(self.taps)
        s.window = int(self.window)
        s.traj_kind = int(self.traj_kind)
        s.n_ctrl = int(self.n_ctrl)
        s.arr_kind = int(self.arr_kind)
        s.arr_n_ctrl = int(self.arr_n_ctrl)
        at = [0.0] * 48
        at[: len(self.arr_traj)] = [float(v) for v in self.arr_traj]
        s.arr_traj[:] = at
        s.arr_duration = float(self.arr_duration)
        if self.window == 2:
            c = np.ascontiguousarray(self.farrow, dtype=np.float64)
            if c.ndim != 2 or c.shape[0] != self.taps:
                raise ValueError("farrow must be taps x (order + 1)")
            s.farrow_order = c.shape[1] - 1
            s.farrow = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            s._keep = c  # the table must outlive the call
        return s


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def image_count(K: int) -> int:
    return int(_load().oracle_image_count(K))


def enumerate_images(scene: Scene) -> dict:
    lib = _load()
    cnt = image_count(scene.K)
    n = np.zeros((cnt, 3), np.int32)
    p = np.zeros((cnt, 3), np.int32)
    e = np.zeros((cnt, 6), np.int32)
    rho = np.zeros(cnt, np.int32)
    tier = np.zeros(cnt, np.int32)
    beta = np.zeros(cnt, np.float64)
    sc = scene.to_c()
    lib.oracle_enumerate(ctypes.byref(sc), n.ctypes.data_as(_I32), p.ctypes.data_as(_I32),
                         e.ctypes.data_as(_I32), rho.ctypes.data_as(_I32),
                         tier.ctypes.data_as(_I32), _dp(beta))
    return dict(n=n, p=p, e=e, rho=rho, tier=tier, beta=beta)


def source_position(scene: Scene, t) -> np.ndarray:
    t = np.ascontiguousarray(np.atleast_1d(t), np.float64)
    out = np.zeros((t.size, 3))
    sc = scene.to_c()
    _load().oracle_source_position(ctypes.byref(sc), _dp(t), t.size, _dp(out))
    return out


def image_distance(scene: Scene, idx: int, t) -> np.ndarray:
    t = np.ascontiguousarray(np.atleast_1d(t), np.float64)
    out = np.zeros(t.size)
    sc = scene.to_c()
    _load().oracle_image_distance(ctypes.byref(sc), int(idx), _dp(t), t.size, _dp(out))
    return out


def knot_delay(scene: Scene, idx: int, t) -> np.ndarray:
    """Delay (s) of image idx at times t under the scene's delay model."""
    t = np.ascontiguousarray(np.atleast_1d(t), np.float64)
    out = np.zeros(t.size)
    sc = scene.to_c()
    _load().oracle_knot_delay(ctypes.byref(sc), int(idx), _dp(t), t.size, _dp(out))
    return out


def knot_delay_cs(scene: Scene, idx: int, t, param_id: int, h: float = 1e-20) -> np.ndarray:
    """Complex-step derivative of knot_delay (s) with respect to one parameter
    (ids < 48 index traj[], 48..53 the wall reflection coefficients, 54..101
    the array trajectory's arr_traj[])."""
    t = np.ascontiguousarray(np.atleast_1d(t), np.float64)
    out = np.zeros(t.size)
    sc = scene.to_c()
    _load().oracle_knot_delay_cs(ctypes.byref(sc), int(idx), _dp(t), t.size, int(param_id), float(h), _dp(out))
    return out


def delay_gain(scene: Scene, idx: int, n) -> tuple:
    n = np.ascontiguousarray(np.atleast_1d(n), np.int64)
    tau, g, d = np.zeros(n.size), np.zeros(n.size), np.zeros(n.size)
    sc = scene.to_c()
    _load().oracle_delay_gain(ctypes.byref(sc), int(idx), n.ctypes.data_as(_I64), n.size,
                              _dp(tau), _dp(g), _dp(d))
    return tau, g, d


def tap_weights(scene: Scene, alpha) -> np.ndarray:
    a = np.ascontiguousarray(np.atleast_1d(alpha), np.float64)
    out = np.zeros((a.size, scene.taps))
    sc = scene.to_c()
    _load().oracle_tap_weights(ctypes.byref(sc), _dp(a), a.size, _dp(out))
    return out


def window(scene: Scene, u) -> np.ndarray:
    u = np.ascontiguousarray(np.atleast_1d(u), np.float64)
    out = np.zeros(u.size)
    sc = scene.to_c()
    _load().oracle_window(ctypes.byref(sc), _dp(u), u.size, _dp(out))
    return out


def y_at(scene: Scene, x: np.ndarray, idx, images: Optional[np.ndarray] = None) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    idx = np.ascontiguousarray(np.atleast_1d(idx), np.int64)
    y = np.zeros(idx.size)
    sc = scene.to_c()
    if images is None:
        il, nil = None, 0
    else:
        images = np.ascontiguousarray(images, np.int32)
        il, nil = images.ctypes.data_as(_I32), images.size
    _load().oracle_y_at(ctypes.byref(sc), _dp(x), x.size, idx.ctypes.data_as(_I64), idx.size,
                        il, nil, _dp(y))
    return y


def synthesize(scene: Scene, x: np.ndarray, n_out: Optional[int] = None) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    n_out = x.size if n_out is None else int(n_out)
    y = np.zeros(n_out)
    sc = scene.to_c()
    _load().oracle_synthesize(ctypes.byref(sc), _dp(x), x.size, n_out, _dp(y))
    return y


def synthesize_envelope(scene: Scene, x: np.ndarray, n_out: Optional[int] = None, delta: float = 1e-4):
    """(y, env): y as synthesize(); env[n] sums, over the image-samples of
    output n whose read position n - tau lies within `delta` samples of an
    integer, |A_i(n)| times the difference between evaluating the taps on
    either side of that integer ((m0, alpha) or (m0 -+ 1, alpha +- 1)). Where
    the tap kernel jumps at the wrap (a low-order Farrow polynomial), the side
    is decided by the precision of the delay, and any result within y +- env
    is an evaluation of the method."""
    x = np.ascontiguousarray(x, np.float64)
    n_out = x.size if n_out is None else int(n_out)
    y, env = np.zeros(n_out), np.zeros(n_out)
    sc = scene.to_c()
    _load().oracle_synthesize_envelope(ctypes.byref(sc), _dp(x), x.size, n_out, float(delta), _dp(y), _dp(env))
    return y, env


def adjoint_x_envelope(scene: Scene, dy: np.ndarray, n_in: int, delta: float = 1e-4):
    """(dx, env): dx as adjoint_x(); env[m] bounds the change of dx[m] when the
    image-samples near the wrap (as in synthesize_envelope) take the other side."""
    dy = np.ascontiguousarray(dy, np.float64)
    dx, env = np.zeros(int(n_in)), np.zeros(int(n_in))
    sc = scene.to_c()
    _load().oracle_adjoint_x_envelope(ctypes.byref(sc), _dp(dy), dy.size, int(n_in), float(delta), _dp(dx),
                                      _dp(env))
    return dx, env


def adjoint_x(scene: Scene, dy: np.ndarray, n_in: int) -> np.ndarray:
    dy = np.ascontiguousarray(dy, np.float64)
    dx = np.zeros(int(n_in))
    sc = scene.to_c()
    _load().oracle_adjoint_x(ctypes.byref(sc), _dp(dy), dy.size, int(n_in), _dp(dx))
    return dx


def loss(scene: Scene, x: np.ndarray, target: np.ndarray) -> float:
    x = np.ascontiguousarray(x, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    sc = scene.to_c()
    return float(_load().oracle_loss(ctypes.byref(sc), _dp(x), x.size, target.size, _dp(target)))


def loss_grad_cs(scene: Scene, x: np.ndarray, target: np.ndarray, param_ids, h: float = 1e-20) -> np.ndarray:
    """Complex-step gradient of 0.5*||y - target||^2; ids < 48 index traj[],
    48..53 index the wall reflection coefficients, 54..101 the array
    trajectory's arr_traj[]."""
    x = np.ascontiguousarray(x, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    ids = np.ascontiguousarray(np.atleast_1d(param_ids), np.int32)
    g = np.zeros(ids.size)
    sc = scene.to_c()
    _load().oracle_loss_grad_cs(ctypes.byref(sc), _dp(x), x.size, target.size, _dp(target),
                                ids.ctypes.data_as(_I32), ids.size, float(h), _dp(g))
    return g


def num_threads() -> int:
    return int(_load().oracle_num_threads())
