"""Seeded synthetic scenes for tests and benchmarks.

This module only draws random numbers and packs them into scene descriptions
(room, walls, microphones, trajectory parameters, source signal). It holds none
of the synthesis arithmetic: both the CUDA path and the CPU oracle receive the
same plain numbers from here.

The paper evaluates on unnamed speech/noise corpora; these seeded signals stand
in for them (white, pink and AR(10) "speech-like" noise).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Sequence, Tuple

import numpy as np

LINE, CIRCLE, SPLINE = 0, 1, 2
HANN, KAISER, FARROW_LS = 0, 1, 2
RHO_INF = 2**31 - 1


@dataclass
class SceneSpec:
    dims: Tuple[float, float, float]
    beta: Tuple[float, ...]                 # walls x=0, x=Lx, y=0, y=Ly, z=0, z=Lz
    mics: np.ndarray                        # (n_mics, 3)
    K: int                                  # image set |n|_1 <= K
    fs: float
    tiers: Sequence[Tuple]                  # (max reflection count, knot rate in Hz[, upsampling U])
    taps: int = 32
    window: int = HANN
    kaiser_beta: float = 8.0
    farrow_order: int = 4                   # window FARROW_LS: polynomial order
    passband: float = 0.9                   # window FARROW_LS: passband edge / pi
    up_halfwidth: int = 4                   # knot upsampler: kernel half-width (knots)
    delay_model: int = 0                    # 0 distance at reception time, 1 emission-time path length
    arr_kind: int = -1                      # microphone array motion: -1 static, else a
    arr_traj: List[float] = field(default_factory=list)   # trajectory a(t) of the source's kinds;
    arr_n_ctrl: int = 0                     # microphones sit at mics + a(t) - a(0)
    arr_duration: float = 1.0
    c: float = 343.0
    traj_kind: int = LINE
    traj: List[float] = field(default_factory=list)
    n_ctrl: int = 0
    duration: float = 1.0
    x: np.ndarray = None                    # float32 source signal
    n_out: int = 0                          # output length (defaults to len(x))
    name: str = ""

    @property
    def n_in(self) -> int:
        return int(self.x.size)

    def tier_steps(self):
        """(max_rho, knot spacing in samples[, upsampling factor]) per tier."""
        out = []
        for tier in self.tiers:
            step = (tier[0], int(round(self.fs / tier[1])))
            out.append(step + (int(tier[2]),) if len(tier) > 2 else step)
        return out


def image_count(K: int) -> int:
    """|n|_1 <= K lattice triples times 8 parities: 8 (2K+1)(2K^2+2K+3)/3."""
    return 8 * (2 * K + 1) * (2 * K * K + 2 * K + 3) // 3


# ---------------------------------------------------------------- signals
def white(seed: int, n: int, std: float = 0.1) -> np.ndarray:
    return (np.random.default_rng(seed).standard_normal(n) * std).astype(np.float32)


def pink(seed: int, n: int, std: float = 0.1) -> np.ndarray:
    w = np.random.default_rng(seed).standard_normal(n)
    W = np.fft.rfft(w)
    k = np.arange(W.size, dtype=np.float64)
    scale = np.zeros_like(k)
    scale[1:] = 1.0 / np.sqrt(k[1:])
    p = np.fft.irfft(W * scale, n)
    return (p / p.std() * std).astype(np.float32)


def ar10(seed: int, n: int, fs: float, std: float = 0.1) -> np.ndarray:
    """Noise through an all-pole filter with 5 conjugate pole pairs (radius
    0.98) at 500, 1500, 2500, 3500 and 4500 Hz."""
    from scipy.signal import lfilter

    poles = []
    for f in (500.0, 1500.0, 2500.0, 3500.0, 4500.0):
        z = 0.98 * np.exp(2j * np.pi * f / fs)
        poles += [z, np.conj(z)]
    a = np.real(np.poly(poles))
    w = np.random.default_rng(seed).standard_normal(n)
    y = lfilter([1.0], a, w)
    return (y / y.std() * std).astype(np.float32)


def sine(n: int, f0: float, fs: float, amp: float = 1.0) -> np.ndarray:
    return (amp * np.sin(2 * np.pi * f0 * np.arange(n) / fs)).astype(np.float32)


# ---------------------------------------------------------------- trajectories
def random_spline(rng, dims, n_ctrl, duration, vmax, margin=0.5):
    """Control points as a random walk inside the room shrunk by `margin`.
    Steps are bounded so that the B-spline speed bound
    3 * segments * max|P_{i+1}-P_i| / T stays <= vmax."""
    segs = n_ctrl - 3
    step_max = vmax * duration / (3.0 * segs)
    lo = np.array([margin] * 3)
    hi = np.array(dims, dtype=np.float64) - margin
    while True:
        pts = [rng.uniform(lo, hi)]
        ok = True
        for _ in range(n_ctrl - 1):
            for _try in range(100):
                d = rng.standard_normal(3)
                d *= rng.uniform(0.0, 1.0) ** (1 / 3) * step_max / np.linalg.norm(d)
                q = pts[-1] + d
                if np.all(q >= lo) and np.all(q <= hi):
                    break
            else:
                ok = False
                break
            pts.append(q)
        if ok:
            return np.array(pts)


def mic_away_from(rng, dims, ctrl, clearance, margin=0.5):
    """Microphone uniform in the room shrunk by `margin`, at least `clearance`
    from the control points' bounding box (the curve lies inside it)."""
    lo = np.array([margin] * 3)
    hi = np.array(dims, dtype=np.float64) - margin
    bl, bh = ctrl.min(0), ctrl.max(0)
    for _ in range(10000):
        m = rng.uniform(lo, hi)
        gap = np.maximum(np.maximum(bl - m, m - bh), 0.0)
        if np.linalg.norm(gap) >= clearance:
            return m
    return None


# ---------------------------------------------------------------- configurations
def config1() -> SceneSpec:
    """5x4x3 m, beta 0.7, 16 kHz, 1 s white noise, line at 1 m/s, |n|_1 <= 3."""
    return SceneSpec(
        dims=(5.0, 4.0, 3.0), beta=(0.7,) * 6, mics=np.array([[2.5, 2.0, 1.2]]), K=3,
        fs=16000.0, tiers=[(1, 16000.0), (RHO_INF, 1000.0)], taps=32, window=HANN,
        traj_kind=LINE, traj=[1.0, 1.0, 1.5, 3.0, 2.0, 0.0, 1.0], duration=1.0,
        x=white(1, 16000), name="room 5x4x3 m, order 3 (504 images), 16 kHz, 1 s, line 1 m/s")


def config2() -> SceneSpec:
    """10x8x4 m, beta ~ U(0.6,0.9), 48 kHz, 4 s pink noise, circle R=2 m at
    1.5 m/s around the microphone, |n|_1 <= 20 (92 168 images)."""
    rng = np.random.default_rng(2)
    beta = tuple(float(b) for b in rng.uniform(0.6, 0.9, 6))
    fs = 48000.0
    return SceneSpec(
        dims=(10.0, 8.0, 4.0), beta=beta, mics=np.array([[5.0, 4.0, 1.5]]), K=20, fs=fs,
        tiers=[(2, 48000.0), (8, 4000.0), (RHO_INF, 500.0)], taps=32, window=KAISER,
        kaiser_beta=8.0, traj_kind=CIRCLE, traj=[5.0, 4.0, 1.5, 2.0, 1.5, 0.0], duration=4.0,
        x=pink(2, int(4 * fs)),
        name="room 10x8x4 m, order 20 (92168 images), 48 kHz, 4 s pink noise, circle 1.5 m/s")


def config2_upsampled(rate_hz: float = 50.0, U: int = 10) -> SceneSpec:
    """The order-20 scene with its last tier (reflection counts above 8, most
    of the images) on band-limited knots: knots at rate_hz, U virtual knots per
    interval (records every fs / (rate_hz U) samples; 50 Hz x 10 keeps the
    500 Hz record spacing of config2)."""
    base = config2()
    return replace(base, tiers=[(2, 48000.0), (8, 4000.0), (RHO_INF, rate_hz, U)],
                   name=base.name + f", last tier on {rate_hz:g} Hz knots upsampled x{U}")


def config3_scene(s: int) -> SceneSpec:
    """One of the 256 batched scenes (seed 1000+s)."""
    rng = np.random.default_rng(1000 + s)
    dims = tuple(float(v) for v in rng.uniform([3, 3, 2.5], [12, 10, 4]))
    beta = tuple(float(b) for b in rng.uniform(0.5, 0.9, 6))
    K = int(rng.integers(6, 13))
    T = float(rng.uniform(1.0, 8.0))
    fs = 16000.0
    n = int(T * fs)
    while True:
        ctrl = random_spline(rng, dims, 4, T, 2.0)
        mic = mic_away_from(rng, dims, ctrl, 0.5)
        if mic is not None:
            break
    x = (rng.standard_normal(n) * 0.1).astype(np.float32)
    return SceneSpec(
        dims=dims, beta=beta, mics=mic[None, :], K=K, fs=fs,
        tiers=[(1, 16000.0), (RHO_INF, 1000.0)], taps=32, window=HANN,
        traj_kind=SPLINE, traj=list(ctrl.ravel()), n_ctrl=4, duration=n / fs, x=x,
        name=f"batched scene {s}")


def config3(n_scenes: int = 256) -> List[SceneSpec]:
    return [config3_scene(s) for s in range(n_scenes)]


def config4_scene(s: int) -> Tuple[SceneSpec, np.ndarray]:
    """Differentiation scene s (seed 2000+s) and its seeded L2 target."""
    rng = np.random.default_rng(2000 + s)
    dims = (6.0, 5.0, 3.0)
    beta = tuple(float(b) for b in rng.uniform(0.5, 0.9, 6))
    fs = 16000.0
    n = int(2 * fs)
    while True:
        ctrl = random_spline(rng, dims, 6, 2.0, 2.0)
        mic = mic_away_from(rng, dims, ctrl, 0.5)
        if mic is not None:
            break
    x = (rng.standard_normal(n) * 0.1).astype(np.float32)
    target = (rng.standard_normal(n) * 0.01).astype(np.float32)
    spec = SceneSpec(
        dims=dims, beta=beta, mics=mic[None, :], K=8, fs=fs,
        tiers=[(1, 16000.0), (RHO_INF, 1000.0)], taps=32, window=HANN,
        traj_kind=SPLINE, traj=list(ctrl.ravel()), n_ctrl=6, duration=2.0, x=x,
        name=f"differentiation scene {s}")
    return spec, target


def config5() -> SceneSpec:
    """15x12x5 m, beta ~ U(0.85,0.95), 48 kHz, 10 s AR(10) noise, 8-mic UCA
    (radius 5 cm), spline up to 3 m/s, |n|_1 <= 25 (177 208 images), 64 taps."""
    rng = np.random.default_rng(5)
    beta = tuple(float(b) for b in rng.uniform(0.85, 0.95, 6))
    dims = (15.0, 12.0, 5.0)
    fs = 48000.0
    centre = np.array([7.5, 6.0, 1.5])
    ang = 2 * np.pi * np.arange(8) / 8
    mics = centre + 0.05 * np.stack([np.cos(ang), np.sin(ang), np.zeros(8)], 1)
    while True:
        ctrl = random_spline(rng, dims, 6, 10.0, 3.0)
        lo, hi = ctrl.min(0), ctrl.max(0)
        gap = np.maximum(np.maximum(lo - centre, centre - hi), 0.0)
        if np.linalg.norm(gap) >= 1.0:
            break
    return SceneSpec(
        dims=dims, beta=beta, mics=mics, K=25, fs=fs,
        tiers=[(2, 48000.0), (8, 4000.0), (RHO_INF, 250.0)], taps=64, window=KAISER,
        kaiser_beta=8.0, traj_kind=SPLINE, traj=list(ctrl.ravel()), n_ctrl=6, duration=10.0,
        x=ar10(5, int(10 * fs), fs),
        name="room 15x12x5 m, order 25 (177208 images), 48 kHz, 10 s, 8-mic array, 64 taps")


def receding_tone(seconds: float = 1.5, fs: float = 16000.0, f0: float = 1000.0) -> SceneSpec:
    """The setting of the paper's first experiment (Sec. III): a dry 1 kHz tone
    from a source moving slowly along a curve away from the microphone (here
    from 0.4 m to 1.9 m in 1.5 s, about 1 m/s), every image on 5 Hz knots
    (the ratio 3200 at 16 kHz). Room, walls and curve are this suite's choice;
    the paper names none."""
    n = int(seconds * fs)
    x = np.sin(2 * np.pi * f0 * np.arange(n) / fs).astype(np.float32)
    ctrl = [1.9, 2.6, 1.5, 2.4, 2.9, 1.6, 3.0, 2.9, 1.5, 3.4, 2.6, 1.4]
    return SceneSpec(dims=(6.0, 5.0, 3.0), beta=(0.8, 0.7, 0.75, 0.8, 0.6, 0.65),
                     mics=np.array([[1.5, 2.5, 1.4]]), K=3, fs=fs, tiers=[(RHO_INF, 5.0)], taps=32,
                     window=HANN, traj_kind=SPLINE, traj=ctrl, n_ctrl=4, duration=n / fs, x=x,
                     name="receding 1 kHz tone, room 6x5x3 m, order 3, 5 Hz knots")


def small_scene(seed: int = 0, K: int = 4, fs: float = 16000.0, seconds: float = 0.25,
                traj_kind: int = SPLINE, window: int = HANN, taps: int = 32,
                tiers=None, n_mics: int = 1, vmax: float = 2.0, farrow_order: int = 4,
                passband: float = 0.9) -> SceneSpec:
    """A small random scene (parity tests at sizes the oracle finishes quickly)."""
    rng = np.random.default_rng(10_000 + seed)
    dims = tuple(float(v) for v in rng.uniform([3, 3, 2.5], [7, 6, 4]))
    beta = tuple(float(b) for b in rng.uniform(0.5, 0.9, 6))
    n = int(seconds * fs)
    T = n / fs
    if tiers is None:
        tiers = [(1, fs), (RHO_INF, fs / 16)]
    if traj_kind == SPLINE:
        ctrl = random_spline(rng, dims, 4, T, vmax)
        mic = mic_away_from(rng, dims, ctrl, 0.5)
        while mic is None:
            ctrl = random_spline(rng, dims, 4, T, vmax)
            mic = mic_away_from(rng, dims, ctrl, 0.5)
        traj, n_ctrl = list(ctrl.ravel()), 4
    elif traj_kind == LINE:
        mic = np.array(dims) * 0.5 + 0.3
        while True:
            p0 = rng.uniform([1, 1, 1], np.array(dims) - 1)
            if np.linalg.norm(p0 - mic) > 1.0:
                break
        d = rng.standard_normal(3)
        traj, n_ctrl = list(p0) + list(d) + [vmax * 0.5], 0
    else:
        cx, cy = dims[0] / 2, dims[1] / 2
        traj, n_ctrl = [cx, cy, 1.2, 1.0, vmax * 0.5, 0.3], 0
        mic = np.array([cx + 0.2, cy - 0.1, 1.5])
    mics = mic[None, :] + np.array([[0.05 * i, -0.03 * i, 0.02 * i] for i in range(n_mics)])
    return SceneSpec(
        dims=dims, beta=beta, mics=mics, K=K, fs=fs, tiers=tiers, taps=taps, window=window,
        farrow_order=farrow_order, passband=passband,
        traj_kind=traj_kind, traj=traj, n_ctrl=n_ctrl, duration=T,
        x=(rng.standard_normal(n) * 0.1).astype(np.float32), name=f"small scene {seed}")


def with_signal(spec: SceneSpec, x: np.ndarray) -> SceneSpec:
    return replace(spec, x=np.asarray(x, np.float32))
