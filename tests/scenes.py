"""Test helpers: turn a workload SceneSpec into the oracle's plain scene."""
import numpy as np

from oracle import api as oracle
from paper_2508_03065_gb300 import workloads as W


def oracle_scene(spec: W.SceneSpec, mic: int = 0, **override) -> oracle.Scene:
    kw = dict(
        dims=spec.dims, beta=spec.beta, mic=list(np.asarray(spec.mics)[mic]), K=spec.K,
        fs=spec.fs, c=spec.c, tiers=spec.tier_steps(), taps=spec.taps, window=spec.window,
        kaiser_beta=spec.kaiser_beta, traj_kind=spec.traj_kind, traj=list(spec.traj),
        n_ctrl=spec.n_ctrl, duration=spec.duration, arr_kind=spec.arr_kind, arr_traj=list(spec.arr_traj),
        arr_n_ctrl=spec.arr_n_ctrl, arr_duration=spec.arr_duration, up_halfwidth=spec.up_halfwidth,
        delay_model=spec.delay_model)
    if spec.window == 2:  # least-squares Farrow design: the oracle's own
        from oracle import gls
        kw["farrow"] = gls.design(spec.taps, spec.farrow_order, spec.passband)
    kw.update(override)
    return oracle.Scene(**kw)


# Precision envelope of a parity comparison: read positions within this many
# samples of an integer may fall on either side in FP32 (the device's delays
# are good to about 1e-6 samples).
WRAP_DELTA = 1e-5


def beyond_envelope(a, ref, env):
    """Relative L2 of the part of a - ref that the oracle's precision envelope
    does not explain: max(|a - ref| - env, 0), over |ref|."""
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    r = np.maximum(np.abs(a - ref) - np.asarray(env, np.float64), 0.0)
    return float(np.linalg.norm(r) / max(np.linalg.norm(ref), 1e-300))


def tile_samples(n_out: int, tile: int, steps=(), mid: bool = True, edge_tiles: int = 8) -> np.ndarray:
    """Output indices for a sampled full-size parity check: the first, middle
    and last output of every output tile of `tile` samples (the synthesis work
    item), and in `edge_tiles` tiles spread over the signal both edges of the
    first two knot intervals (n mod N in {0, N - 1}) of every knot spacing N > 1
    in `steps`."""
    idx = []
    for t0 in range(0, n_out, tile):
        t1 = min(t0 + tile, n_out) - 1
        idx += [t0, t1] + ([(t0 + t1) // 2] if mid else [])
    n_tiles = (n_out + tile - 1) // tile
    for k in np.linspace(0, n_tiles - 1, min(edge_tiles, n_tiles)).astype(int):
        t0 = int(k) * tile
        for N in steps:
            if N <= 1:
                continue
            j = (t0 + N - 1) // N  # first knot at or after the tile start
            for kn in (j, j + 1):
                idx += [kn * N - 1, kn * N, kn * N + N - 1]
    idx = np.unique(np.asarray(idx, np.int64))
    return idx[(idx >= 0) & (idx < n_out)]


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_length_scene() -> W.SceneSpec:
    """The longest signal the library takes: 2^24 samples (17.5 min at 16 kHz),
    a circle so that the source stays in the room, order 2, one 500 Hz tier."""
    from dataclasses import replace
    n = 1 << 24
    spec = W.small_scene(seed=50, K=2, traj_kind=W.CIRCLE, seconds=1.0, tiers=[(W.RHO_INF, 500.0)])
    rng = np.random.default_rng(50)
    return replace(spec, x=(rng.standard_normal(n) * 0.1).astype(np.float32), duration=n / spec.fs)
