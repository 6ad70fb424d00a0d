"""Seeded random sweeps of the forward synthesis and of dL/dx against the FP64
oracle.

Each case draws one scene from the options the library takes together: sample
rate, taps and tap-weight design (Hann, Kaiser, least-squares Farrow of order
1..4), trajectory kind, one to four tiers with random knot spacings, band-limited
tiers (upsampling factor and kernel half-width), emission-time delays, a moving
microphone array, one to three microphones and an output shorter or longer
than the input. Parity bar: relative L2 <= 1e-5 per microphone beyond the
oracle's precision envelope (read positions within 1e-5 samples of an integer
may take either side; this only matters for the least-squares Farrow designs,
whose taps jump there), and the device error word stays clear. The reverse-mode sweep draws from the same space
without band-limited tiers and emission-time delays, and compares dL/dx for a
random upstream gradient with the oracle's transpose sum.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import WRAP_DELTA, beyond_envelope, oracle_scene

pytestmark = pytest.mark.gpu
TOL = 1e-5
N_CASES = 32


def random_spec(i: int, reverse: bool = False) -> W.SceneSpec:
    """Random scene i; reverse=True keeps to what reverse mode takes (linear
    knots, delays at reception time)."""
    rng = np.random.default_rng((8000 if reverse else 7000) + i)
    fs = float(rng.choice([8000.0, 16000.0, 22050.0, 44100.0, 48000.0]))
    window = int(rng.choice([W.HANN, W.KAISER, W.FARROW_LS]))
    taps = int(rng.choice([8, 16, 24, 32, 64]))
    kind = int(rng.choice([W.LINE, W.CIRCLE, W.SPLINE]))
    K = int(rng.integers(0, 6))
    seconds = float(rng.uniform(0.02, 0.1))
    n_mics = int(rng.integers(1, 4))
    retarded = not reverse and rng.random() < 0.3
    # tiers: increasing reflection-count bounds, knot spacings N samples (rate fs / N);
    # a band-limited tier takes N = U * M virtual-knot spacing M
    n_t = int(rng.integers(1, 5))
    bounds = sorted(rng.choice(np.arange(0, 9), size=n_t - 1, replace=False).tolist()) + [W.RHO_INF]
    tiers = []
    for b in bounds:
        if not retarded and not reverse and rng.random() < 0.35:
            U = int(rng.choice([2, 3, 4, 8, 16]))
            M = int(rng.choice([1, 2, 4, 6, 12]))
            tiers.append((b, fs / (U * M), U))
        else:
            tiers.append((b, fs / int(rng.choice([1, 2, 3, 5, 8, 12, 16, 32, 48, 96]))))
    spec = W.small_scene(seed=500 + i, K=K, fs=fs, seconds=seconds, traj_kind=kind, window=window, taps=taps,
                         tiers=tiers, n_mics=n_mics, farrow_order=int(rng.integers(1, 5)),
                         passband=float(rng.uniform(0.5, 0.95)))
    spec = replace(spec, delay_model=1 if retarded else 0, up_halfwidth=int(rng.choice([2, 4, 6, 8])))
    if rng.random() < 0.3:  # the array drifts slowly along a line
        d = rng.standard_normal(3)
        spec = replace(spec, arr_kind=W.LINE, arr_traj=[0.0, 0.0, 0.0] + list(d) + [0.3],
                       arr_duration=spec.duration)
    choice = int(rng.integers(0, 3))
    n_out = spec.n_in if choice == 0 else (spec.n_in // 2 + 1 if choice == 1 else spec.n_in + 300)
    return replace(spec, n_out=n_out, name=f"random scene {i}")


@pytest.mark.parametrize("i", range(N_CASES))
def test_random_scene_parity(i):
    spec = random_spec(i)
    room = api.Room.from_spec(spec)
    ws = api.Workspace()
    y = api.synthesize([room], [torch.from_numpy(spec.x).cuda()], n_out=[spec.n_out], workspace=ws)[0]
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    y = y.cpu().numpy().astype(np.float64)
    assert y.shape == (len(spec.mics), spec.n_out)
    for m in range(len(spec.mics)):
        ref, env = oracle.synthesize_envelope(oracle_scene(spec, m), spec.x.astype(np.float64), spec.n_out,
                                              WRAP_DELTA)
        err = beyond_envelope(y[m], ref, env)
        assert err < TOL, (spec.name, m, err)


@pytest.mark.parametrize("i", range(12))
def test_random_scene_dx_parity(i):
    spec = random_spec(i, reverse=True)
    room = api.Room.from_spec(spec)
    rng = np.random.default_rng(9000 + i)
    dy = rng.standard_normal((len(spec.mics), spec.n_out)).astype(np.float32)
    x = torch.from_numpy(spec.x).cuda()
    y = api.synthesize([room], [x], n_out=[spec.n_out])[0]
    dx = api.synthesize_backward([room], [x], [torch.from_numpy(dy).cuda()], want_params=False,
                                 want_beta=False)[0][0]
    torch.cuda.synchronize()
    assert y.shape == dy.shape
    dx = dx.cpu().numpy().astype(np.float64)
    ref, env = np.zeros(spec.n_in), np.zeros(spec.n_in)
    for m in range(len(spec.mics)):
        r, e = oracle.adjoint_x_envelope(oracle_scene(spec, m), dy[m].astype(np.float64), spec.n_in, WRAP_DELTA)
        ref += r
        env += e
    err = beyond_envelope(dx, ref, env)
    assert err < TOL, (spec.name, err)


def _has_option_tiers(spec) -> bool:
    return spec.delay_model == 1 or any(len(t) == 3 and t[2] > 1 for t in spec.tiers)


# the random scenes with upsampled tiers or emission-time delays
OPTION_CASES = [i for i in range(N_CASES) if _has_option_tiers(random_spec(i))]


@pytest.mark.parametrize("i", OPTION_CASES[:12])
def test_random_option_scene_dx_parity(i):
    # reverse mode on the forward generator's scenes that upsample a tier or
    # take emission-time delays
    spec = random_spec(i)
    room = api.Room.from_spec(spec)
    dy = np.random.default_rng(9200 + i).standard_normal((len(spec.mics), spec.n_out)).astype(np.float32)
    x = torch.from_numpy(spec.x).cuda()
    ws = api.Workspace()
    dx = api.synthesize_backward([room], [x], [torch.from_numpy(dy).cuda()], want_params=False,
                                 want_beta=False, workspace=ws)[0][0]
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    dx = dx.cpu().numpy().astype(np.float64)
    ref, env = np.zeros(spec.n_in), np.zeros(spec.n_in)
    for m in range(len(spec.mics)):
        r, e = oracle.adjoint_x_envelope(oracle_scene(spec, m), dy[m].astype(np.float64), spec.n_in, WRAP_DELTA)
        ref += r
        env += e
    err = beyond_envelope(dx, ref, env)
    assert err < TOL, (spec.name, err)


def test_random_batch_equals_single_calls():
    # one batched launch over 8 heterogeneous random scenes (taps and window
    # shared, as a batch requires) equals the per-scene calls bitwise
    specs = [replace(random_spec(i), taps=32, window=W.KAISER) for i in range(8)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    # in one tile configuration (the automatic choice may differ between a
    # batch and one of its scenes)
    ys = api.synthesize(rooms, xs, n_out=[s.n_out for s in specs], tile_config=11)
    for r, s, x, yb in zip(rooms, specs, xs, ys):
        assert torch.equal(yb, api.synthesize([r], [x], n_out=[s.n_out], tile_config=11)[0]), s.name


def test_random_backward_batch_equals_single_calls():
    specs = [replace(random_spec(i, reverse=True), taps=32, window=W.HANN) for i in range(6)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    dys = [torch.from_numpy(np.random.default_rng(9100 + i).standard_normal((len(s.mics), s.n_out))
                            .astype(np.float32)).cuda() for i, s in enumerate(specs)]
    batched = api.synthesize_backward(rooms, xs, dys)
    for r, s, x, dy, got in zip(rooms, specs, xs, dys, batched):
        one = api.synthesize_backward([r], [x], [dy])[0]
        for a, b in zip(got, one):
            assert torch.equal(a, b), s.name
