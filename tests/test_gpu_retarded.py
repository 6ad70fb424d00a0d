"""GPU parity of emission-time (retarded) delays (delay_model 1) against the
FP64 oracle, through the C ABI.

At every knot the image's distance is the path length c tau of the sound
reaching the microphone at the knot time, c tau = |r_i(t - tau) - m(t)|; delay
and gain follow from it as for reception-time distances. Cases: every
trajectory kind, Hann and Kaiser taps, a dense tier (every sample a knot),
several microphones, a moving array, 48 kHz, batches mixing both models, and
the order-20 scene at full size on sampled outputs. Tolerance: relative L2
<= 1e-5, as for the reception-time model.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import _lib, api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2, tile_samples

pytestmark = pytest.mark.gpu
TOL = 1e-5


def gpu_run(specs, n_out=None, tile_config=None):
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    ws = api.Workspace()
    ys = api.synthesize(rooms, xs, n_out=n_out, workspace=ws, tile_config=tile_config)
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    return [y.cpu().numpy().astype(np.float64) for y in ys]


def oracle_full(spec, mic=0):
    return oracle.synthesize(oracle_scene(spec, mic), spec.x.astype(np.float64))


CASES = [
    dict(seed=51, K=4, traj_kind=W.SPLINE, vmax=3.0),
    dict(seed=52, K=4, traj_kind=W.CIRCLE, window=W.KAISER, seconds=0.4),
    dict(seed=53, K=3, traj_kind=W.SPLINE, tiers=[(0, 16000.0), (3, 2000.0), (W.RHO_INF, 250.0)]),
    dict(seed=54, K=3, traj_kind=W.SPLINE, fs=48000.0, seconds=0.08, window=W.KAISER,
         tiers=[(2, 48000.0), (W.RHO_INF, 500.0)]),
    dict(seed=55, K=5, traj_kind=W.CIRCLE, taps=64, tiers=[(W.RHO_INF, 16000.0)], seconds=0.1),
]


@pytest.mark.parametrize("kw", CASES)
def test_emission_time_parity(kw):
    spec = replace(W.small_scene(**kw), delay_model=1)
    y = gpu_run([spec])[0]
    assert rel_l2(y[0], oracle_full(spec)) < TOL


def test_models_differ_and_still_source_agrees():
    spec = W.small_scene(seed=56, K=3, traj_kind=W.CIRCLE, seconds=0.3)
    a, b = gpu_run([spec, replace(spec, delay_model=1)])
    assert rel_l2(b[0], a[0]) > 100 * TOL
    still = replace(spec, traj=list(spec.traj[:4]) + [0.0, spec.traj[5]])
    c, d = gpu_run([still, replace(still, delay_model=1)])
    assert rel_l2(d[0], c[0]) < 1e-6


def test_emission_time_multi_mic_moving_array():
    spec = W.small_scene(seed=57, K=3, n_mics=2, traj_kind=W.SPLINE, seconds=0.3,
                         tiers=[(1, 16000.0), (W.RHO_INF, 1000.0)])
    spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=[0.0, 0.0, 0.0, 0.2, 0.6, 0.0],
                   arr_duration=spec.duration, delay_model=1)
    y = gpu_run([spec])[0]
    for m in range(2):
        assert rel_l2(y[m], oracle_full(spec, m)) < TOL


def test_batch_mixing_delay_models():
    specs = [W.small_scene(seed=58, K=2), replace(W.small_scene(seed=59, K=3, traj_kind=W.CIRCLE), delay_model=1),
             replace(W.small_scene(seed=60, K=2, traj_kind=W.SPLINE), delay_model=1)]
    ys = gpu_run(specs, tile_config=11)  # one configuration for both (bitwise comparison)
    for s, y in zip(specs, ys):
        assert np.array_equal(y, gpu_run([s], tile_config=11)[0])
        assert rel_l2(y[0], oracle_full(s)) < TOL


def test_order20_emission_time_full_size_sampled():
    spec = replace(W.config2(), delay_model=1)
    y = gpu_run([spec])[0][0]
    idx = tile_samples(spec.n_in, 1536, [N for _, N, *_ in spec.tier_steps()])
    ref = oracle.y_at(oracle_scene(spec), spec.x.astype(np.float64), idx)
    assert rel_l2(y[idx], ref) < TOL


def test_emission_time_refuses_upsampled_tiers():
    spec = replace(W.small_scene(seed=61, K=2), delay_model=1)
    x = torch.from_numpy(spec.x).cuda()
    ups = replace(spec, tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)])
    with pytest.raises(_lib.MsrcError):
        api.synthesize([api.Room.from_spec(ups)], [x])


@pytest.mark.parametrize("n_out", [1, 7, 1000, 6000])
def test_emission_time_output_lengths(n_out):
    """Outputs shorter and longer than the input, down to one sample."""
    spec = replace(W.small_scene(seed=62, K=3, traj_kind=W.CIRCLE, seconds=0.25), delay_model=1)
    y = gpu_run([spec], n_out=[n_out])[0]
    ref = oracle.synthesize(oracle_scene(spec), spec.x.astype(np.float64), n_out)
    assert y.shape == (1, n_out)
    assert rel_l2(y[0], ref) < TOL or np.max(np.abs(y[0] - ref)) < 1e-9


def test_emission_time_free_field_receding_source():
    """Free field (walls absorbing), a source receding from the microphone: the
    GPU's emission-time output equals the oracle's, whose closed form the pins
    check."""
    spec = W.small_scene(seed=63, K=0, traj_kind=W.LINE, seconds=0.5)
    spec = replace(spec, beta=(0.0,) * 6, delay_model=1)
    y = gpu_run([spec])[0]
    assert rel_l2(y[0], oracle_full(spec)) < TOL


def test_emission_time_every_tile_config():
    """Every synthesis tile configuration gives the same emission-time result."""
    spec = replace(W.small_scene(seed=64, K=3, traj_kind=W.SPLINE, seconds=0.3), delay_model=1)
    ref = oracle_full(spec)
    for cfg in range(api.tile_configs()):
        y = gpu_run([spec], tile_config=cfg)[0]
        assert rel_l2(y[0], ref) < TOL, cfg
