"""GPU parity of band-limited knot upsampling (tiers with U > 1) against the
FP64 oracle, through the C ABI.

The tier's distance is sampled at knots every N_c samples, interpolated to
virtual knots every N_c / U samples by the windowed-sinc kernel of half-width
Q knots, then linearly (Sec. II-C). Cases: several (rate, U, Q) layouts from
U = 4 to U = 100, every trajectory kind whose extension stays in the room, a
moving array, multiple microphones, a batch mixing linear and upsampled
tiers, and 48 kHz. Tolerance as for the linear tiers: relative L2 <= 1e-5.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api
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
    # 500 Hz knots, 8 virtual knots per interval (records every 4 samples)
    (dict(seed=11, K=3, traj_kind=W.SPLINE, tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)]), 4),
    # 5 Hz knots on a 1 s circle, U = 100 (records every 32 samples)
    (dict(seed=12, K=2, traj_kind=W.CIRCLE, seconds=1.0, tiers=[(1, 16000.0), (W.RHO_INF, 5.0, 100)]), 4),
    # three tiers, two of them upsampled, a short kernel, Kaiser taps
    (dict(seed=13, K=3, traj_kind=W.SPLINE, window=W.KAISER,
          tiers=[(0, 16000.0), (3, 2000.0, 4), (W.RHO_INF, 250.0, 16)]), 2),
    # the widest kernel
    (dict(seed=14, K=2, traj_kind=W.CIRCLE, seconds=0.5, tiers=[(W.RHO_INF, 100.0, 40)]), 8),
    # 48 kHz
    (dict(seed=16, K=3, traj_kind=W.SPLINE, fs=48000.0, seconds=0.08, window=W.KAISER,
          tiers=[(2, 48000.0), (W.RHO_INF, 1000.0, 12)]), 4),
]


@pytest.mark.parametrize("kw,Q", CASES)
def test_upsampled_tier_parity(kw, Q):
    spec = replace(W.small_scene(**kw), up_halfwidth=Q)
    y = gpu_run([spec])[0]
    assert rel_l2(y[0], oracle_full(spec)) < TOL


def test_upsampling_changes_the_result():
    """The upsampled tier is not the linear one (the test above would pass
    trivially if U were ignored): on the 5 Hz circle they differ by far more
    than the tolerance."""
    kw = dict(seed=12, K=2, traj_kind=W.CIRCLE, seconds=1.0)
    lin = W.small_scene(**kw, tiers=[(1, 16000.0), (W.RHO_INF, 5.0)])
    ups = W.small_scene(**kw, tiers=[(1, 16000.0), (W.RHO_INF, 5.0, 100)])
    a, b = gpu_run([lin, ups])
    assert rel_l2(a[0], b[0]) > 100 * TOL


def test_upsampled_multi_mic_and_moving_array():
    spec = W.small_scene(seed=15, K=2, n_mics=2, traj_kind=W.SPLINE, seconds=0.5,
                         tiers=[(1, 16000.0), (W.RHO_INF, 200.0, 10)])
    spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=[0.0, 0.0, 0.0, 0.2, 0.4, 0.0],
                   arr_duration=spec.duration)
    y = gpu_run([spec])[0]
    for m in range(2):
        assert rel_l2(y[m], oracle_full(spec, m)) < TOL


def test_batch_mixing_linear_and_upsampled_tiers():
    specs = [W.small_scene(seed=17, K=2, tiers=[(1, 16000.0), (W.RHO_INF, 1000.0)]),
             replace(W.small_scene(seed=18, K=3, tiers=[(1, 16000.0), (W.RHO_INF, 400.0, 5)]), up_halfwidth=3),
             W.small_scene(seed=19, K=2, traj_kind=W.CIRCLE, tiers=[(W.RHO_INF, 250.0, 32)])]
    ys = gpu_run(specs, tile_config=11)  # one configuration for both (bitwise comparison)
    single = [gpu_run([s], tile_config=11)[0] for s in specs]
    for s, y, y1 in zip(specs, ys, single):
        assert np.array_equal(y, y1)
        assert rel_l2(y[0], oracle_full(s)) < TOL


@pytest.mark.parametrize("rate,U", [(50.0, 10), (5.0, 100)])
def test_order20_upsampled_full_size_sampled(rate, U):
    """The order-20, 48 kHz, 4 s scene (92 168 images) with its last tier on
    band-limited knots, in the bench's launch configuration: the first, middle
    and last output of every output tile and knot-interval edges, each evaluated
    by the oracle one by one."""
    spec = W.config2_upsampled(rate, U)
    y = gpu_run([spec])[0][0]
    steps = spec.tier_steps()
    # knot intervals and the virtual knots' intervals of the upsampled tier
    idx = tile_samples(spec.n_in, 1536, [t[1] for t in steps] + [t[1] // t[2] for t in steps if len(t) > 2])
    ref = oracle.y_at(oracle_scene(spec), spec.x.astype(np.float64), idx)
    assert rel_l2(y[idx], ref) < TOL


@pytest.mark.parametrize("n_out", [1, 7, 1000, 6000])
def test_upsampled_output_lengths(n_out):
    """Outputs shorter and longer than the input (the knot table then reaches
    past the path's end), down to one sample."""
    spec = replace(W.small_scene(seed=20, K=2, traj_kind=W.CIRCLE, seconds=0.25,
                                 tiers=[(0, 16000.0), (W.RHO_INF, 250.0, 16)]), up_halfwidth=3)
    y = gpu_run([spec], n_out=[n_out])[0]
    ref = oracle.synthesize(oracle_scene(spec), spec.x.astype(np.float64), n_out)
    assert y.shape == (1, n_out)
    assert rel_l2(y[0], ref) < TOL or np.max(np.abs(y[0] - ref)) < 1e-9


def test_upsampled_every_tile_config():
    """Every synthesis tile configuration gives the same band-limited result
    (the record scratch and block sizes depend on the configuration)."""
    spec = W.small_scene(seed=21, K=3, traj_kind=W.CIRCLE, seconds=0.3,
                         tiers=[(1, 16000.0), (W.RHO_INF, 200.0, 10)])
    ref = oracle_full(spec)
    for cfg in range(api.tile_configs()):
        y = gpu_run([spec], tile_config=cfg)[0]
        assert rel_l2(y[0], ref) < TOL, cfg
