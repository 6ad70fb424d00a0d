"""GPU parity of the reverse mode with respect to the microphone array's
trajectory (msrc_synthesize_backward_ex, darray), through the C ABI.

The microphones sit at m + a(t) - a(0) (Sec. II-A's distance with moving
receivers); dL/d(array trajectory parameters) is compared with the FP64
oracle's complex step (ids 54..101 of oracle.loss_grad_cs), summed over the
microphones: line, circle and spline arrays on linear tiers, a band-limited
tier and emission-time delays (relative <= 1e-4 norm-wise; per component 1e-3
relative above a floor of 2e-5 of the largest component). A still array gives
zeros; asking for the array gradient leaves the other outputs bitwise
unchanged; a batch equals the per-scene calls bitwise.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene

pytestmark = pytest.mark.gpu

ARRAYS = {
    W.LINE: ([0.0, 0.0, 0.0, 0.3, 0.9, 0.2, 0.8], 0, [57, 58, 59, 60]),
    W.CIRCLE: ([0.0, 0.0, 0.0, 0.12, 0.6, 0.4], 0, [57, 58, 59]),
    W.SPLINE: ([0.0, 0.0, 0.0, 0.05, 0.02, 0.0, 0.08, 0.07, 0.01, 0.1, 0.12, 0.03], 4, [57, 58, 61, 63, 64, 65]),
}


def _with_array(spec, kind):
    traj, n_ctrl, _ = ARRAYS[kind]
    return replace(spec, arr_kind=kind, arr_traj=list(traj), arr_n_ctrl=n_ctrl, arr_duration=spec.duration)


def _bwd(specs, dys, **kw):
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    dyt = [torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda().reshape(r.n_mics, -1)
           for d, r in zip(dys, rooms)]
    ws = api.Workspace()
    out = api.synthesize_backward(rooms, xs, dyt, workspace=ws, **kw)
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    return out


def _cs_array_case(spec, ids):
    n_m = len(spec.mics)
    x = spec.x.astype(np.float64)
    target = np.random.default_rng(8).standard_normal((n_m, spec.n_in)) * 0.01
    dy, g_cs = [], np.zeros(len(ids))
    for m in range(n_m):
        sc = oracle_scene(spec, m)
        dy.append(oracle.synthesize(sc, x) - target[m])
        g_cs += oracle.loss_grad_cs(sc, x, target[m], ids)
    (_, _, _, da), = _bwd([spec], [np.stack(dy)], want_dx=False, want_array=True)
    got = da.cpu().numpy()[[i - 54 for i in ids]]
    assert np.linalg.norm(got - g_cs) <= 1e-4 * np.linalg.norm(g_cs), (got, g_cs)
    scale = np.max(np.abs(g_cs))
    assert np.all(np.abs(got - g_cs) <= 1e-3 * np.abs(g_cs) + 2e-5 * scale), (got, g_cs)


@pytest.mark.parametrize("kind", [W.LINE, W.CIRCLE, W.SPLINE])
def test_array_gradient_linear_tiers(kind):
    spec = _with_array(W.small_scene(seed=81, K=2, seconds=0.03, traj_kind=W.SPLINE), kind)
    _cs_array_case(spec, ARRAYS[kind][2])


def test_array_gradient_two_microphones_dense_knots():
    spec = W.small_scene(seed=82, K=2, seconds=0.1, window=W.KAISER, traj_kind=W.CIRCLE, n_mics=2,
                         tiers=[(1, 16000.0), (W.RHO_INF, 16000.0 / 12)])
    _cs_array_case(_with_array(spec, W.CIRCLE), ARRAYS[W.CIRCLE][2])


def test_array_gradient_upsampled_tier():
    spec = W.small_scene(seed=83, K=2, seconds=0.04, traj_kind=W.SPLINE, tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)])
    _cs_array_case(_with_array(replace(spec, up_halfwidth=4), W.LINE), ARRAYS[W.LINE][2])


@pytest.mark.parametrize("kind", [W.LINE, W.SPLINE])
def test_array_gradient_emission_time(kind):
    spec = replace(W.small_scene(seed=84, K=2, seconds=0.03, traj_kind=W.CIRCLE), delay_model=1)
    _cs_array_case(_with_array(spec, kind), ARRAYS[kind][2])


def test_still_array_zero_and_other_outputs_unchanged():
    moving = _with_array(W.small_scene(seed=85, K=2, seconds=0.05), W.CIRCLE)
    still = W.small_scene(seed=86, K=2, seconds=0.05)
    dys = [np.random.default_rng(9).standard_normal((1, s.n_in)) for s in (moving, still)]
    with_arr = _bwd([moving, still], dys, want_array=True)
    without = _bwd([moving, still], dys)
    for a, b in zip(with_arr, without):
        for u, v in zip(a[:3], b):
            assert torch.equal(u, v)
    assert torch.count_nonzero(with_arr[1][3]) == 0
    assert torch.count_nonzero(with_arr[0][3]) > 0


def test_array_gradient_batch_equals_single():
    specs = [_with_array(W.small_scene(seed=87, K=2, seconds=0.05), W.LINE),
             _with_array(replace(W.small_scene(seed=88, K=2, seconds=0.04, traj_kind=W.CIRCLE), delay_model=1),
                         W.SPLINE),
             _with_array(replace(W.small_scene(seed=89, K=2, seconds=0.04, traj_kind=W.SPLINE,
                                               tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)]), up_halfwidth=4),
                         W.CIRCLE)]
    specs = [replace(s, taps=32) for s in specs]
    dys = [np.random.default_rng(10 + i).standard_normal((1, s.n_in)) for i, s in enumerate(specs)]
    batched = _bwd(specs, dys, want_array=True)
    for i, s in enumerate(specs):
        single = _bwd([s], [dys[i]], want_array=True)[0]
        for u, v in zip(batched[i], single):
            assert torch.equal(u, v), (i, s.name)
