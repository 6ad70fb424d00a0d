"""GPU parity of the reverse mode (msrc_synthesize_backward) through the C ABI.

- dL/dx against the FP64 oracle's transpose sum (relative L2 <= 1e-5) and the
  dot-product identity <A x, v> = <x, A^T v> on the GPU;
- dL/d(trajectory parameters) and dL/d(wall coefficients) against the oracle's
  complex-step gradient (relative <= 1e-4);
- on a full-size differentiation scene (room 6x5x3 m, order 8, 2 s at 16 kHz):
  central differences with Richardson extrapolation of the FP64 oracle on a
  sampled-output loss (<= 1e-4 relative), and of the FP32 GPU forward on the
  full loss (norm-wise, bounded by FP32 rounding / h);
- batched equals per-scene; bitwise reproducible; the autograd Function.
"""
import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import max_length_scene, oracle_scene, rel_l2

pytestmark = pytest.mark.gpu


def _bwd(spec, dy, **kw):
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    dyt = torch.from_numpy(np.ascontiguousarray(dy, np.float32)).cuda().reshape(room.n_mics, -1)
    dx, dp, db = api.synthesize_backward([room], [x], [dyt], **kw)[0]
    torch.cuda.synchronize()
    return (dx.cpu().numpy().astype(np.float64) if dx is not None else None,
            dp.cpu().numpy() if dp is not None else None, db.cpu().numpy() if db is not None else None)


@pytest.mark.parametrize("kw", [
    dict(seed=60, K=4, window=W.HANN, taps=32),
    dict(seed=61, K=3, window=W.KAISER, taps=32, traj_kind=W.CIRCLE),
    dict(seed=62, K=3, window=W.HANN, taps=64, traj_kind=W.LINE, seconds=0.08),
    dict(seed=63, K=4, window=W.KAISER, taps=16, tiers=[(0, 16000.0), (3, 2000.0), (W.RHO_INF, 400.0)]),
    dict(seed=71, K=3, window=W.FARROW_LS, taps=32, farrow_order=4, passband=0.9),
])
def test_dx_matches_oracle_transpose(kw):
    spec = W.small_scene(**kw)
    dy = np.random.default_rng(kw["seed"]).standard_normal(spec.n_in)
    dx, _, _ = _bwd(spec, dy, want_params=False, want_beta=False)
    ref = oracle.adjoint_x(oracle_scene(spec), dy, spec.n_in)
    assert rel_l2(dx, ref) < 1e-5


def test_dx_multi_mic():
    spec = W.small_scene(seed=64, K=3, n_mics=2)
    dy = np.random.default_rng(1).standard_normal((2, spec.n_in))
    dx, _, _ = _bwd(spec, dy, want_params=False, want_beta=False)
    ref = sum(oracle.adjoint_x(oracle_scene(spec, m), dy[m], spec.n_in) for m in range(2))
    assert rel_l2(dx, ref) < 1e-5


# Signals longer than one time group (12 tiles of 1024 samples): every group of
# tiles orders the images by their distance at its own middle, so the images of
# a block differ from group to group (1.6 s: three groups, the last one tile).
@pytest.mark.parametrize("kw", [
    dict(seed=74, K=3, seconds=1.0, window=W.HANN, taps=32, n_mics=2),
    dict(seed=75, K=3, seconds=1.6, window=W.KAISER, taps=32),
])
def test_dx_several_time_groups(kw):
    spec = W.small_scene(**kw)
    n_m = len(spec.mics)
    dy = np.random.default_rng(kw["seed"]).standard_normal((n_m, spec.n_in))
    dx, _, _ = _bwd(spec, dy, want_params=False, want_beta=False)
    ref = sum(oracle.adjoint_x(oracle_scene(spec, m), dy[m], spec.n_in) for m in range(n_m))
    assert rel_l2(dx, ref) < 1e-5


def test_dx_groups_of_two_full_blocks():
    # a tier with knots every 96 samples holds 256 images per block, and the
    # dx kernel's groups take two such blocks (one correlation for 512 images)
    spec = W.small_scene(seed=77, K=6, seconds=0.1, window=W.HANN, taps=32,
                         tiers=[(1, 16000.0), (W.RHO_INF, 16000.0 / 96)])
    dy = np.random.default_rng(77).standard_normal(spec.n_in)
    dx, _, _ = _bwd(spec, dy, want_params=False, want_beta=False)
    ref = oracle.adjoint_x(oracle_scene(spec), dy, spec.n_in)
    assert rel_l2(dx, ref) < 1e-5


def test_param_and_beta_gradients_several_time_groups():
    spec = W.small_scene(seed=76, K=2, seconds=1.6, window=W.HANN, taps=16)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    target = np.random.default_rng(4).standard_normal(spec.n_in) * 0.01
    _, dp, db = _bwd(spec, oracle.synthesize(sc, x) - target, want_dx=False)
    ids = [0, 2, 4, 7, 9, 11]
    g_cs = oracle.loss_grad_cs(sc, x, target, ids + [48, 49, 50, 51, 52, 53])
    got = np.concatenate([dp[ids], db])
    assert np.linalg.norm(got - g_cs) <= 1e-4 * np.linalg.norm(g_cs), (got, g_cs)


def test_dot_product_identity_on_gpu():
    spec = W.small_scene(seed=65, K=5, seconds=0.3)
    room = api.Room.from_spec(spec)
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.standard_normal(spec.n_in).astype(np.float32)).cuda()
    v = torch.from_numpy(rng.standard_normal(spec.n_in).astype(np.float32)).cuda()
    y = api.synthesize([room], [x])[0][0]
    dx = api.synthesize_backward([room], [x], [v[None]], want_params=False, want_beta=False)[0][0]
    lhs = float(torch.dot(y.double(), v.double()))
    rhs = float(torch.dot(x.double(), dx.double()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_dot_product_identity_at_maximum_length():
    # reverse mode over the longest signal the library takes (2^24 samples):
    # <A x, v> = <x, A^T v> with v leaning on A x so that neither side is small
    spec = max_length_scene()
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    y = api.synthesize([room], [x])[0][0]
    rng = np.random.default_rng(3)
    v = y / y.norm() * float(np.sqrt(spec.n_in)) + torch.from_numpy(
        rng.standard_normal(spec.n_in).astype(np.float32)).cuda()
    dx = api.synthesize_backward([room], [x], [v[None]], want_params=False, want_beta=False)[0][0]
    assert dx.shape == (spec.n_in,) and bool(torch.isfinite(dx).all())
    lhs = float(torch.dot(y.double(), v.double()))
    rhs = float(torch.dot(x.double(), dx.double()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("kw,ids", [
    (dict(seed=66, K=2, seconds=0.03, window=W.HANN, traj_kind=W.SPLINE), [0, 1, 2, 4, 7, 11]),
    (dict(seed=67, K=2, seconds=0.03, window=W.HANN, traj_kind=W.CIRCLE), [0, 1, 3, 4, 5]),
    (dict(seed=68, K=2, seconds=0.03, window=W.HANN, traj_kind=W.LINE), [0, 1, 2, 3, 6]),
    # knot spacings that do not divide the 1024-sample tile: a knot's samples
    # fall in two or more tiles (spacing 12, and 1600 > one tile)
    (dict(seed=69, K=2, seconds=0.1, window=W.KAISER, taps=32, traj_kind=W.SPLINE,
          tiers=[(1, 16000.0), (W.RHO_INF, 16000.0 / 12)]), [0, 3, 5, 8, 10]),
    (dict(seed=70, K=2, seconds=0.25, window=W.HANN, taps=16, traj_kind=W.CIRCLE,
          tiers=[(0, 16000.0), (W.RHO_INF, 10.0)]), [0, 1, 3, 4, 5]),
    (dict(seed=72, K=2, seconds=0.03, window=W.FARROW_LS, taps=16, farrow_order=3, passband=0.8,
          traj_kind=W.SPLINE), [0, 2, 4, 9]),
])
def test_param_and_beta_gradients_match_complex_step(kw, ids):
    spec = W.small_scene(**kw)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    target = np.random.default_rng(3).standard_normal(spec.n_in) * 0.01
    y_ref = oracle.synthesize(sc, x)
    _, dp, db = _bwd(spec, y_ref - target, want_dx=False)
    g_cs = oracle.loss_grad_cs(sc, x, target, ids + [48, 49, 50, 51, 52, 53])
    got = np.concatenate([dp[ids], db])
    assert np.linalg.norm(got - g_cs) <= 1e-4 * np.linalg.norm(g_cs), (got, g_cs)
    big = np.abs(g_cs) > 1e-2 * np.max(np.abs(g_cs))
    assert np.all(np.abs(got - g_cs)[big] <= 1e-3 * np.abs(g_cs)[big])


def _fd(f, h):
    # central differences at h and h/2 with Richardson extrapolation
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def test_full_size_differentiation_scene_vs_oracle_finite_differences():
    # One of the 16 differentiation scenes at full size: 6x5x3 m, order 8 (6664
    # images), 2 s at 16 kHz, 6 control points. Loss 0.5 sum over 400 sampled
    # outputs of (y - y*)^2 with a seeded target. Reference: FP64 oracle central
    # differences (h = 1e-3 m, 1e-4) with Richardson extrapolation.
    spec, target = W.config4_scene(0)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    idx = np.linspace(0, spec.n_in - 1, 400).astype(np.int64)

    def oloss(traj=None, beta=None):
        s2 = oracle.Scene(**{**sc.__dict__, "traj": traj if traj is not None else sc.traj,
                             "beta": beta if beta is not None else sc.beta})
        return 0.5 * float(np.sum((oracle.y_at(s2, x, idx) - target[idx]) ** 2))

    dy = np.zeros(spec.n_in)
    dy[idx] = oracle.y_at(sc, x, idx) - target[idx]
    _, dp, db = _bwd(spec, dy, want_dx=False)
    for pid in (1, 6, 13):
        def f(dlt, pid=pid):
            tr = list(sc.traj); tr[pid] += dlt
            return oloss(traj=tr)
        ref = _fd(f, 1e-3)
        assert abs(dp[pid] - ref) <= 1e-4 * abs(ref), (pid, dp[pid], ref)
    for w in (0, 3):
        def f(dlt, w=w):
            bt = list(sc.beta); bt[w] += dlt
            return oloss(beta=bt)
        ref = _fd(f, 1e-4)
        assert abs(db[w] - ref) <= 1e-4 * abs(ref), (w, db[w], ref)


def test_full_size_gpu_forward_finite_differences():
    # Same scene, full loss, differences of the FP32 GPU forward itself. The
    # FP32 rounding of y (~1e-7 relative) divided by h bounds the agreement at a
    # few 1e-4; checked norm-wise over control-point coordinates and walls.
    spec, target = W.config4_scene(0)
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    tgt = torch.from_numpy(target).cuda().double()
    p0 = np.array(spec.traj, np.float64)
    b0 = np.array(spec.beta, np.float64)

    def loss(params, beta):
        room.set_trajectory(spec.traj_kind, params, spec.duration, spec.mics, spec.n_ctrl)
        room.set_reflection(beta)
        y = api.synthesize([room], [x])[0][0].double()
        return 0.5 * float(torch.sum((y - tgt) ** 2))

    room.set_trajectory(spec.traj_kind, p0, spec.duration, spec.mics, spec.n_ctrl)
    room.set_reflection(b0)
    y = api.synthesize([room], [x])[0]
    _, dp, db = api.synthesize_backward([room], [x], [(y[0].double() - tgt).float()[None]], want_dx=False)[0]
    got, ref = [], []
    for pid in range(0, 18, 2):
        def f(dlt, pid=pid):
            p = p0.copy(); p[pid] += dlt
            return loss(p, b0)
        got.append(float(dp[pid])); ref.append(_fd(f, 2e-3))
    for w in range(6):
        def f(dlt, w=w):
            b = b0.copy(); b[w] += dlt
            return loss(p0, b)
        got.append(float(db[w])); ref.append(_fd(f, 2e-4))
    got, ref = np.array(got), np.array(ref)
    assert np.linalg.norm(got - ref) <= 5e-4 * np.linalg.norm(ref), (got, ref)


def test_backward_batched_equals_single_and_reproducible():
    specs = [W.small_scene(seed=70 + i, K=3 + i, seconds=0.05 + 0.03 * i) for i in range(3)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    dys = [torch.randn(1, s.n_in, device="cuda") for s in specs]
    batched = api.synthesize_backward(rooms, xs, dys)
    again = api.synthesize_backward(rooms, xs, dys)
    for i in range(3):
        single = api.synthesize_backward([rooms[i]], [xs[i]], [dys[i]])[0]
        for a, b, c in zip(batched[i], single, again[i]):
            assert torch.equal(a, b) and torch.equal(a, c)


def test_autograd_function():
    spec = W.small_scene(seed=80, K=3, seconds=0.05)
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda().requires_grad_(True)
    params = torch.tensor(np.array(spec.traj + [0.0] * (48 - len(spec.traj))), dtype=torch.float64,
                          requires_grad=True)
    beta = torch.tensor(spec.beta, dtype=torch.float64, requires_grad=True)
    y = api.synthesize_ad(room, x, params, beta)
    loss = (y.double() ** 2).sum() * 0.5
    loss.backward()
    dx, dp, db = api.synthesize_backward([room], [x.detach()], [y.detach()])[0]
    assert torch.equal(x.grad, dx)
    assert torch.equal(params.grad, dp.cpu())
    assert torch.equal(beta.grad, db.cpu())


def test_moving_array_reverse_mode():
    # dx against the oracle transpose and source-trajectory / wall gradients
    # against the complex step, with microphones on a moving array
    from dataclasses import replace
    spec = W.small_scene(seed=73, K=2, seconds=0.03, window=W.HANN, traj_kind=W.SPLINE)
    spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=[0.0, 0.0, 0.0, 0.1, 0.5, 0.3], arr_duration=spec.duration)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    dy = np.random.default_rng(74).standard_normal(spec.n_in)
    dx, _, _ = _bwd(spec, dy, want_params=False, want_beta=False)
    assert rel_l2(dx, oracle.adjoint_x(sc, dy, spec.n_in)) < 1e-5
    target = np.random.default_rng(3).standard_normal(spec.n_in) * 0.01
    y_ref = oracle.synthesize(sc, x)
    _, dp, db = _bwd(spec, y_ref - target, want_dx=False)
    ids = [0, 1, 5, 9]
    g_cs = oracle.loss_grad_cs(sc, x, target, ids + [48, 49, 50, 51, 52, 53])
    got = np.concatenate([dp[ids], db])
    assert np.linalg.norm(got - g_cs) <= 1e-4 * np.linalg.norm(g_cs), (got, g_cs)

