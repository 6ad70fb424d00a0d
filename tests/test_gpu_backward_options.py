"""GPU parity of the reverse mode (msrc_synthesize_backward) on the tiers whose
delays are not linear in the knot positions, through the C ABI:
band-limited knot upsampling (tiers with U > 1, Sec. II-C) and emission-time
delays (delay model 1, Sec. II-A read with the distance from the emission
point).

- dL/dx against the FP64 oracle's transpose sum (relative L2 <= 1e-5), one and
  several microphones, a moving array; the dot-product identity on the GPU;
- dL/d(trajectory parameters) and dL/d(wall coefficients) against the oracle's
  complex-step gradient (relative <= 1e-4 norm-wise; per component 1e-3
  relative above a floor of 2e-5 of the largest component);
- the differentiation scene's room and path (6x5x3 m, 2 s at 16 kHz, order 4)
  with an upsampled tier and with emission-time delays: central differences
  with Richardson extrapolation of the FP64 oracle on a sampled-output loss
  (<= 1e-4 relative);
- a batch mixing linear, upsampled and emission-time scenes equals the
  per-scene calls bitwise, and a repeated call is bitwise identical;
- outputs shorter and longer than the input, the direct path alone, and six
  small random scenes (trajectory kind, window, taps, tier layout, U, Q, array
  motion) against the complex step.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2

pytestmark = pytest.mark.gpu

# upsampled tiers: (scene, kernel half-width Q)
BL = [
    (dict(seed=11, K=3, traj_kind=W.SPLINE, seconds=0.1, tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)]), 4),
    (dict(seed=13, K=3, traj_kind=W.SPLINE, window=W.KAISER, seconds=0.1,
          tiers=[(0, 16000.0), (3, 2000.0, 4), (W.RHO_INF, 250.0, 16)]), 2),
    (dict(seed=14, K=2, traj_kind=W.CIRCLE, seconds=0.25, tiers=[(W.RHO_INF, 100.0, 40)]), 8),
    (dict(seed=16, K=3, traj_kind=W.SPLINE, fs=48000.0, seconds=0.05, window=W.KAISER,
          tiers=[(2, 48000.0), (W.RHO_INF, 1000.0, 12)]), 4),
]
# emission-time delays
RET = [
    dict(seed=21, K=3, traj_kind=W.SPLINE, seconds=0.1),
    dict(seed=22, K=3, traj_kind=W.CIRCLE, seconds=0.1, window=W.KAISER, taps=16),
    dict(seed=23, K=2, traj_kind=W.LINE, seconds=0.08, tiers=[(1, 16000.0), (W.RHO_INF, 16000.0 / 12)]),
]


def _bl(kw, Q):
    return replace(W.small_scene(**kw), up_halfwidth=Q)


def _ret(kw):
    return replace(W.small_scene(**kw), delay_model=1)


def _bwd(spec, dy, **kw):
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    dyt = torch.from_numpy(np.ascontiguousarray(dy, np.float32)).cuda().reshape(room.n_mics, -1)
    ws = api.Workspace()
    dx, dp, db = api.synthesize_backward([room], [x], [dyt], workspace=ws, **kw)[0]
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    return (dx.cpu().numpy().astype(np.float64) if dx is not None else None,
            dp.cpu().numpy() if dp is not None else None, db.cpu().numpy() if db is not None else None)


def _dx_case(spec, seed):
    dy = np.random.default_rng(seed).standard_normal((len(spec.mics), spec.n_in))
    dx, _, _ = _bwd(spec, dy, want_params=False, want_beta=False)
    ref = sum(oracle.adjoint_x(oracle_scene(spec, m), dy[m], spec.n_in) for m in range(len(spec.mics)))
    assert rel_l2(dx, ref) < 1e-5


@pytest.mark.parametrize("kw,Q", BL)
def test_dx_upsampled_tiers(kw, Q):
    _dx_case(_bl(kw, Q), kw["seed"])


@pytest.mark.parametrize("kw", RET)
def test_dx_emission_time(kw):
    _dx_case(_ret(kw), kw["seed"])


def test_dx_multi_mic_and_moving_array():
    kw, Q = BL[0]
    _dx_case(_bl(dict(kw, n_mics=2), Q), 31)
    spec = _ret(dict(RET[0], n_mics=2))
    _dx_case(replace(spec, arr_kind=W.CIRCLE, arr_traj=[0.0, 0.0, 0.0, 0.1, 0.5, 0.3], arr_duration=spec.duration),
             32)


@pytest.mark.parametrize("spec", [_bl(*BL[1]), _ret(RET[1])], ids=["upsampled", "emission-time"])
def test_dot_product_identity(spec):
    room = api.Room.from_spec(spec)
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.standard_normal(spec.n_in).astype(np.float32)).cuda()
    v = torch.from_numpy(rng.standard_normal(spec.n_in).astype(np.float32)).cuda()
    y = api.synthesize([room], [x])[0][0]
    dx = api.synthesize_backward([room], [x], [v[None]], want_params=False, want_beta=False)[0][0]
    lhs = float(torch.dot(y.double(), v.double()))
    rhs = float(torch.dot(x.double(), dx.double()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def _cs_case(spec, ids, n_out=None):
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    n_out = spec.n_in if n_out is None else n_out
    target = np.random.default_rng(3).standard_normal(n_out) * 0.01
    y_ref = oracle.synthesize(sc, x, n_out)
    _, dp, db = _bwd(spec, y_ref - target, want_dx=False)
    g_cs = oracle.loss_grad_cs(sc, x, target, ids + [48, 49, 50, 51, 52, 53])
    got = np.concatenate([dp[ids], db])
    assert np.linalg.norm(got - g_cs) <= 1e-4 * np.linalg.norm(g_cs), (got, g_cs)
    # per component: 1e-3 relative, above a floor of 2e-5 of the largest
    # component (the FP32 sums' rounding where a component cancels)
    scale = np.max(np.abs(g_cs))
    assert np.all(np.abs(got - g_cs) <= 1e-3 * np.abs(g_cs) + 2e-5 * scale), (got, g_cs)


@pytest.mark.parametrize("kw,Q,ids", [
    (dict(seed=41, K=2, seconds=0.03, traj_kind=W.SPLINE, tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)]), 4,
     [0, 1, 2, 4, 7, 11]),
    (dict(seed=42, K=2, seconds=0.05, traj_kind=W.CIRCLE, tiers=[(W.RHO_INF, 200.0, 20)]), 6, [0, 1, 3, 4, 5]),
    (dict(seed=43, K=2, seconds=0.03, traj_kind=W.SPLINE, window=W.KAISER,
          tiers=[(0, 16000.0), (2, 2000.0, 4), (W.RHO_INF, 500.0, 16)]), 2, [0, 3, 5, 8, 10]),
])
def test_upsampled_param_and_beta_gradients_match_complex_step(kw, Q, ids):
    _cs_case(_bl(kw, Q), ids)


@pytest.mark.parametrize("kw,ids", [
    (dict(seed=51, K=2, seconds=0.03, traj_kind=W.SPLINE), [0, 1, 2, 4, 7, 11]),
    (dict(seed=52, K=2, seconds=0.03, traj_kind=W.CIRCLE), [0, 1, 3, 4, 5]),
    (dict(seed=53, K=2, seconds=0.03, traj_kind=W.LINE), [0, 1, 2, 3, 6]),
    (dict(seed=54, K=2, seconds=0.1, window=W.KAISER, traj_kind=W.SPLINE,
          tiers=[(1, 16000.0), (W.RHO_INF, 16000.0 / 12)]), [0, 3, 5, 8, 10]),
])
def test_emission_time_param_and_beta_gradients_match_complex_step(kw, ids):
    _cs_case(_ret(kw), ids)


@pytest.mark.parametrize("which", ["upsampled", "emission-time"])
def test_gradients_with_a_shorter_output(which):
    if which == "upsampled":
        spec = _bl(dict(seed=44, K=2, seconds=0.04, traj_kind=W.SPLINE, tiers=[(1, 16000.0), (W.RHO_INF, 500.0, 8)]), 4)
    else:
        spec = _ret(dict(seed=45, K=2, seconds=0.04, traj_kind=W.CIRCLE))
    ids = [0, 1, 4] if which == "upsampled" else [0, 1, 3, 4]
    _cs_case(spec, ids, n_out=spec.n_in // 2 + 3)


def test_emission_time_moving_array_gradients():
    spec = _ret(dict(seed=55, K=2, seconds=0.03, traj_kind=W.SPLINE))
    spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=[0.0, 0.0, 0.0, 0.1, 0.5, 0.3], arr_duration=spec.duration)
    _cs_case(spec, [0, 1, 5, 9])


def _fd(f, h):
    # central differences at h and h/2 with Richardson extrapolation
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("variant", ["upsampled", "emission-time"])
def test_differentiation_scene_vs_oracle_finite_differences(variant):
    # The first differentiation scene's room, path and signal (6x5x3 m, 2 s at
    # 16 kHz, 6 control points) at order 4, with its last tier on 200 Hz knots
    # upsampled x8 (records every 10 samples), or with emission-time delays.
    # Loss 0.5 sum over 120 sampled outputs of (y - y*)^2 with the scene's
    # target. Reference: FP64 oracle central differences (h = 1e-3 m, 1e-4)
    # with Richardson extrapolation.
    spec, target = W.config4_scene(0)
    spec = replace(spec, K=4)
    if variant == "upsampled":
        spec = replace(spec, tiers=[(1, 16000.0), (W.RHO_INF, 200.0, 8)], up_halfwidth=4)
    else:
        spec = replace(spec, delay_model=1)
    sc = oracle_scene(spec)
    x = spec.x.astype(np.float64)
    idx = np.linspace(0, spec.n_in - 1, 120).astype(np.int64)

    def oloss(traj=None, beta=None):
        s2 = replace(sc, traj=traj if traj is not None else sc.traj, beta=beta if beta is not None else sc.beta)
        return 0.5 * float(np.sum((oracle.y_at(s2, x, idx) - target[idx]) ** 2))

    dy = np.zeros(spec.n_in)
    dy[idx] = oracle.y_at(sc, x, idx) - target[idx]
    _, dp, db = _bwd(spec, dy, want_dx=False)
    for pid in (1, 13):
        def f(dlt, pid=pid):
            tr = list(sc.traj)
            tr[pid] += dlt
            return oloss(traj=tr)
        ref = _fd(f, 1e-3)
        assert abs(dp[pid] - ref) <= 1e-4 * abs(ref), (pid, dp[pid], ref)

    def fb(dlt):
        bt = list(sc.beta)
        bt[0] += dlt
        return oloss(beta=tuple(bt))
    ref = _fd(fb, 1e-4)
    assert abs(db[0] - ref) <= 1e-4 * abs(ref), (db[0], ref)


def test_batch_mixing_delay_kinds_equals_single_and_reproducible():
    specs = [replace(W.small_scene(seed=60, K=3, seconds=0.05), taps=32),
             replace(_bl(*BL[0]), taps=32),
             replace(_ret(RET[0]), taps=32)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    dys = [torch.randn(1, s.n_in, device="cuda") for s in specs]
    batched = api.synthesize_backward(rooms, xs, dys)
    again = api.synthesize_backward(rooms, xs, dys)
    for i in range(len(specs)):
        single = api.synthesize_backward([rooms[i]], [xs[i]], [dys[i]])[0]
        for a, b, c in zip(batched[i], single, again[i]):
            assert torch.equal(a, b) and torch.equal(a, c), specs[i].name


@pytest.mark.parametrize("which", ["upsampled", "emission-time"])
@pytest.mark.parametrize("n_out_kind", ["shorter", "longer", "direct-path-only"])
def test_output_lengths_and_free_field(which, n_out_kind):
    # outputs shorter and longer than the input (the knots past the input's end,
    # a last tile that is partly empty) and a scene of the direct path alone
    # (order 0), against the oracle's transpose
    kw = dict(BL[0][0]) if which == "upsampled" else dict(RET[0])
    if n_out_kind == "direct-path-only":
        kw["K"] = 0
    spec = _bl(kw, BL[0][1]) if which == "upsampled" else _ret(kw)
    n_out = {"shorter": spec.n_in // 2 + 1, "longer": spec.n_in + 700, "direct-path-only": spec.n_in}[n_out_kind]
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    dy = np.random.default_rng(77).standard_normal((1, n_out))
    ws = api.Workspace()
    dx = api.synthesize_backward([room], [x], [torch.from_numpy(dy.astype(np.float32)).cuda()], want_params=False,
                                 want_beta=False, workspace=ws)[0][0]
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    ref = oracle.adjoint_x(oracle_scene(spec), dy[0], spec.n_in)
    assert rel_l2(dx.cpu().numpy().astype(np.float64), ref) < 1e-5


def _random_option_spec(i):
    # a small random scene with band-limited tiers or emission-time delays:
    # random trajectory kind, window, taps, tier layout (U, Q), microphones and
    # array motion, for the complex-step comparison
    rng = np.random.default_rng(9500 + i)
    retarded = bool(i % 2)
    fs = float(rng.choice([16000.0, 22050.0, 48000.0]))
    kind = int(rng.choice([W.LINE, W.CIRCLE, W.SPLINE]))
    tiers = []
    for b in sorted(rng.choice(np.arange(0, 3), size=1, replace=False).tolist()) + [W.RHO_INF]:
        if not retarded and (b == W.RHO_INF or rng.random() < 0.5):  # the last tier upsampled
            U = int(rng.choice([2, 4, 8]))
            M = int(rng.choice([2, 4, 6]))
            tiers.append((b, fs / (U * M), U))
        else:
            tiers.append((b, fs / int(rng.choice([1, 4, 12, 32]))))
    spec = W.small_scene(seed=600 + i, K=int(rng.integers(1, 3)), fs=fs, seconds=float(rng.uniform(0.02, 0.035)),
                         traj_kind=kind, window=int(rng.choice([W.HANN, W.KAISER])),
                         taps=int(rng.choice([16, 32])), tiers=tiers)
    spec = replace(spec, delay_model=1 if retarded else 0, up_halfwidth=int(rng.choice([2, 4])))
    if rng.random() < 0.4:
        d = rng.standard_normal(3)
        spec = replace(spec, arr_kind=W.LINE, arr_traj=[0.0, 0.0, 0.0] + list(d) + [0.3], arr_duration=spec.duration)
    return spec


@pytest.mark.parametrize("i", range(6))
def test_random_option_scene_gradients_match_complex_step(i):
    spec = _random_option_spec(i)
    ids = {W.LINE: [0, 1, 2, 6], W.CIRCLE: [0, 1, 3, 4, 5], W.SPLINE: [0, 1, 4, 8]}[spec.traj_kind]
    _cs_case(spec, ids)
