"""Python front end of the msrc library (PyTorch for device memory and streams).

    room = Room.from_spec(spec)                    # workloads.SceneSpec or keywords
    y = synthesize([room], [x_cuda])[0]            # (n_mics, n_out) float32 on the GPU

Every step of the synthesis runs in the library's CUDA kernels; this module only
marshals pointers, sizes and streams through the C ABI.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Room:
    """A shoebox room with its image-source settings, trajectory and microphones."""

    def __init__(self, dims, beta, fs, max_order, tiers, taps=32, window=0, kaiser_beta=8.0,
                 c=343.0, farrow_order=4, passband=0.9, upsample_halfwidth=4, delay_model=0):
        """tiers: (max reflection count, knot rate in Hz[, upsampling factor U]);
        U > 1 recovers the distance between knots band-limited (see
        msrc_room_desc.tier_upsample). window: 0 Hann- or 1 Kaiser-windowed sinc
        taps, 2 a least-squares Farrow design of order `farrow_order` fitted up
        to `passband` * pi. delay_model: 0 distance at the reception time, 1
        emission-time (retarded) path length (see msrc_room_desc.delay_model)."""
        lib = _lib.load()
        d = _lib.RoomDesc()
        d.dims[:] = [float(v) for v in dims]
        d.beta[:] = [float(v) for v in beta]
        d.c = float(c)
        d.fs = float(fs)
        d.max_order = int(max_order)
        d.n_tiers = len(tiers)
        rho = [0] * 4
        rate = [1.0] * 4
        up = [1] * 4
        for t, tier in enumerate(tiers):
            rho[t] = int(min(tier[0], 2**31 - 1))
            rate[t] = float(tier[1])
            up[t] = int(tier[2]) if len(tier) > 2 else 1
        d.tier_max_rho[:] = rho
        d.tier_rate_hz[:] = rate
        d.tier_upsample[:] = up
        d.upsample_halfwidth = int(upsample_halfwidth)
        d.delay_model = int(delay_model)
        d.taps = int(taps)
        d.window = int(window)
        d.kaiser_beta = float(kaiser_beta)
        d.farrow_order = int(farrow_order)
        d.passband = float(passband)
        self._desc = d
        h = ctypes.c_void_p()
        _lib.check(lib.msrc_create_room(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n_mics = 0
        self.fs = float(fs)

    @classmethod
    def from_spec(cls, spec) -> "Room":
        room = cls(spec.dims, spec.beta, spec.fs, spec.K, spec.tiers, spec.taps, spec.window,
                   spec.kaiser_beta, spec.c, spec.farrow_order, spec.passband,
                   getattr(spec, "up_halfwidth", 4), getattr(spec, "delay_model", 0))
        room.set_trajectory(spec.traj_kind, spec.traj, spec.duration, spec.mics, spec.n_ctrl)
        if getattr(spec, "arr_kind", -1) >= 0:
            room.set_array_trajectory(spec.arr_kind, spec.arr_traj, spec.arr_duration, spec.arr_n_ctrl)
        return room

    def set_trajectory(self, kind: int, params: Sequence[float], duration: float, mics,
                       n_ctrl: int = 0) -> None:
        lib = _lib.load()
        t = _lib.TrajDesc()
        t.kind = int(kind)
        t.n_ctrl = int(n_ctrl)
        p = [0.0] * 48
        p[: len(params)] = [float(v) for v in params]
        t.params[:] = p
        t.duration_s = float(duration)
        m = np.ascontiguousarray(np.asarray(mics, np.float64).reshape(-1, 3))
        _lib.check(lib.msrc_set_trajectory(self._h, ctypes.byref(t),
                                           m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           int(m.shape[0])))
        self.n_mics = int(m.shape[0])
        self.traj_kind, self.n_ctrl, self.duration = int(kind), int(n_ctrl), float(duration)
        self.mics = m.copy()
        self.params = np.array(p, np.float64)

    def set_array_trajectory(self, kind: Optional[int], params: Sequence[float] = (), duration: float = 1.0,
                             n_ctrl: int = 0) -> None:
        """Moves the microphones rigidly along a trajectory a(t): microphone m
        sits at its set_trajectory position + a(t) - a(0). kind=None makes
        the array static again."""
        lib = _lib.load()
        if kind is None:
            _lib.check(lib.msrc_set_array_trajectory(self._h, None))
            return
        t = _lib.TrajDesc()
        t.kind = int(kind)
        t.n_ctrl = int(n_ctrl)
        p = [0.0] * 48
        p[: len(params)] = [float(v) for v in params]
        t.params[:] = p
        t.duration_s = float(duration)
        _lib.check(lib.msrc_set_array_trajectory(self._h, ctypes.byref(t)))

    def positions(self, times) -> np.ndarray:
        """Source positions (n x 3) of the trajectory at the given times (s)."""
        lib = _lib.load()
        t = np.ascontiguousarray(np.asarray(times, np.float64).reshape(-1))
        out = np.zeros((t.size, 3), np.float64)
        _lib.check(lib.msrc_trajectory_positions(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 t.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def suggest_knot_rates(self, tol_samples: float, max_step: int = 4096) -> list:
        """Per tier, the lowest knot rate (Hz, fs / integer) whose linear
        interpolation keeps every image delay within tol_samples (see
        msrc_suggest_knot_rates)."""
        lib = _lib.load()
        out = (ctypes.c_double * 4)()
        _lib.check(lib.msrc_suggest_knot_rates(self._h, float(tol_samples), int(max_step), out))
        return [float(out[t]) for t in range(self._desc.n_tiers)]

    def suggest_bandlimited_rates(self, tol_samples: float) -> list:
        """Per tier, the lowest knot rate (Hz, fs / integer) at which the
        band-limited upsampler reproduces the delays of the tier's nearest
        images within tol_samples (see msrc_suggest_bandlimited_rates)."""
        lib = _lib.load()
        out = (ctypes.c_double * 4)()
        _lib.check(lib.msrc_suggest_bandlimited_rates(self._h, float(tol_samples), out))
        return [float(out[t]) for t in range(self._desc.n_tiers)]

    def set_reflection(self, beta) -> None:
        lib = _lib.load()
        b = np.ascontiguousarray(np.asarray(beta, np.float64).reshape(6))
        _lib.check(lib.msrc_set_reflection(self._h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        self._desc.beta[:] = [float(v) for v in b]

    @property
    def handle(self):
        return self._h

    def image_count(self):
        lib = _lib.load()
        cnt = ctypes.c_int64()
        per = (ctypes.c_int64 * 4)()
        _lib.check(lib.msrc_room_image_count(self._h, ctypes.byref(cnt), per))
        return int(cnt.value), [int(v) for v in per[: self._desc.n_tiers]]

    def fit_error(self) -> float:
        lib = _lib.load()
        e = ctypes.c_double()
        _lib.check(lib.msrc_room_fit_error(self._h, ctypes.byref(e)))
        return float(e.value)

    def farrow_table(self, which: int = 0) -> np.ndarray:
        """The Farrow table the kernels use, shape (4 segments, P powers, taps):
        h(k; alpha) = sum_q table[s, q, k + L/2] w^q with s = floor(4 alpha),
        w = 4 alpha - s - 1/2 (which 0: synthesis, P = 5; 1: gradient, P = 6)."""
        lib = _lib.load()
        L = int(self._desc.taps)
        out = np.zeros(4 * 6 * L, np.float32)
        P = ctypes.c_int32()
        _lib.check(lib.msrc_room_farrow_table(self._h, int(which), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              ctypes.byref(P)))
        return out[:4 * P.value * L].reshape(4, P.value, L).copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.msrc_destroy_room(h)
            self._h = None


class Workspace:
    """Grow-only device workspace (a torch uint8 buffer, 256-byte aligned)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.buf: Optional[torch.Tensor] = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        return self.buf


_default_ws = {}


def _workspace(device) -> Workspace:
    key = str(torch.device(device))
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def _cfg(tile_config: Optional[int]) -> int:
    return _lib.TILE_DEFAULT if tile_config is None else int(tile_config)


def workspace_size(rooms: Sequence[Room], n_in: Sequence[int], n_out: Sequence[int], backward: bool = False,
                   tile_config: Optional[int] = None):
    """(forward bytes in the tile configuration `tile_config` (None = the
    process default), reverse-mode bytes or 0 unless `backward`)."""
    lib = _lib.load()
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    fwd, bwd = ctypes.c_size_t(), ctypes.c_size_t()
    _lib.check(lib.msrc_workspace_size_cfg(hs, len(rooms), _lib.i64_array(n_in), _lib.i64_array(n_out),
                                           _cfg(tile_config), ctypes.byref(fwd),
                                           ctypes.byref(bwd) if backward else None))
    return int(fwd.value), int(bwd.value)


def synthesize(rooms: Sequence[Room], xs: Sequence[torch.Tensor], n_out: Optional[Sequence[int]] = None,
               out: Optional[Sequence[torch.Tensor]] = None, workspace: Optional[Workspace] = None,
               stream: Optional[torch.cuda.Stream] = None, tile_config: Optional[int] = None) -> List[torch.Tensor]:
    """Forward synthesis (Eq. 8) of every room; returns (n_mics, n_out) float32
    tensors. tile_config: a synthesis tile configuration for this call (e.g.
    autotune's pick), None = the process default."""
    lib = _lib.load()
    if len(rooms) != len(xs) or len(rooms) == 0:
        raise ValueError("need one signal per room")
    xs = [x.contiguous() for x in xs]
    for x in xs:
        if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 1:
            raise ValueError("signals must be 1-D float32 CUDA tensors")
    n_in = [int(x.numel()) for x in xs]
    n_out = list(n_in) if n_out is None else [int(v) for v in n_out]
    dev = xs[0].device
    if out is None:
        out = [torch.empty((r.n_mics, no), dtype=torch.float32, device=dev) for r, no in zip(rooms, n_out)]
    ws = workspace or _workspace(dev)
    fwd, _ = workspace_size(rooms, n_in, n_out, tile_config=tile_config)
    buf = ws.get(fwd)
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    _lib.check(lib.msrc_synthesize_cfg(hs, len(rooms), _lib.ptr_array([x.data_ptr() for x in xs]),
                                       _lib.i64_array(n_in), _lib.ptr_array([y.data_ptr() for y in out]),
                                       _lib.i64_array(n_out), _cfg(tile_config), ctypes.c_void_p(buf.data_ptr()),
                                       buf.numel(), _stream_handle(stream)))
    return list(out)


def synthesize_host(rooms: Sequence[Room], xs_host: Sequence[torch.Tensor], ys_host: Sequence[torch.Tensor],
                    workspace: Optional[Workspace] = None, stream: Optional[torch.cuda.Stream] = None,
                    device="cuda") -> None:
    """Same as synthesize() with host (ideally pinned) buffers; the copies in
    both directions are enqueued by the library on `stream`. The caller
    synchronises before reading ys_host."""
    lib = _lib.load()
    n_in = [int(x.numel()) for x in xs_host]
    n_out = [int(y.shape[-1]) for y in ys_host]
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    fwd, _ = workspace_size(rooms, n_in, n_out)
    io = ctypes.c_size_t()
    _lib.check(lib.msrc_host_io_bytes(hs, len(rooms), _lib.i64_array(n_in), _lib.i64_array(n_out),
                                      ctypes.byref(io)))
    ws = workspace or _workspace(device)
    buf = ws.get(fwd + int(io.value))
    _lib.check(lib.msrc_synthesize_host(hs, len(rooms), _lib.ptr_array([x.data_ptr() for x in xs_host]),
                                        _lib.i64_array(n_in), _lib.ptr_array([y.data_ptr() for y in ys_host]),
                                        _lib.i64_array(n_out), ctypes.c_void_p(buf.data_ptr()),
                                        buf.numel(), _stream_handle(stream)))


def workspace_errors(workspace: Workspace, stream: Optional[torch.cuda.Stream] = None) -> int:
    lib = _lib.load()
    flags = ctypes.c_uint32()
    st = lib.msrc_workspace_errors(ctypes.c_void_p(workspace.buf.data_ptr()), _stream_handle(stream),
                                   ctypes.byref(flags))
    if st not in (_lib.OK, _lib.ERR_TIMEOUT):
        _lib.check(st)
    return int(flags.value)


def measure_alu_peaks(stream: Optional[torch.cuda.Stream] = None):
    """(FP32, FP64) fused multiply-add peaks of the current GPU in TFLOP/s,
    measured (see msrc_measure_alu_peaks)."""
    scratch = torch.empty(16, dtype=torch.uint8, device="cuda")
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().msrc_measure_alu_peaks(ctypes.c_void_p(scratch.data_ptr()), _stream_handle(stream),
                                                   ctypes.byref(f32), ctypes.byref(f64)))
    return float(f32.value), float(f64.value)


def set_tile_config(cfg: int) -> None:
    """Sets the process default tile configuration (calls with tile_config=None)."""
    _lib.check(_lib.load().msrc_set_tile_config(int(cfg)))


def tile_configs() -> int:
    return int(_lib.load().msrc_tile_configs())


def profile_enable(on: bool = True) -> None:
    _lib.check(_lib.load().msrc_profile_enable(1 if on else 0))


def profile_read():
    """Milliseconds per phase (setup, prefilter, synthesis, reduction) summed over
    the calls since the last read, and the number of calls."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int32()
    _lib.check(_lib.load().msrc_profile_read(ms, ctypes.byref(n)))
    return [float(v) for v in ms], int(n.value)


def synthesize_backward(rooms: Sequence[Room], xs: Sequence[torch.Tensor], dys: Sequence[torch.Tensor],
                        want_dx: bool = True, want_params: bool = True, want_beta: bool = True,
                        workspace: Optional[Workspace] = None, stream: Optional[torch.cuda.Stream] = None,
                        want_array: bool = False):
    """Reverse mode of synthesize(): for upstream gradients dys[r] of shape
    (n_mics, n_out) returns, per room, (dx, dparams, dbeta): dL/dx (float32,
    n_in), dL/d trajectory parameters (float64, 48, laid out like the
    trajectory parameters) and dL/d wall reflection coefficients (float64, 6),
    each None when not requested. With want_array, a fourth entry: dL/d of the
    microphone array's trajectory parameters (float64, 48; zeros for a room
    without array motion)."""
    lib = _lib.load()
    xs = [x.contiguous() for x in xs]
    dys = [d.contiguous().float() for d in dys]
    n_in = [int(x.numel()) for x in xs]
    n_out = [int(d.shape[-1]) for d in dys]
    dev = xs[0].device
    dx = [torch.empty(n, dtype=torch.float32, device=dev) for n in n_in] if want_dx else None
    dp = [torch.zeros(48, dtype=torch.float64, device=dev) for _ in rooms] if want_params else None
    db = [torch.zeros(6, dtype=torch.float64, device=dev) for _ in rooms] if want_beta else None
    da = [torch.zeros(48, dtype=torch.float64, device=dev) for _ in rooms] if want_array else None
    _, bwd = workspace_size(rooms, n_in, n_out, backward=True)
    ws = workspace or _workspace(dev)
    buf = ws.get(bwd)
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    arr = lambda ts: _lib.ptr_array([t.data_ptr() for t in ts]) if ts is not None else None  # noqa: E731
    _lib.check(lib.msrc_synthesize_backward_ex(hs, len(rooms), arr(xs), _lib.i64_array(n_in), arr(dys),
                                               _lib.i64_array(n_out), arr(dx), arr(dp), arr(db), arr(da),
                                               ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                                               _stream_handle(stream)))
    out = []
    for r in range(len(rooms)):
        row = (dx[r] if dx else None, dp[r] if dp else None, db[r] if db else None)
        out.append(row + (da[r],) if want_array else row)
    return out


class MovingSourceSynthesis(torch.autograd.Function):
    """y = synthesis(x; trajectory parameters, wall coefficients) with gradients
    for all three. `params` (48) and `beta` (6) are float64 tensors; the room
    keeps its geometry, tiers, taps and microphones."""

    @staticmethod
    def forward(ctx, x, params, beta, room: Room):
        p = params.detach().cpu().numpy().astype(np.float64)
        room.set_trajectory(room.traj_kind, p, room.duration, room.mics, room.n_ctrl)
        room.set_reflection(beta.detach().cpu().numpy())
        y = synthesize([room], [x.detach().float()])[0]
        ctx.room = room
        ctx.save_for_backward(x)
        ctx.params_device, ctx.beta_device = params.device, beta.device
        return y

    @staticmethod
    def backward(ctx, dy):
        (x,) = ctx.saved_tensors
        need_x, need_p, need_b = ctx.needs_input_grad[:3]
        dx, dp, db = synthesize_backward([ctx.room], [x.detach().float()], [dy], want_dx=need_x,
                                         want_params=need_p, want_beta=need_b)[0]
        return (dx if need_x else None, dp.to(ctx.params_device) if need_p else None,
                db.to(ctx.beta_device) if need_b else None, None)


def synthesize_ad(room: Room, x: torch.Tensor, params: torch.Tensor, beta: torch.Tensor) -> torch.Tensor:
    """Differentiable forward synthesis of one room (see MovingSourceSynthesis)."""
    return MovingSourceSynthesis.apply(x, params, beta, room)


class Batch:
    """A planned batched synthesis (msrc_batch_*): descriptors uploaded once,
    kernels only per run, optionally replayed from a captured CUDA graph.
    Signals and outputs are bound at creation; tile_config (None = the
    process default) is frozen then too."""

    def __init__(self, rooms: Sequence[Room], xs: Sequence[torch.Tensor], n_out: Optional[Sequence[int]] = None,
                 stream: Optional[torch.cuda.Stream] = None, tile_config: Optional[int] = None):
        lib = _lib.load()
        self.rooms = list(rooms)
        self.xs = [x.contiguous() for x in xs]
        self.n_in = [int(x.numel()) for x in self.xs]
        self.n_out = list(self.n_in) if n_out is None else [int(v) for v in n_out]
        dev = self.xs[0].device
        self.ys = [torch.empty((r.n_mics, no), dtype=torch.float32, device=dev)
                   for r, no in zip(self.rooms, self.n_out)]
        fwd, _ = workspace_size(self.rooms, self.n_in, self.n_out, tile_config=tile_config)
        self.ws = torch.empty(fwd, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        h = ctypes.c_void_p()
        hs = _lib.ptr_array([r.handle.value for r in self.rooms])
        _lib.check(lib.msrc_batch_create_cfg(hs, len(self.rooms), _lib.ptr_array([x.data_ptr() for x in self.xs]),
                                             _lib.i64_array(self.n_in),
                                             _lib.ptr_array([y.data_ptr() for y in self.ys]),
                                             _lib.i64_array(self.n_out), _cfg(tile_config),
                                             ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                             _stream_handle(self.stream), ctypes.byref(h)))
        self._h = h

    def run(self, use_graph: bool = True) -> List[torch.Tensor]:
        _lib.check(_lib.load().msrc_batch_run(self._h, 1 if use_graph else 0, _stream_handle(self.stream)))
        return self.ys

    def work(self) -> int:
        """Image-samples per run (images x output samples x microphones)."""
        return sum(r.image_count()[0] * no * r.n_mics for r, no in zip(self.rooms, self.n_out))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.msrc_batch_destroy(h)
            self._h = None


def autotune(rooms: Sequence[Room], xs: Sequence[torch.Tensor], n_out: Optional[Sequence[int]] = None,
             reps: int = 3, cache_path: Optional[str] = None, stream: Optional[torch.cuda.Stream] = None) -> int:
    """The fastest synthesis tile configuration for this workload (pass it as
    tile_config to synthesize / Batch), cached in a JSON file
    (MSRC_AUTOTUNE_CACHE, else ~/.cache/msrc_autotune.json) keyed by GPU and
    workload shape. The process default is left as it is."""
    import json
    import os

    lib = _lib.load()
    xs = [x.contiguous() for x in xs]
    n_in = [int(x.numel()) for x in xs]
    n_out = list(n_in) if n_out is None else [int(v) for v in n_out]
    dev = xs[0].device
    # the work's shape: images, lengths, taps and the per-tier knot layout and
    # delay model that decide the record prologue
    key = json.dumps([torch.cuda.get_device_name(dev), len(rooms),
                      sum(r.image_count()[0] for r in rooms), sum(n_out), sum(n_in),
                      sorted({int(r._desc.taps) for r in rooms}),
                      sorted({(int(r._desc.delay_model), tuple(float(v) for v in r._desc.tier_rate_hz),
                               tuple(int(v) for v in r._desc.tier_upsample)) for r in rooms})])
    path = cache_path or os.environ.get("MSRC_AUTOTUNE_CACHE") or os.path.expanduser("~/.cache/msrc_autotune.json")
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return int(cache[key]["best"])
    ys = [torch.empty((r.n_mics, no), dtype=torch.float32, device=dev) for r, no in zip(rooms, n_out)]
    need = 0
    for c in range(tile_configs()):
        need = max(need, workspace_size(rooms, n_in, n_out, tile_config=c)[0])
    ws = _workspace(dev).get(need)
    ms = (ctypes.c_double * tile_configs())()
    best = ctypes.c_int32()
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    _lib.check(lib.msrc_autotune(hs, len(rooms), _lib.ptr_array([x.data_ptr() for x in xs]), _lib.i64_array(n_in),
                                 _lib.ptr_array([y.data_ptr() for y in ys]), _lib.i64_array(n_out),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream), int(reps), ms,
                                 ctypes.byref(best)))
    cache[key] = {"best": int(best.value), "ms": [float(v) for v in ms]}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return int(best.value)
