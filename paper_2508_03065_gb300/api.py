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
                 c=343.0):
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
        for t, (r, hz) in enumerate(tiers):
            rho[t] = int(min(r, 2**31 - 1))
            rate[t] = float(hz)
        d.tier_max_rho[:] = rho
        d.tier_rate_hz[:] = rate
        d.taps = int(taps)
        d.window = int(window)
        d.kaiser_beta = float(kaiser_beta)
        self._desc = d
        h = ctypes.c_void_p()
        _lib.check(lib.msrc_create_room(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n_mics = 0
        self.fs = float(fs)

    @classmethod
    def from_spec(cls, spec) -> "Room":
        room = cls(spec.dims, spec.beta, spec.fs, spec.K, spec.tiers, spec.taps, spec.window,
                   spec.kaiser_beta, spec.c)
        room.set_trajectory(spec.traj_kind, spec.traj, spec.duration, spec.mics, spec.n_ctrl)
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


def workspace_size(rooms: Sequence[Room], n_in: Sequence[int], n_out: Sequence[int]):
    lib = _lib.load()
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    fwd, bwd = ctypes.c_size_t(), ctypes.c_size_t()
    _lib.check(lib.msrc_workspace_size(hs, len(rooms), _lib.i64_array(n_in), _lib.i64_array(n_out),
                                       ctypes.byref(fwd), ctypes.byref(bwd)))
    return int(fwd.value), int(bwd.value)


def synthesize(rooms: Sequence[Room], xs: Sequence[torch.Tensor], n_out: Optional[Sequence[int]] = None,
               out: Optional[Sequence[torch.Tensor]] = None, workspace: Optional[Workspace] = None,
               stream: Optional[torch.cuda.Stream] = None) -> List[torch.Tensor]:
    """Forward synthesis (Eq. 8) of every room; returns (n_mics, n_out) float32 tensors."""
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
    fwd, _ = workspace_size(rooms, n_in, n_out)
    buf = ws.get(fwd)
    hs = _lib.ptr_array([r.handle.value for r in rooms])
    _lib.check(lib.msrc_synthesize(hs, len(rooms), _lib.ptr_array([x.data_ptr() for x in xs]),
                                   _lib.i64_array(n_in), _lib.ptr_array([y.data_ptr() for y in out]),
                                   _lib.i64_array(n_out), ctypes.c_void_p(buf.data_ptr()),
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


def set_tile_config(cfg: int) -> None:
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
