"""Allocation-free entry point (msrc_synthesize_noalloc) against msrc_synthesize.

msrc_synthesize_noalloc is for callers that may not allocate device memory (a
plug-in whose host application owns the device pool, a real-time audio
thread): it runs the same synthesis in a fixed scratch array inside the
library. This test calls it twice in a row through the C ABI and checks each
output against the ordinary entry point (caller workspace) within the parity
tolerance and the calls' device error word (msrc_noalloc_errors), that an
oversized scene is refused, and that a bounded wait that gives up inside an
allocation-free call is reported through that error word. The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2508_03065_gb300 import _lib, api
from paper_2508_03065_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _noalloc(lib, room, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.msrc_synthesize_noalloc(room.handle, ctypes.c_void_p(x.data_ptr()), x.numel(),
                                       ctypes.c_void_p(y.data_ptr()), y.shape[-1], stream)


def _errors(lib):
    flags = ctypes.c_uint32(0xFFFFFFFF)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.msrc_noalloc_errors(stream, ctypes.byref(flags))
    return st, int(flags.value)


def _rel(a, b):
    a, b = a.double(), b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_workspace_path_twice():
    lib = _lib.load()
    specs = [W.small_scene(seed=50, K=4, seconds=0.15, n_mics=2),
             W.small_scene(seed=51, K=3, seconds=0.1, window=W.KAISER)]
    for spec in specs:
        room = api.Room.from_spec(spec)
        x = torch.from_numpy(spec.x).cuda()
        ref = api.synthesize([room], [x])[0].clone()
        for _ in range(2):
            y = torch.full((room.n_mics, spec.n_in), float("nan"), device="cuda")
            st = _noalloc(lib, room, x, y)
            assert st == _lib.OK, lib.msrc_last_error()
            torch.cuda.synchronize()
            assert _errors(lib) == (_lib.OK, 0)
            assert torch.isfinite(y).all()
            for m in range(room.n_mics):
                assert _rel(y[m], ref[m]) <= TOL


def test_noalloc_rejects_scene_beyond_scratch():
    lib = _lib.load()
    spec = W.config2()  # order 20, 4 s at 48 kHz: far above the fixed scratch
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    y = torch.zeros((1, spec.n_in), device="cuda")
    st = _noalloc(lib, room, x, y)
    assert st == _lib.ERR_WORKSPACE
    assert b"scratch" in lib.msrc_last_error()
    assert torch.count_nonzero(y) == 0


def test_noalloc_reports_a_wait_that_gave_up():
    # the test hook makes every window staging wait for bytes that never come:
    # the bounded wait gives up, and the allocation-free call's error word says so
    lib = _lib.load()
    spec = W.small_scene(seed=52, K=3, seconds=0.1)
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    y = torch.zeros((room.n_mics, spec.n_in), device="cuda")
    assert _noalloc(lib, room, x, y) == _lib.OK
    torch.cuda.synchronize()
    good = y.clone()
    assert _errors(lib) == (_lib.OK, 0)
    assert lib.msrc_test_stall_window_copies(16) == _lib.OK
    try:
        assert _noalloc(lib, room, x, y) == _lib.OK
        torch.cuda.synchronize()
    finally:
        assert lib.msrc_test_stall_window_copies(0) == _lib.OK
    st, flags = _errors(lib)
    assert st == _lib.ERR_TIMEOUT and flags & 1
    # read and cleared: the next call is clean and gives the same result
    assert _noalloc(lib, room, x, y) == _lib.OK
    torch.cuda.synchronize()
    assert _errors(lib) == (_lib.OK, 0)
    assert torch.equal(y, good)
