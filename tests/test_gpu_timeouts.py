"""The bounded waits give up, report and leave the context usable.

With the test hook msrc_test_stall_window_copies, every shared-window staging
waits for 16 bytes that no copy delivers: the mbarrier wait runs out after
about one second, each block records the timeout bit in the workspace's error
word and stops. Checked for the synthesis and the reverse-mode gradient kernel:
the launch returns within seconds, msrc_workspace_errors reports bit 1 (and
MSRC_ERR_TIMEOUT), and the next call on the same context and workspace gives
the same result as before, bit for bit.
"""
import time

import numpy as np
import pytest
import torch

from paper_2508_03065_gb300 import _lib, api
from paper_2508_03065_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _stalled(fn):
    lib = _lib.load()
    assert lib.msrc_test_stall_window_copies(16) == _lib.OK
    try:
        t0 = time.time()
        fn()
        torch.cuda.synchronize()
        return time.time() - t0
    finally:
        assert lib.msrc_test_stall_window_copies(0) == _lib.OK


def test_synthesis_wait_times_out_and_context_survives():
    spec = W.small_scene(seed=3, K=3)
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    ws = api.Workspace()
    good = api.synthesize([room], [x], workspace=ws)[0].clone()
    assert api.workspace_errors(ws) == 0
    elapsed = _stalled(lambda: api.synthesize([room], [x], workspace=ws))
    assert elapsed < 20.0
    assert api.workspace_errors(ws) & 1
    again = api.synthesize([room], [x], workspace=ws)[0]
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    assert torch.equal(again, good)


def test_gradient_wait_times_out_and_context_survives():
    spec = W.small_scene(seed=4, K=3)
    room = api.Room.from_spec(spec)
    x = torch.from_numpy(spec.x).cuda()
    dy = torch.from_numpy(np.random.default_rng(4).standard_normal((1, spec.n_in)).astype(np.float32)).cuda()
    ws = api.Workspace()
    good = api.synthesize_backward([room], [x], [dy], workspace=ws)[0]
    assert api.workspace_errors(ws) == 0
    elapsed = _stalled(lambda: api.synthesize_backward([room], [x], [dy], workspace=ws))
    assert elapsed < 20.0
    assert api.workspace_errors(ws) & 1
    again = api.synthesize_backward([room], [x], [dy], workspace=ws)[0]
    torch.cuda.synchronize()
    assert api.workspace_errors(ws) == 0
    for a, b in zip(again, good):
        assert torch.equal(a, b)
