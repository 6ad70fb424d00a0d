"""Static-response splicing: the conventional way of simulating a moving source,
against which the paper's first experiment (Sec. III) compares the method.

The source is frozen at positions sampled along its path at a frame rate (25 Hz
in that comparison); each frame's output comes from the static image-source
synthesis of the frozen source, and consecutive frames are either switched
hard at the frame boundary or cross-faded linearly over the frame. Every static
synthesis runs in this library's kernels (one batched call over all frames);
only the frame assembly is elementwise tensor arithmetic.

Frame f starts at sample f*Nf (Nf = fs / frame_rate) with the source at
s(f*Nf/fs). With P >= (largest delay) + L/2 + Nf samples of lead-in, the
static output of frame f on [f*Nf - P + Nf, (f+1)*Nf) depends only on the
signal, so frame f is an independent scene whose input is the signal from
f*Nf - P + ... (zero before the start).
"""
from __future__ import annotations

import math
from dataclasses import replace
from typing import Optional

import numpy as np
import torch

from . import api

LINE = 0


def delay_bound(spec) -> int:
    """Samples of the largest image delay of the room: every image of order K
    lies within 2 K max(L) + 2 |room diagonal| of the microphone (plus 1 m)."""
    dmax = 2.0 * spec.K * max(spec.dims) + 2.0 * math.sqrt(sum(d * d for d in spec.dims)) + 1.0
    return int(math.ceil(dmax * spec.fs / spec.c)) + 2


def static_splice(spec, x: torch.Tensor, frame_rate: float = 25.0, crossfade: bool = True,
                  n_out: Optional[int] = None) -> torch.Tensor:
    """Spliced static responses for the scene `spec` (a workloads.SceneSpec
    with a still microphone array) and the signal x (1-D float32 CUDA tensor).
    Returns (n_mics, n_out) on x's device."""
    if getattr(spec, "arr_kind", -1) >= 0:
        raise ValueError("static splicing needs still microphones")
    n = int(x.numel())
    n_out = n if n_out is None else int(n_out)
    nf = int(round(spec.fs / frame_rate))
    if nf < 1:
        raise ValueError("frame rate above the sample rate")
    frames = (n_out + nf - 1) // nf + 1
    lead = delay_bound(spec) + spec.taps // 2 + nf
    path = api.Room.from_spec(spec)
    pos = path.positions(np.arange(frames) * nf / spec.fs)
    rooms = []
    for f in range(frames):
        still = replace(spec, traj_kind=LINE, traj=list(pos[f]) + [1.0, 0.0, 0.0, 0.0], n_ctrl=0)
        rooms.append(api.Room.from_spec(still))
    pad = torch.zeros(lead + frames * nf + nf, dtype=torch.float32, device=x.device)
    pad[lead:lead + n] = x
    # frame f's scene: input pad[f*nf : f*nf + lead + nf], i.e. the signal from
    # f*nf - lead; its output index j is the sample f*nf - lead + j
    xs = [pad[f * nf: f * nf + lead + nf] for f in range(frames)]
    ys = api.synthesize(rooms, xs, n_out=[lead + nf] * frames)
    n_mics = ys[0].shape[0]
    out = torch.empty((n_mics, frames * nf), dtype=torch.float32, device=x.device)
    lam = torch.arange(nf, dtype=torch.float32, device=x.device) / nf
    for f in range(frames - 1):
        cur = ys[f][:, lead: lead + nf]                       # samples f*nf .. f*nf + nf - 1
        if crossfade:
            nxt = ys[f + 1][:, lead - nf: lead]               # the same samples from frame f + 1
            out[:, f * nf:(f + 1) * nf] = (1.0 - lam) * cur + lam * nxt
        else:
            out[:, f * nf:(f + 1) * nf] = cur
    out[:, (frames - 1) * nf:] = ys[frames - 1][:, lead: lead + nf]
    return out[:, :n_out]
