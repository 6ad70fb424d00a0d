"""Static-response splicing (the comparison of the paper's first experiment,
Sec. III) on the GPU: parity with the same splicing built from the FP64 oracle,
and the experiment itself -- a 1 kHz tone from a source receding along a slow
curve, simulated by the method with 5 Hz knots and by 25 Hz splicing -- where
splicing shows phase and gain steps at its frame boundaries and the method
does not."""
import math
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api, motion_metrics, splicing
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2

pytestmark = pytest.mark.gpu


def _oracle_splice(spec, x, frame_rate, crossfade):
    # the same framing, every static response from the FP64 oracle
    n = x.size
    nf = int(round(spec.fs / frame_rate))
    frames = (n + nf - 1) // nf + 1
    dmax = 2.0 * spec.K * max(spec.dims) + 2.0 * math.sqrt(sum(d * d for d in spec.dims)) + 1.0
    lead = int(math.ceil(dmax * spec.fs / spec.c)) + 2 + spec.taps // 2 + nf
    pos = oracle.source_position(oracle_scene(spec), np.arange(frames) * nf / spec.fs)
    pad = np.zeros(lead + frames * nf + nf)
    pad[lead:lead + n] = x
    ys = [oracle.synthesize(oracle_scene(spec, traj_kind=0, traj=list(pos[f]) + [1.0, 0.0, 0.0, 0.0], n_ctrl=0),
                            pad[f * nf: f * nf + lead + nf], lead + nf) for f in range(frames)]
    out = np.zeros(frames * nf)
    lam = np.arange(nf) / nf
    for f in range(frames - 1):
        cur = ys[f][lead: lead + nf]
        out[f * nf:(f + 1) * nf] = (1 - lam) * cur + lam * ys[f + 1][lead - nf: lead] if crossfade else cur
    out[(frames - 1) * nf:] = ys[-1][lead: lead + nf]
    return out[:n]


@pytest.mark.parametrize("crossfade", [False, True])
def test_splicing_matches_oracle(crossfade):
    spec = W.small_scene(seed=30, K=2, seconds=0.1, traj_kind=W.LINE)
    y = splicing.static_splice(spec, torch.from_numpy(spec.x).cuda(), frame_rate=50.0, crossfade=crossfade)
    ref = _oracle_splice(spec, spec.x.astype(np.float64), 50.0, crossfade)
    assert rel_l2(y[0].cpu().numpy(), ref) < 1e-5


def test_first_experiment_steps():
    spec = W.receding_tone()
    fs, f0 = spec.fs, 1000.0
    xt = torch.from_numpy(spec.x).cuda()
    y_m = api.synthesize([api.Room.from_spec(spec)], [xt])[0][0].cpu().numpy()
    y_h = splicing.static_splice(spec, xt, frame_rate=25.0, crossfade=False)[0].cpu().numpy()
    frame = int(fs / 25.0)
    m = motion_metrics.continuity(y_m, fs, f0, frame, skip=3000)
    h = motion_metrics.continuity(y_h, fs, f0, frame, skip=3000)
    assert m["phase_step_rad"] < 0.02 and m["gain_step"] < 0.01
    assert h["phase_step_rad"] > 5 * max(m["phase_step_rad"], 1e-3)
    assert h["gain_step"] > 5 * max(m["gain_step"], 1e-4)
