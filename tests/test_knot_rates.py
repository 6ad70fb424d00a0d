"""Knot rates chosen from the motion (msrc_suggest_knot_rates; Sec. II-C:
dense knots for the direct sound and low orders, sparse for high orders).

Host only, no GPU. The suggested rates are checked against the FP64 oracle:
with them, linear interpolation between knots keeps every image's delay
within the requested tolerance of the dense (every-sample) delay.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import api as oracle
from paper_2508_03065_gb300 import api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene


def _max_delay_error(spec, rates):
    steps = [int(round(spec.fs / r)) for r in rates]
    tiered = oracle_scene(replace(spec, tiers=[(t[0], spec.fs / s) for t, s in zip(spec.tiers, steps)]))
    dense = oracle_scene(replace(spec, tiers=[(t[0], spec.fs) for t in spec.tiers]))
    n = np.arange(spec.n_in)
    worst = np.zeros(len(spec.tiers))
    tab = oracle.enumerate_images(dense)
    for i in range(tab["tier"].size):
        t0, _, _ = oracle.delay_gain(dense, i, n)
        t1, _, _ = oracle.delay_gain(tiered, i, n)
        worst[tab["tier"][i]] = max(worst[tab["tier"][i]], np.max(np.abs(t1 - t0)))
    return worst


def test_still_source_gets_the_sparsest_knots():
    spec = W.small_scene(seed=71, K=2, traj_kind=W.LINE)
    spec = replace(spec, traj=list(spec.traj[:6]) + [0.0])
    rates = api.Room.from_spec(spec).suggest_knot_rates(1e-3, max_step=400)
    assert rates == [spec.fs / 400] * 2


@pytest.mark.parametrize("kw,arr", [
    (dict(seed=72, K=3, traj_kind=W.SPLINE, tiers=[(1, 16000.0), (4, 1000.0), (W.RHO_INF, 1000.0)]), None),
    (dict(seed=73, K=3, traj_kind=W.CIRCLE, tiers=[(0, 16000.0), (W.RHO_INF, 1000.0)]), [0.0, 0.0, 0.0, 0.2, 0.5, 0.0]),
])
@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_suggested_rates_meet_the_delay_tolerance(kw, arr, tol):
    spec = W.small_scene(**kw)
    if arr is not None:
        spec = replace(spec, arr_kind=W.CIRCLE, arr_traj=arr, arr_duration=spec.duration)
    rates = api.Room.from_spec(spec).suggest_knot_rates(tol, max_step=2000)
    assert all(rates[t] >= rates[t + 1] for t in range(len(rates) - 1))   # sparser for farther tiers
    worst = _max_delay_error(spec, rates)
    assert np.all(worst <= tol)
    # and not wastefully dense: the sparsest-knot tier uses a good part of its budget
    assert worst[-1] >= tol / 40 or rates[-1] == spec.fs / 2000


def _max_bl_delay_error(spec, rates, Q):
    """Largest |tau| difference between band-limited knots at `rates` (a
    virtual knot at every sample, so only the upsampler's error remains) and
    the dense delays, over every image and sample (oracle)."""
    steps = [int(round(spec.fs / r)) for r in rates]
    tiered = oracle_scene(replace(spec, up_halfwidth=Q,
                                  tiers=[(t[0], spec.fs / s, s) for t, s in zip(spec.tiers, steps)]))
    dense = oracle_scene(replace(spec, tiers=[(t[0], spec.fs) for t in spec.tiers]))
    n = np.arange(spec.n_in)
    worst = np.zeros(len(spec.tiers))
    tab = oracle.enumerate_images(dense)
    for i in range(tab["tier"].size):
        t0, _, _ = oracle.delay_gain(dense, i, n)
        t1, _, _ = oracle.delay_gain(tiered, i, n)
        worst[tab["tier"][i]] = max(worst[tab["tier"][i]], np.max(np.abs(t1 - t0)))
    return worst


@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_bandlimited_rates_meet_the_delay_tolerance(tol):
    """Sec. II-C: knots at a rate chosen from the motion recover the distance
    band-limited. On a 1 s circle the suggested rates are a few Hz to tens of
    Hz, and the upsampled delays of every image stay within the tolerance."""
    spec = W.small_scene(seed=12, K=1, traj_kind=W.CIRCLE, seconds=1.0,
                         tiers=[(0, 16000.0), (W.RHO_INF, 1000.0)])
    room = api.Room.from_spec(spec)
    rates = room.suggest_bandlimited_rates(tol)
    assert all(r < 100.0 for r in rates)
    worst = _max_bl_delay_error(spec, rates, Q=4)
    assert np.all(worst <= 1.5 * tol)
    # a quarter of the rate is not enough
    assert np.any(_max_bl_delay_error(spec, [r / 4 for r in rates], Q=4) > tol)
