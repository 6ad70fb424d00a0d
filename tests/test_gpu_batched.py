"""Batched synthesis (one persistent launch over many scenes), its CUDA-graph
replay and the autotuner, through the C ABI."""
import json

import numpy as np
import pytest
import torch

from oracle import api as oracle
from paper_2508_03065_gb300 import api
from paper_2508_03065_gb300 import workloads as W
from tests.scenes import oracle_scene, rel_l2, tile_samples

pytestmark = pytest.mark.gpu


def _scenes(n=6):
    # uneven durations, room sizes and orders, as in the 256-scene batch
    return [W.config3_scene(s) for s in range(n)]


def test_batch_graph_replay_matches_direct_and_oracle():
    specs = [W.small_scene(seed=90 + i, K=2 + i, seconds=0.04 + 0.05 * i, n_mics=1 + i % 2) for i in range(5)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    direct = [y.clone() for y in api.synthesize(rooms, xs)]
    b = api.Batch(rooms, xs)
    for use_graph in (False, True, True):
        ys = b.run(use_graph)
        b.stream.synchronize()
        for y, d in zip(ys, direct):
            assert torch.equal(y, d)
    for spec, d in zip(specs, direct):
        for m in range(d.shape[0]):
            ref = oracle.synthesize(oracle_scene(spec, m), spec.x.astype(np.float64))
            assert rel_l2(d[m].double().cpu().numpy(), ref) < 1e-5


def test_batched_config3_scenes_match_single_and_sampled_oracle():
    specs = _scenes(6)
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    # batched and single calls agree bitwise in one tile configuration (the
    # automatic choice may differ between a batch and one of its scenes)
    b = api.Batch(rooms, xs, tile_config=11)
    ys = [y.clone() for y in b.run(True)]
    b.stream.synchronize()
    for i, spec in enumerate(specs):
        single = api.synthesize([rooms[i]], [xs[i]], tile_config=11)[0]
        assert torch.equal(single, ys[i])
        idx = np.linspace(0, spec.n_in - 1, 12).astype(np.int64)
        ref = oracle.y_at(oracle_scene(spec), spec.x.astype(np.float64), idx)
        assert rel_l2(ys[i][0].double().cpu().numpy()[idx], ref) < 1e-5


def test_autotuner_picks_and_caches(tmp_path):
    specs = [W.small_scene(seed=95, K=5, seconds=0.5)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    path = str(tmp_path / "tune.json")
    before = api.synthesize(rooms, xs)[0].clone()
    best = api.autotune(rooms, xs, reps=2, cache_path=path)
    assert 0 <= best < api.tile_configs()
    data = json.load(open(path))
    (entry,) = data.values()
    assert entry["best"] == best and min(v for v in entry["ms"] if v > 0) == entry["ms"][best]
    assert api.autotune(rooms, xs, reps=2, cache_path=path) == best  # from the cache
    y = api.synthesize(rooms, xs, tile_config=best)[0]
    ref = oracle.synthesize(oracle_scene(specs[0]), specs[0].x.astype(np.float64))
    assert rel_l2(y[0].double().cpu().numpy(), ref) < 1e-5
    # the tuner returns its pick; calls without a configuration are unchanged
    assert torch.equal(api.synthesize(rooms, xs)[0], before)


def test_batched_config3_full_size_sampled():
    """All 256 batched scenes in one graph-replayed persistent launch, in the
    tile configuration chosen for their knot layout (14: knot records, 768-sample
    tiles), checked on the first, middle and last output of every output tile
    and on knot-interval edges of every 8th scene, which the oracle evaluates
    one by one."""
    specs = [W.config3_scene(s) for s in range(256)]
    rooms = [api.Room.from_spec(s) for s in specs]
    xs = [torch.from_numpy(s.x).cuda() for s in specs]
    b = api.Batch(rooms, xs, tile_config=14)
    ys = [y.clone() for y in b.run(True)]
    b.stream.synchronize()
    for i in range(0, 256, 8):
        spec = specs[i]
        # every output tile of configuration 14 (768 samples) and knot-interval edges
        idx = tile_samples(spec.n_in, 768, [N for _, N in spec.tier_steps()], edge_tiles=4)
        ref = oracle.y_at(oracle_scene(spec), spec.x.astype(np.float64), idx)
        got = ys[i][0].double().cpu().numpy()[idx]
        assert rel_l2(got, ref) < 1e-5 or np.max(np.abs(got - ref)) < 1e-9, i
