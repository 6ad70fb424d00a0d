"""Host side of the multi-GPU path on CPU (gloo, world size 2): scene
sharding and the whole-job throughput reduction. No GPU is touched."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2508_03065_gb300 import multigpu
from paper_2508_03065_gb300 import workloads as W


def test_shard_scenes_partition_and_balance():
    work = [float(W.image_count(k) * n) for k, n in zip(range(3, 13), [16000, 32000, 8000, 64000] * 3)]
    for world in (1, 2, 3, 8):
        shards = multigpu.shard_scenes(work, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(work)))
        loads = [sum(work[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(work) + 1e-9
    assert multigpu.shard_scenes(work, 2) == multigpu.shard_scenes(list(work), 2)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    work = [10.0, 7.0, 5.0, 3.0, 3.0, 1.0]
    mine = multigpu.shard_scenes(work, world)[rank]
    local_work = sum(work[i] for i in mine)
    local_ms = 100.0 + 50.0 * rank
    value, ms = multigpu.job_throughput(local_work, local_ms)
    dist.barrier()
    q.put((rank, mine, value, ms))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_gloo_sharding_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, v0, ms0), (_, s1, v1, ms1) = res
    assert sorted(s0 + s1) == list(range(6)) and not set(s0) & set(s1)
    assert ms0 == ms1 == 150.0                       # the slowest rank's time
    assert abs(v0 - 29.0 / 0.150) < 1e-9 and v0 == v1  # all ranks' work / max time
