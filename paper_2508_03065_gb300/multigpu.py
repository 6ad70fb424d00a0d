"""Scene sharding across ranks (one process per GPU).

Scenes are independent (every image, and so every scene, is synthesised on
its own: Sec. II-C), so several GPUs take disjoint sets of scenes and no
collective touches the data path. The only collectives are on the control
path: a barrier around timed regions and the max-over-ranks of elapsed time.
"""
from __future__ import annotations

from typing import List, Sequence


def shard_scenes(work: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time assignment of scenes (by estimated work, e.g.
    images x output samples x microphones) to `world` ranks. Deterministic:
    ties go to the lower scene index and the lower rank. Returns the scene
    indices of every rank in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(work[i])
    return [sorted(s) for s in out]


def job_throughput(local_work: float, local_ms: float, group=None) -> tuple:
    """Whole-job throughput over ranks: the work of all ranks divided by the
    slowest rank's time. Returns (units per second, max milliseconds)."""
    import torch
    import torch.distributed as dist

    if group is None and not (dist.is_available() and dist.is_initialized()):
        return local_work / (local_ms * 1e-3), local_ms
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    w = torch.tensor([local_work], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    ms = float(t.item())
    return float(w.item()) / (ms * 1e-3), ms
