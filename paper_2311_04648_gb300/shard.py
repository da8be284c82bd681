"""Assignment of independent scenes to ranks (one GPU each) and the final gather.

Independent scenes need no exchange while they run: each rank steps its own subset as one
batch and the per-scene results are gathered once at the end.  Scenes go to ranks by
greedy bin packing on their cost (spheres x steps): largest first, each to the rank with
the least load so far (ties to the lowest rank), which keeps the slowest rank within one
scene's cost of the average.  Host logic only; nothing here touches the method's
arithmetic.
"""
from __future__ import annotations

from typing import Sequence


def assign(costs: Sequence[float], n_ranks: int) -> list[list[int]]:
    """Scene indices per rank, each list ascending."""
    if n_ranks < 1:
        raise ValueError("need at least one rank")
    order = sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k))
    load = [0.0] * n_ranks
    parts: list[list[int]] = [[] for _ in range(n_ranks)]
    for k in order:
        r = min(range(n_ranks), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += float(costs[k])
    return [sorted(p) for p in parts]


def loads(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> list[float]:
    return [float(sum(costs[k] for k in p)) for p in parts]


def gather_results(local: dict, n_scenes: int, group=None) -> list:
    """Per-scene results of all ranks in scene order.  `local` maps this rank's scene
    indices to their results; every rank receives the full list (torch.distributed
    object all-gather, so any backend works)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, local, group=group)
    out = [None] * n_scenes
    for part in got:
        for k, v in part.items():
            if out[k] is not None:
                raise RuntimeError(f"scene {k} reported by two ranks")
            out[k] = v
    missing = [k for k in range(n_scenes) if out[k] is None]
    if missing:
        raise RuntimeError(f"scenes without a result: {missing[:8]}")
    return out
