"""Network inference over several GPUs: targets sharded across ranks.

Greedy parent selection of one target is independent of every other target
(each target's loop reads the shared series and nothing else), so a network
is inferred by handing targets to ranks round-robin, one GPU per rank, with
no collective inside any target's inference.  The per-target results are
combined once at the end with an all-gather over the default process group
(any backend; NCCL on GPUs, gloo in the CPU tests).  Without an initialised
process group the whole network runs in this process.
"""
from __future__ import annotations

from typing import Callable


def targets_of_rank(n_targets: int, world: int, rank: int) -> list:
    """Targets of one rank: rank, rank + world, rank + 2 world, ..."""
    if world < 1 or not 0 <= rank < world or n_targets < 0:
        raise ValueError("bad world/rank/target count")
    return list(range(rank, n_targets, world))


def _group():
    try:
        import torch.distributed as dist
    except ImportError:          # pragma: no cover - torch is a dependency
        return None, 1, 0
    if dist.is_available() and dist.is_initialized():
        return dist, dist.get_world_size(), dist.get_rank()
    return None, 1, 0


def infer_network(series, n_targets: int, select: Callable | None = None, **kw) -> dict:
    """Parents of targets 0 .. n_targets-1.

    ``select(series, target, **kw)`` runs one target's greedy loop and returns
    a picklable result (default: ``mte_select_target`` of this package on the
    rank's current device).  Each rank runs its own targets; every rank
    returns the same ``{target: result}`` dict for all targets.
    """
    if select is None:
        from . import mte_select_target as select
    dist, world, rank = _group()
    mine = {t: select(series, t, **kw) for t in targets_of_rank(n_targets, world, rank)}
    if dist is None:
        return mine
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    out = {}
    for part in parts:
        for t, res in part.items():
            if t in out:
                raise RuntimeError(f"target {t} inferred by two ranks")
            out[t] = res
    if sorted(out) != list(range(n_targets)):
        raise RuntimeError("some targets were not inferred")
    return out
