"""Multi-GPU sharding of one exact volume: one process per GPU, each enumerating the work
ranges u with u % world == rank, then one exchange step — an exact all-reduce of the partial
sums (128-bit volume as four 32-bit limbs, cells, singular, ties), and a re-lift for every rank
when any shard met a tie.  The exchange runs over torch.distributed (NCCL on GPUs, gloo on CPU
ranks); nothing else is communicated."""

from __future__ import annotations

import torch
import torch.distributed as dist

from ._lib import BinodegError

MAX_LIFTINGS = 8  # the library's re-lift cap
_KEYS = ("cells", "singular", "ties")


def _device(group) -> torch.device:
    backend = dist.get_backend(group)
    return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")


def combine(partial: dict, group=None) -> dict:
    """Exact sum of the ranks' partial results (an all-reduce of seven int64 words)."""
    v = int(partial["nvol"])
    limbs = [(v >> (32 * i)) & 0xFFFFFFFF for i in range(4)]
    t = torch.tensor(limbs + [int(partial[k]) for k in _KEYS], dtype=torch.int64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    w = t.cpu().tolist()
    out = dict(partial)
    out["nvol"] = sum(w[i] << (32 * i) for i in range(4))
    for i, k in enumerate(_KEYS):
        out[k] = w[4 + i]
    return out


def check_same_work_list(info: dict, group=None) -> None:
    """Every rank must shard the same work list (same items and ranges)."""
    t = torch.tensor([info["items"], info["ranges"], -info["items"], -info["ranges"]], dtype=torch.int64,
                     device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    mx = t.cpu().tolist()
    if mx[0] != -mx[2] or mx[1] != -mx[3]:
        raise BinodegError(1, "ranks built different work lists (plan options or GPU models differ)")


def volume(plan, seed: int = 0, group=None, stream=None) -> dict:
    """The exact volume of `plan`'s points, sharded over the ranks of `group`."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    check_same_work_list(plan.info(), group)
    for attempt in range(MAX_LIFTINGS):
        plan.launch(seed=seed, attempt=attempt, stream=stream, shard=rank, shards=world)
        total = combine(plan.read(), group)
        if total["ties"] == 0:
            total["relifts"] = attempt
            return total
    raise BinodegError(3, "every allowed lifting had ties")
