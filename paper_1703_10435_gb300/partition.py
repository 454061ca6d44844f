"""Static partition of the coarse elements over ranks (the MPI version's
partition T_H^r of the paper, Sec. 4.1.2): contiguous K ranges, one per rank,
and the gather of the per-element blocks that a rank computed."""
from __future__ import annotations


def k_range(n_K: int, rank: int, world: int) -> tuple[int, int]:
    """[K_begin, K_end) of `rank`: contiguous, the first n_K % world ranks one longer."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_K, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_blocks(blocks: dict, K0: int, K1: int, n_K: int, group=None) -> dict:
    """All-gather per-element arrays (first axis = K in [K0, K1)) into full
    (n_K, ...) arrays on every rank; `blocks` maps name -> torch tensor."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = {}
    for name, t in blocks.items():
        parts = [None] * world
        dist.all_gather_object(parts, (K0, K1, t.cpu()), group=group)
        full = torch.empty((n_K,) + tuple(t.shape[1:]), dtype=t.dtype)
        for a, b, piece in parts:
            full[a:b] = piece
        out[name] = full
    return out
