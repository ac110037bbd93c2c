"""Sharding one LSCV_h selection over the ranks of a process group.

Every rank holds all samples (n d 4 bytes) and evaluates a contiguous range
of the pair-triangle tiles with ``kde_lscv_tile_sums`` on its own GPU; the 2
n_h FP64 exponential sums are added across ranks with one all-reduce; every
rank then finishes g(h) and the argmin with ``kde_lscv_merge``.  Range
boundaries fall on item boundaries (multiples of the tiles-per-item count K)
so each rank evaluates exactly the items a single-GPU run would.
"""
from __future__ import annotations

import numpy as np


def tile_shards(n_tiles: int, world: int, K: int = 1):
    """Contiguous [begin, end) tile ranges, one per rank, covering [0, n_tiles)
    once, with interior boundaries on multiples of K and tile counts as equal
    as that allows (tiles carry almost equal numbers of pairs)."""
    if world < 1 or n_tiles < 0 or K < 1:
        raise ValueError("bad shard arguments")
    rows = -(-n_tiles // K)
    out = []
    for r in range(world):
        b = min(n_tiles, (rows * r // world) * K)
        e = min(n_tiles, (rows * (r + 1) // world) * K)
        out.append((b, e))
    return out


def allreduce_sum(arr: np.ndarray, group=None) -> np.ndarray:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return arr
    backend = dist.get_backend(group)
    t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64))
    if backend == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def sharded_lscv(x, h, opts=None, group=None, tile: int | None = None):
    """LSCV_h selection of device samples x (d, n) sharded over `group`.
    Returns (result dict, g) on every rank."""
    import torch.distributed as dist

    from . import gbkde

    d, n = int(x.shape[0]), int(x.shape[1])
    h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    T = tile or (opts.tile if opts is not None and opts.tile else (32 if n <= 2048 else 128))
    K = shard_item_tiles(n, d, h.size, opts)
    b, e = tile_shards(gbkde.kde_tile_count(n, T), world, K)[rank]
    s1, s2 = gbkde.kde_lscv_tile_sums(x, h, b, e, opts)
    s = allreduce_sum(np.concatenate([s1, s2]), group)
    logdet = gbkde.kde_lscv_logdet(x)
    return gbkde.kde_lscv_merge(n, d, logdet, h, s[: h.size], s[h.size:])


def shard_item_tiles(n: int, d: int, n_h: int, opts=None) -> int:
    """Tiles per item of the single-GPU geometry (explicit in opts, else 1:
    any multiple of K keeps item boundaries; 1 is always valid)."""
    if opts is not None and opts.tiles_per_item:
        return int(opts.tiles_per_item)
    return 1
