"""Sharding one LSCV_h or PLUGIN selection over the ranks of a process group.

Every rank holds all samples (n d 4 bytes) and evaluates a contiguous range
of the pair-triangle tiles on its own GPU.

* LSCV_h: ``kde_lscv_tile_sums`` over the rank's range, one all-reduce of the
  2 n_h FP64 exponential sums, then ``kde_lscv_merge`` (g(h) and the argmin)
  on every rank.
* PLUGIN (Sec. 4.4.1): sigma from the prologue gives g1 on every rank
  (``kde_plugin_merge`` stage 8); ``kde_psi_tile_sums`` of psi_6 at g1 over
  the rank's range, one all-reduce of one FP64 value, stage 6 gives psi_6 and
  g2 on every rank; the same for psi_4 at g2, and stage 4 gives h: two
  exchanges, one after each all-pairs pass.

Range boundaries fall on item boundaries (multiples of the single-GPU
geometry's tiles per item, ``kde_item_tiles``), so each rank evaluates
exactly the items a single-GPU run would; only the FP64 order in which the
item sums are added differs.
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
    geo = gbkde.kde_item_tiles(n, d, h.size, opts, h=h)
    T = tile or geo["lscv_tile"]
    K = shard_item_tiles(n, d, h.size, opts, h=h)
    b, e = tile_shards(gbkde.kde_tile_count(n, T), world, K)[rank]
    s1, s2 = gbkde.kde_lscv_tile_sums(x, h, b, e, opts)
    s = allreduce_sum(np.concatenate([s1, s2]), group)
    logdet = gbkde.kde_lscv_logdet(x)
    return gbkde.kde_lscv_merge(n, d, logdet, h, s[: h.size], s[h.size:])


def shard_item_tiles(n: int, d: int, n_h: int, opts=None, h=None) -> int:
    """Tiles per LSCV item of the single-GPU geometry on the grid h (None:
    the default grid of n_h points): explicit in opts, else the library's
    rule for this size and grid on this device."""
    if opts is not None and opts.tiles_per_item:
        return int(opts.tiles_per_item)
    from . import gbkde
    return int(gbkde.kde_item_tiles(n, d, n_h, opts, h=h)["lscv_K"])


def sharded_plugin(x, opts=None, group=None):
    """PLUGIN selection of univariate device samples x (1, n) sharded over
    `group`: two all-reduces of one FP64 value each.  Returns the result dict
    on every rank."""
    import torch.distributed as dist

    from . import gbkde

    n = int(x.shape[-1])
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    geo = gbkde.kde_item_tiles(n, 1, 0, opts)
    b, e = tile_shards(gbkde.kde_tile_count(n, geo["psi_tile"]), world, geo["psi_K"])[rank]
    sigma = float(np.sqrt(gbkde.kde_sample_covariance(x)[0, 0]))
    res = gbkde.kde_plugin_merge(n, 8, sigma)
    for r, pilot in ((6, "g1"), (4, "g2")):
        part = gbkde.kde_psi_tile_sums(x, r, res[pilot], b, e, opts)
        total = float(allreduce_sum(np.array([part]), group)[0])
        res = gbkde.kde_plugin_merge(n, r, total, res)
    return res
