"""Host logic of sharded LSCV_h on CPU: the tile partition, and a world-size-2
gloo run of all-reduce + kde_lscv_merge.  Each rank's exponential sums over
its tile range come from the FP64 oracle (standing in for that rank's GPU),
so the merge path is exercised without a GPU."""
import os
import socket

import numpy as np
import pytest

from paper_1505_01998_gb300.shard import tile_shards
from tests._helpers import built_lib


@pytest.mark.parametrize("n_tiles,world,K", [(0, 2, 1), (1, 2, 1), (10, 3, 1), (528, 4, 7),
                                             (131328, 8, 216), (99, 1, 5), (7, 8, 2)])
def test_tile_shards_cover_once_on_item_boundaries(n_tiles, world, K):
    sh = tile_shards(n_tiles, world, K)
    assert len(sh) == world
    assert sh[0][0] == 0 and sh[-1][1] == n_tiles
    for (b, e), (b2, _) in zip(sh, sh[1:]):
        assert e == b2 and b <= e
        assert e % K == 0 or e == n_tiles
    sizes = [e - b for b, e in sh]
    assert max(sizes) - min(sizes) <= K


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1505_01998_gb300 import datagen, gbkde
    from paper_1505_01998_gb300.shard import allreduce_sum, tile_shards

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, d, T = 333, 2, 32
    x = datagen.correlated_mixture(n, d, seed=77).astype(np.float64)
    h = oracle.grid_default(n, d, 24)
    tiles = gbkde.kde_tile_count(n, T)
    b, e = tile_shards(tiles, world, 3)[rank]
    s1 = np.zeros(h.size)
    s2 = np.zeros(h.size)
    for t in range(b, e):
        l, q = gbkde.kde_tile_coords(t)
        a1, a2, _ = oracle.lscv_sums(x, h, block=(q * T, q * T + T, l * T, l * T + T), threads=1)
        s1 += a1
        s2 += a2
    s = allreduce_sum(np.concatenate([s1, s2]))
    _, S = oracle.mean_cov(x)
    res, g = gbkde.kde_lscv_merge(n, d, float(np.log(np.linalg.det(S))), h, s[:h.size], s[h.size:])
    np.save(os.path.join(out_dir, f"g{rank}.npy"), g)
    np.save(os.path.join(out_dir, f"arg{rank}.npy"), np.array([res["argmin"]]))
    dist.destroy_process_group()


def test_gloo_two_ranks_merge_equals_oracle(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_1505_01998_gb300 import datagen

    built_lib()
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    n, d = 333, 2
    x = datagen.correlated_mixture(n, d, seed=77).astype(np.float64)
    h = oracle.grid_default(n, d, 24)
    ref = oracle.lscv_h(x, h)
    g0 = np.load(tmp_path / "g0.npy")
    g1 = np.load(tmp_path / "g1.npy")
    assert np.array_equal(g0, g1)  # every rank finishes the same way
    assert np.allclose(g0, ref["g"], rtol=1e-11, atol=1e-14)
    assert int(np.load(tmp_path / "arg0.npy")[0]) == ref["argmin"]
