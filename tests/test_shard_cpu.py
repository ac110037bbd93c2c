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


def test_plugin_merge_steps_match_the_oracle_chain():
    """The host steps of a sharded PLUGIN selection (Sec. 4.4.1) from the
    oracle's own sigma and full pair sums give the oracle's chain."""
    import oracle
    from paper_1505_01998_gb300 import datagen

    kde = built_lib()
    x = datagen.skewed_column(700, seed=41)[0].astype(np.float64)
    n = x.size
    ref = oracle.plugin(x)
    r = kde.kde_plugin_merge(n, 8, ref["sigma"])
    assert r["psi8_ns"] == pytest.approx(ref["psi8_ns"], rel=1e-14)
    assert r["g1"] == pytest.approx(ref["g1"], rel=1e-14)
    r = kde.kde_plugin_merge(n, 6, oracle.psi_pair_sum(x, 6, r["g1"]), r)
    assert r["psi6"] == pytest.approx(ref["psi6"], rel=1e-12)
    assert r["g2"] == pytest.approx(ref["g2"], rel=1e-12)
    r = kde.kde_plugin_merge(n, 4, oracle.psi_pair_sum(x, 4, r["g2"]), r)
    assert r["psi4"] == pytest.approx(ref["psi4"], rel=1e-12)
    assert r["h"] == pytest.approx(ref["h"], rel=1e-12)
    assert r["h_plugin"] == r["h"] == r["h_data"] and r["status"] == 0


def test_plugin_merge_rejects_out_of_order_and_degenerate_steps():
    kde = built_lib()
    with pytest.raises(kde.KdeError) as e:
        kde.kde_plugin_merge(100, 6, -1.0)  # no g1 yet
    assert e.value.status == kde.KDE_EINVAL
    r = kde.kde_plugin_merge(100, 8, 1.0)
    with pytest.raises(kde.KdeError) as e:
        kde.kde_plugin_merge(100, 6, 1e6, r)  # psi_6 >= 0: g2 undefined
    assert e.value.status == kde.KDE_EDEGENERATE
    with pytest.raises(kde.KdeError) as e:
        kde.kde_plugin_merge(100, 8, 0.0)
    assert e.value.status == kde.KDE_EDEGENERATE
    with pytest.raises(kde.KdeError):
        kde.kde_plugin_merge(100, 5, 1.0, r)


def _plugin_rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1505_01998_gb300 import datagen, gbkde
    from paper_1505_01998_gb300.shard import allreduce_sum, tile_shards

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, T, K = 517, 32, 3
    x = datagen.mixture_1d(n, seed=78)[0].astype(np.float64)
    b, e = tile_shards(gbkde.kde_tile_count(n, T), world, K)[rank]

    def part(r, g):  # this rank's tiles, from the oracle standing in for its GPU
        s = 0.0
        for t in range(b, e):
            l, q = gbkde.kde_tile_coords(t)
            s += oracle.psi_pair_sum(x, r, g, threads=1, block=(q * T, q * T + T, l * T, l * T + T))
        return s

    _, S = oracle.mean_cov(x)
    res = gbkde.kde_plugin_merge(n, 8, float(np.sqrt(S[0, 0])))
    for r, pilot in ((6, "g1"), (4, "g2")):
        total = float(allreduce_sum(np.array([part(r, res[pilot])]))[0])
        res = gbkde.kde_plugin_merge(n, r, total, res)
    np.save(os.path.join(out_dir, f"p{rank}.npy"),
            np.array([res[k] for k in ("g1", "psi6", "g2", "psi4", "h")]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_sharded_plugin_equals_oracle(tmp_path, world):
    """Sharded PLUGIN host logic with `world` gloo ranks: each rank's psi_6
    and psi_4 sums over its tiles (oracle blocks), two all-reduces, the chain
    on every rank; every rank ends with the oracle's bandwidth."""
    import torch.multiprocessing as mp

    import oracle
    from paper_1505_01998_gb300 import datagen

    built_lib()
    mp.start_processes(_plugin_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    x = datagen.mixture_1d(517, seed=78)[0].astype(np.float64)
    ref = oracle.plugin(x)
    outs = [np.load(tmp_path / f"p{r}.npy") for r in range(world)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])  # every rank holds the same chain
    want = np.array([ref[k] for k in ("g1", "psi6", "g2", "psi4", "h")])
    assert np.allclose(outs[0], want, rtol=1e-11, atol=0)
