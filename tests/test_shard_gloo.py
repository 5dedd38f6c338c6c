"""One sky on several GPUs (bench.py --gpus N): particles and halos are partitioned by index,
every rank fills full map planes with its share, and one all-reduce sums the planes.  The host
logic runs here on two gloo ranks on the CPU, with the oracle's assign and deposit standing in
for the GPU kernels of each rank: the reduced maps must equal the maps of the unsplit sky (the
deposit and the halo paste are linear in their inputs), and the job reports the slowest rank's
step time."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2201_02632_gb300 import inputs as I
from paper_2201_02632_gb300 import shard


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sky():
    lc = I.lightcone(n_part=6000, n_halo=12, npix=64, side_deg=0.5, seed=77)
    return lc


def _maps_of(orc, lc, models, plo, phi, hlo, hhi):
    g = orc.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    parts = {k: v[plo:phi] for k, v in lc.parts.items()}
    a = orc.pp_assign(parts, lc.Mp, lc.halos.pos, models, g)
    y, b = orc.pp_deposit(a, g)
    c = lc.halos
    hy, hb = orc.hp_map(c.thx[hlo:hhi], c.thy[hlo:hhi], c.vlos[hlo:hhi], models[hlo:hhi], g,
                        rtol=1e-9)
    return np.stack([y, b, hy[0], hb[0]])


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc

    r, w, _ = bench.rank_env()
    lc = _sky()
    models = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)  # every rank: all halos
    plo, phi = shard.shard_range(lc.parts["x"].size, r, w)
    hlo, hhi = shard.shard_range(lc.halos.M.size, r, w)
    buf = torch.from_numpy(_maps_of(orc, lc, models, plo, phi, hlo, hhi))
    shard.reduce_maps(buf, w)
    t = bench.max_over_ranks(5.0 + 2.0 * r, w, torch.device("cpu"))  # rank 1 is the slower
    out[r] = (buf.numpy(), t, (plo, phi), (hlo, hhi))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_one_sky(orc):
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    lc = _sky()
    models = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    whole = _maps_of(orc, lc, models, 0, lc.parts["x"].size, 0, lc.halos.M.size)
    assert np.abs(whole[0]).max() > 0 and np.abs(whole[2]).max() > 0
    for r in range(world):
        got = res[r][0]
        for k in range(4):  # PP y, b and HP y, b: the sum of the shares is the whole sky
            np.testing.assert_allclose(got[k], whole[k], rtol=1e-12,
                                       atol=1e-12 * np.abs(whole[k]).max())
        assert res[r][1] == 7.0  # both ranks see the slowest rank's step time
    # the shares partition the particles and the halos
    assert res[0][2][0] == 0 and res[0][2][1] == res[1][2][0] and res[1][2][1] == 6000
    assert res[0][3][1] == res[1][3][0]


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (7, 3), (10, 4), (5_000_000, 8)])
def test_shard_range_partitions(n, world):
    spans = [shard.shard_range(n, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (a, b), (c, d) in zip(spans, spans[1:]):
        assert b == c
    sizes = [b - a for a, b in spans]
    assert max(sizes) - min(sizes) <= 1


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    buf = torch.ones(2, 3)
    assert shard.reduce_maps(buf, 1) is buf
    with pytest.raises(ValueError):
        shard.shard_range(5, 2, 2)
