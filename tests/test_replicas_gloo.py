"""The multi-GPU path of bench.py is replicas only: each rank pastes its own light-cone and
the job reports the slowest rank's step time and the units of all ranks.  Its host logic
(replica seeds, max over ranks, whole-job rate) is checked here with two gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2201_02632_gb300 import inputs as I


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.rank_env()
    t_step = 5.0 + 2.0 * r  # rank 1 is the slower one
    t = bench.max_over_ranks(t_step, w, torch.device("cpu"))
    out[r] = (t, bench.job_rate(1000, w, t), bench.replica_seed(r, I.SEED_BASE))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 7.0  # both ranks see the max of 5 and 7 ms
    assert res[0][1] == pytest.approx(2 * 1000 / 7e-3)  # units of all ranks / slowest time
    assert res[0][2] != res[1][2]  # each replica draws its own sky


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_rate(4_000_000, 1, 8.0) == pytest.approx(5e8)
