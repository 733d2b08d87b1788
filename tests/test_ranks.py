"""The multi-GPU host logic (one independent problem per rank, a barrier, the
slowest rank's time, whole-job throughput) with world_size 2 over gloo on the
CPU: the same calls the benchmark makes under torchrun with NCCL."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2409_10876_gb300 import inputs, ranks


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = ranks.dist_env()
        assert (r, w, local) == (rank, world, rank)
        cfg = inputs.config_tiny()
        case = inputs.make_case(cfg, ranks.rank_seed(7, r))
        ranks.barrier(w)
        local_ms = 10.0 + 5.0 * r                         # rank 1 is the slower one
        job_ms = ranks.job_time_ms(local_ms, w)
        out[rank] = (job_ms, ranks.job_value(w, 100, job_ms), float(case["sos_true"].sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                     # both ranks see the slowest time
    assert res[0][1] == res[1][1] == 2 * 100 / 0.015           # ranks x steps / slowest time
    assert res[0][2] != res[1][2]                              # different problems


def test_single_rank_needs_no_process_group():
    assert ranks.job_time_ms(12.5, 1) == 12.5
    assert ranks.job_value(1, 50, 100.0) == 500.0
    assert ranks.rank_seed(3, 0) == 3
