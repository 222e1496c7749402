"""The multi-GPU bookkeeping of bench.py (independent replicas, max-over-ranks
step time, whole-job throughput) on two CPU ranks with the gloo backend."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2203_07329_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert replicas.env() == (ws, rank, rank)
    replicas.barrier()
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    mx = replicas.max_over_ranks(ms)
    out[rank] = (mx, replicas.job_throughput(32, mx, ws))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_throughput():
    ws, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        mx, thr = out[r]
        assert mx == 150.0                      # every rank sees the slowest rank's time
        assert thr == pytest.approx(2 * 32 / 0.150)  # whole-job lambda-solves/s


def test_single_process_defaults():
    from paper_2203_07329_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(32, 500.0, 1) == pytest.approx(64.0)
