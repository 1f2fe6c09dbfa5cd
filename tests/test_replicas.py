"""The multi-rank bench logic on CPU with the gloo backend (two ranks):
units add up, time is the slowest rank's, and every rank sees the same."""
import os

import pytest


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2606_10019_gb300 import replicas as R
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, secs = R.combine(100.0 * (rank + 1), 1.5 + rank)
    out[rank] = (units, secs, R.rank_stream(2, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_two_ranks_gloo():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][:2] == (300.0, 2.5) and out[1][:2] == (300.0, 2.5)
    assert out[0][2] == 2 and out[1][2] == 102


def test_combine_single_process_is_identity():
    from paper_2606_10019_gb300 import replicas as R
    assert R.combine(7.0, 3.0) == (7.0, 3.0)
