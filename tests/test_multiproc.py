"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2):
each rank runs independent replicas (own seed), the job time is the slowest
rank's, the value counts every rank's spin-updates, and the job's best of
every event is the lowest energy over the ranks with that rank's selection."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms_local = 100.0 + 50.0 * rank
    ms = bench.reduce_step_ms(ms_local, ws, dist, torch.device("cpu"))
    out[rank] = (bench.rank_seed(rank), ms, bench.job_value(1_000_000, ws, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_sum_units():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    seeds = {out[r][0] for r in range(ws)}
    assert len(seeds) == ws
    assert out[0][1] == out[1][1] == 150.0
    assert out[0][2] == pytest.approx(2 * 1_000_000 / 0.150)


def _best_worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import numpy as np
    import bench
    row0 = np.array([0, 3, 5, 9])
    # three events; rank 1 is better on event 0, tied on event 1, worse on event 2
    E = np.array([[-5.0, -2.0, -7.0], [-6.0, -2.0, -1.0]])[rank]
    T = np.full(9, rank + 1, np.uint8)
    Ej, win, Tj = bench.best_across_ranks(E, T, row0, dist, torch.device("cpu"))
    out[rank] = (Ej.tolist(), win.tolist(), Tj.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_best_of_every_event():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_best_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert out[0] == out[1]
    Ej, win, Tj = out[0]
    assert Ej == [-6.0, -2.0, -7.0]
    assert win == [1, 0, 0]   # the tie goes to the lowest rank
    assert Tj == [2, 2, 2, 1, 1, 1, 1, 1, 1]


def test_single_rank_has_no_collective():
    import bench
    assert bench.reduce_step_ms(12.5, 1) == 12.5
    assert bench.job_value(10, 1, 1000.0) == 10.0
    import numpy as np
    E, win, T = bench.best_across_ranks([-1.0, -2.0], np.ones(4, np.uint8), [0, 2, 4])
    assert E.tolist() == [-1.0, -2.0] and win.tolist() == [0, 0] and T.tolist() == [1, 1, 1, 1]
