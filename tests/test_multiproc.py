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


def test_reference_arm_under_torchrun_prints_one_line():
    """The reference arm launched as the driver launches N > 1 (torchrun, two
    ranks on 127.0.0.1): rank 0 alone times the oracle and prints one JSON
    line; the other rank exits 0 without work. Loads no part of the library."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--workload", "event100", "--steps", "1",
           "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=root, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
