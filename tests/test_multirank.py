"""The multi-GPU path's host logic on CPU with gloo, world size 2: each rank gets its
own batch (weak scaling), and the whole-job figures take the slowest rank's times and
the sum of every rank's units.  (No GPU: the same reduction runs over NCCL on GPUs.)"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2206_13574_gb300 import synth
    g, qs = synth.make_config(2, n_queries=40)
    mine = bench.rank_queries(g, qs, rank)
    t_step, t_e2e, bp, cells = bench.reduce_ranks(0.10 + 0.05 * rank, 0.20 - 0.05 * rank,
                                                  int(mine.lengths().sum()), 1000 * (rank + 1),
                                                  torch.device("cpu"))
    out.put((rank, t_step, t_e2e, bp, cells, int(mine.lengths().sum()), mine.query(0)[:32]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, t0, e0, bp0, c0, own0, head0), (_, t1, e1, bp1, c1, own1, head1) = got
    assert t0 == t1 == pytest.approx(0.15)           # slowest rank's device step
    assert e0 == e1 == pytest.approx(0.20)           # slowest rank's end-to-end step
    assert bp0 == bp1 == own0 + own1                 # every rank's aligned bases
    assert c0 == c1 == 3000
    assert head0 != head1                            # distinct batches per rank


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.reduce_ranks(0.5, 0.7, 123, 456, torch.device("cpu")) == (0.5, 0.7, 123, 456)
