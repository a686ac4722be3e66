"""Multi-rank bookkeeping of the replica mode on CPU: two gloo ranks (world size 2).

Each rank draws its own sample range, the whole-job time is the slowest rank's, and the
per-sample rows gathered after the run are every rank's rows in rank order."""
import os
import socket

import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2601_21005_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        n = 3
        idx = list(replicas.sample_range(rank, n))
        # a rank-dependent "elapsed time" and rows that encode (rank, sample)
        ms = replicas.max_over_ranks(10.0 + 5.0 * rank, dist)
        sig = torch.tensor([[complex(rank, i), complex(-i, rank)] for i in idx], dtype=torch.complex128)
        x = torch.tensor([float(i) for i in idx], dtype=torch.float64)
        sg, xg = replicas.gather_rows(sig, x, dist)
        all_idx = [None] * world
        dist.all_gather_object(all_idx, idx)
        q.put((rank, ms, sg.numpy().tolist(), xg.numpy().tolist(), all_idx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, sg, xg, all_idx in out:
        assert ms == 15.0                                      # max over ranks, on every rank
        flat = [i for r in all_idx for i in r]
        assert len(set(flat)) == len(flat)                     # disjoint sample ranges
        assert xg == [float(i) for i in flat]                  # rank order
        for j, i in enumerate(flat):
            r = j // 3
            assert sg[j] == [complex(r, i), complex(-i, r)]
    assert out[0][2] == out[1][2]


def test_single_process_and_throughput():
    s = torch.zeros(2, 3, dtype=torch.complex128)
    x = torch.zeros(2, dtype=torch.float64)
    assert replicas.gather_rows(s, x) == (s, x)
    assert replicas.max_over_ranks(7.5) == 7.5
    assert list(replicas.sample_range(2, 3, stride=10)) == [20, 21, 22]
    # 4 ranks x 5 steps x 1e9 units in 2 s
    assert replicas.job_throughput(1e9, 5, 4, 2000.0) == pytest.approx(1e10)
    with pytest.raises(ValueError):
        replicas.sample_range(0, 11, stride=10)
    with pytest.raises(ValueError):
        replicas.job_throughput(1.0, 1, 1, 0.0)
