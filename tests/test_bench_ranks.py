"""Multi-rank path of bench.py on CPU (gloo, world size 2).

With N GPUs every rank analyses its own sample and nothing but the timing
and the window totals crosses ranks: the job's time is the slowest rank's
timed region, its work the windows all ranks analysed (weak scaling).
These tests run that host logic as two gloo processes.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        env = bench.rank_env()
        bench.barrier()
        secs = [0.5, 2.0, 1.0, 0.25][rank]
        wins = [1000, 3000, 5, 7][rank]
        sec, tot = bench.reduce_over_ranks(secs, wins, torch.device("cpu"))
        r = bench.workload(rank, 400)
        rs = synth.generate(r, threads=1)
        digest = int(np.bitwise_xor.reduce(rs.bases[: 150 * 64].view(np.uint64)))
        q.put((rank, env, sec, tot, r.seed, r.n_reads, r.n_genomes, rs.n_bases, digest))
        bench.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_reduce_and_own_samples(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    secs = [0.5, 2.0, 1.0, 0.25][:world]
    wins = [1000, 3000, 5, 7][:world]
    for rank, env, sec, tot, seed, n_reads, n_genomes, n_bases, digest in out:
        assert env == (world, rank, rank)
        assert sec == max(secs)           # slowest rank's timed region
        assert tot == sum(wins)           # every rank's windows
        assert n_reads == 400 and n_bases == 400 * 150
        assert n_genomes == out[0][6]
    # independent samples: same recipe shape, another seed, other reads
    assert len({o[4] for o in out}) == world
    assert len({o[8] for o in out}) == world


def test_single_rank_is_identity():
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(1.5, 42, torch.device("cpu")) == (1.5, 42)
