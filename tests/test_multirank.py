"""Multi-rank bookkeeping of bench.py on CPU with gloo (world size 2): the job's
step time is the slowest rank's on every rank, the value counts every rank's
queries, every rank builds from the same symbols and draws its own queries."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2505_03372_gb300 import workloads

    ms = bench.job_ms(10.0 + 5.0 * rank, dist)
    w = workloads.Workload("t", 7, 4096, 16, 1, "uniform", 1.0, {"access": 64, "rank": 64, "select": 64})
    sym = workloads.make_symbols(w.n, w.sigma, 1, "uniform", seed=workloads.SEED_BASE + w.index, device="cpu")
    q = workloads.make_queries(w, sym, seed=bench.rank_seed(workloads.SEED_BASE + 0x100, rank))
    syms = [torch.zeros_like(sym) for _ in range(world)]
    dist.all_gather(syms, sym)
    acc = [torch.zeros_like(q["access_i"]) for _ in range(world)]
    dist.all_gather(acc, q["access_i"])
    out[rank] = (ms, bench.job_value(world, 192, ms), all(torch.equal(syms[0], s) for s in syms),
                 not torch.equal(acc[0], acc[1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_share_the_build_and_split_the_queries():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value, same_symbols, own_queries = out[r]
        assert ms == 15.0                                  # the slowest rank's step time, on every rank
        assert value == pytest.approx(2 * 192 / 15e-3 / 1e6)  # both ranks' queries
        assert same_symbols and own_queries


def test_single_rank_is_unchanged():
    import bench

    assert bench.job_ms(12.5, None) == 12.5
    assert bench.rank_seed(100, 0) == 100
    assert bench.job_value(1, 3_000_000, 10.0) == pytest.approx(300.0)
