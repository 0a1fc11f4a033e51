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


def _tree_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2505_03372_gb300 import workloads

    buf, views, sigmas, q = workloads.make_batch(ntrees=37, seed=workloads.SEED_BASE + 3, device="cpu",
                                                 log_n=(4, 12), log_q=(2, 6))
    lo, hi = bench.shard_range(len(views), rank, world)
    b2, v2, s2, q2 = workloads.batch_subset(views, sigmas, q, lo, hi)
    # every tree of the share is the batch's tree, 16-byte aligned in the new buffer
    same = all(torch.equal(a, views[lo + k]) for k, a in enumerate(v2))
    aligned = all((v.data_ptr() - b2.data_ptr()) % 16 == 0 for v in v2)
    # the share's queries are exactly the batch's queries of trees [lo, hi), renumbered
    m = (q["tree"] >= lo) & (q["tree"] < hi)
    qok = torch.equal(q2["tree"].long() + lo, q["tree"][m].long()) and torch.equal(q2["arg"], q["arg"][m])
    counts = torch.tensor([hi - lo, q2["tree"].numel()], dtype=torch.int64)
    dist.all_reduce(counts)
    ranges = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(ranges, torch.tensor([lo, hi], dtype=torch.int64))
    out[rank] = (same, aligned, qok, counts.tolist(), [r.tolist() for r in ranges], q["tree"].numel(), s2 == sigmas[lo:hi])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_the_batched_trees():
    """The batched workload under torchrun: each rank takes a contiguous range
    of the drawn trees (no collective on the data path); together the ranks
    cover every tree and every query exactly once."""
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_tree_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        same, aligned, qok, counts, ranges, total_q, sig_ok = out[r]
        assert same and aligned and qok and sig_ok
        assert counts == [37, total_q]
        assert ranges == [[0, 19], [19, 37]]
