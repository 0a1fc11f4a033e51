"""Batched trees (one graph launch) against the CPU oracle, tree by tree."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402
from guard import guarded, intact  # noqa: E402

pytestmark = pytest.mark.gpu
U64MAX = np.iinfo(np.uint64).max


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _expected(views, sigmas, q):
    tree = q["tree"].cpu().numpy()
    kind = q["kind"].cpu().numpy()
    c = q["c"].cpu().numpy().view(np.uint32)
    arg = q["arg"].cpu().numpy().view(np.uint64)
    want = np.full(tree.size, U64MAX, np.uint64)
    for i, (v, s) in enumerate(zip(views, sigmas)):
        S = v.cpu().numpy().view(np.uint16)
        o1 = oracle.O1(S, s)
        for kd, f in ((0, lambda m: o1.access(arg[m]).astype(np.uint64)), (1, lambda m: o1.rank(c[m], arg[m])),
                      (2, lambda m: o1.select(c[m], arg[m]))):
            m = (tree == i) & (kind == kd)
            if m.any():
                want[m] = f(m)
    return want


@pytest.mark.parametrize("K,qthreads", [(4096, 256), (1024, 128), (8192, 512)])
def test_batch_matches_oracle(K, qthreads):
    buf, views, sigmas, q = workloads.make_batch(ntrees=40, seed=K + qthreads, log_n=(0, 17), log_q=(2, 10),
                                                 sigmas=(2, 3, 4, 96, 256, 1000, 65536))
    # one empty tree too
    views = list(views) + [buf[:0]]
    sigmas = list(sigmas) + [7]
    with wt.Batch(views, sigmas, sample_k=K, query_threads=qthreads) as b:
        nq = q["arg"].numel()
        out, full = guarded(nq, torch.int64)
        b.set_queries(q["tree"], q["kind"], q["c"], q["arg"], out=out)
        want = _expected(views, sigmas, q)
        for _ in range(2):  # the graph can be launched again
            out.fill_(0)
            b.run()
            assert b.status_sync() == wt.WT_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
            assert intact(full, nq), "the batch wrote outside its output"
        # every tree's structure equals the naive oracle tree
        for i, (v, s) in enumerate(zip(views, sigmas)):
            S = v.cpu().numpy().view(np.uint16)
            o2 = oracle.O2Tree(S, s, K=K)
            t = b.tree(i)
            inf = t.info()
            assert inf.levels == o2.L
            for l in range(o2.L):
                assert inf.level_size[l] == o2.level_size(l)
                for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
                    assert np.array_equal(t.export(what, l), o2.export(what, l)), (i, l, what)
            assert np.array_equal(t.export(wt.EXPORT_C), o2.export(oracle.EXPORT_C))
            assert np.array_equal(t.export(wt.EXPORT_NODES), o2.export(oracle.EXPORT_NODES))
            t.close()


def test_batch_tree_view_answers_queries_and_bad_tree_ids():
    buf, views, sigmas, q = workloads.make_batch(ntrees=6, seed=7, log_n=(12, 16), log_q=(4, 6))
    with wt.Batch(views, sigmas) as b:
        bad = torch.tensor([len(views), 1 << 20], dtype=torch.int32, device="cuda")
        kind = torch.zeros(2, dtype=torch.uint8, device="cuda")
        out = b.set_queries(bad, kind, torch.zeros(2, dtype=torch.int32, device="cuda"),
                            torch.zeros(2, dtype=torch.int64, device="cuda"))
        b.run()
        b.status_sync()
        assert out.cpu().numpy().view(np.uint64).tolist() == [U64MAX, U64MAX]
        t = b.tree(3)
        S = views[3].cpu().numpy().view(np.uint16)
        i = torch.arange(0, S.size, 97, dtype=torch.int64, device="cuda")
        assert np.array_equal(t.access(i).cpu().numpy().view(np.uint32), S[::97].astype(np.uint32))
        t.close()


@pytest.mark.slow
def test_batch_of_256_trees_from_the_workload_law_matches_oracle():
    """256 trees drawn as the batched workload draws them: n = floor(2^U(10, 24))
    uint16 symbols, sigma uniform from {4, 256, 65536}, floor(2^U(4, 16)) mixed
    queries per tree.  The draw holds sigma = 65536 trees with n >= 2^22 (the
    large-tile path of the batched level pass).  Every tree's levels, counters,
    samples, C and node table against the naive oracle tree; every answer
    against the definitions."""
    buf, views, sigmas, q = workloads.make_batch(ntrees=256, seed=workloads.SEED_BASE + 304)
    assert sum(1 for v, s in zip(views, sigmas) if s == 65536 and v.numel() >= 1 << 22) >= 5
    with wt.Batch(views, sigmas) as b:
        out = b.set_queries(q["tree"], q["kind"], q["c"], q["arg"])
        b.run()
        assert b.status_sync() == wt.WT_OK
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, _expected(views, sigmas, q))
        for i, (v, s) in enumerate(zip(views, sigmas)):
            S = v.cpu().numpy().view(np.uint16)
            o2 = oracle.O2Tree(S, s, K=4096)
            t = b.tree(i)
            inf = t.info()
            assert inf.levels == o2.L
            for l in range(o2.L):
                assert inf.level_size[l] == o2.level_size(l) and inf.level_ones[l] == o2.level_ones(l), (i, l)
                for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
                    assert np.array_equal(t.export(what, l), o2.export(what, l)), (i, l, what)
            assert np.array_equal(t.export(wt.EXPORT_C), o2.export(oracle.EXPORT_C))
            assert np.array_equal(t.export(wt.EXPORT_NODES), o2.export(oracle.EXPORT_NODES))
            t.close()


def test_autotuned_options_are_exact(tmp_path):
    """The autotuner's choice (timed on the GPU, cached in a temporary file)
    builds and answers exactly: every answer against the definitions."""
    from paper_2505_03372_gb300 import autotune

    buf, views, sigmas, q = workloads.make_batch(ntrees=64, seed=workloads.SEED_BASE + 21, log_n=(8, 18),
                                                 log_q=(3, 10))
    opts = autotune.tune_batch(views, sigmas, q, cache_path=str(tmp_path / "tune.json"), stride=4, reps=1)
    assert set(opts) == {"sample_k", "query_threads", "lp_ctas_per_sm"}
    with wt.Batch(views, sigmas, **opts) as b:
        out = b.set_queries(q["tree"], q["kind"], q["c"], q["arg"])
        b.run()
        assert b.status_sync() == wt.WT_OK
        assert np.array_equal(out.cpu().numpy().view(np.uint64), _expected(views, sigmas, q))
    # every level-pass grid gives the same answers
    for lp in (1, 3):
        with wt.Batch(views, sigmas, lp_ctas_per_sm=lp) as b:
            out = b.set_queries(q["tree"], q["kind"], q["c"], q["arg"])
            b.run()
            assert b.status_sync() == wt.WT_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint64), _expected(views, sigmas, q))
