"""Batched trees (one graph launch) against the CPU oracle, tree by tree."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402

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
        out = b.set_queries(q["tree"], q["kind"], q["c"], q["arg"])
        want = _expected(views, sigmas, q)
        for _ in range(2):  # the graph can be launched again
            out.fill_(0)
            b.run()
            assert b.status_sync() == wt.WT_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
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
