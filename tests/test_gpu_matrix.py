"""GPU parity of the wavelet matrix layout (wt_options.layout = WT_LAYOUT_MATRIX):
every level's bits, L1/L2 counters and select samples against the oracle's
matrix, and every query against the definitional oracle O1, for all three
symbol widths, power-of-two and other alphabets, sizes spanning several tiles
with ragged tails, and the degenerate alphabets."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu

NP_OF_W = {1: np.uint8, 2: np.uint16, 4: np.uint32}
U64MAX = np.iinfo(np.uint64).max
U32MAX = np.iinfo(np.uint32).max


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


@pytest.mark.parametrize("n,sigma,w,dist", [(1000, 2, 1, "uniform"), (100003, 96, 1, "zipf"), (300001, 256, 1, "uniform"),
                                            (65536 * 3 + 5, 1000, 2, "uniform"), (200000, 65536, 2, "zipf"),
                                            (150001, 70000, 4, "uniform"), (5, 3, 1, "uniform")])
@pytest.mark.parametrize("K", [256, 4096])
def test_matrix_matches_oracle(n, sigma, w, dist, K):
    sym = workloads.make_symbols(n, sigma, w, dist, 1.0, seed=n + sigma, device="cuda")
    S = sym.cpu().numpy().view(NP_OF_W[w])
    om = oracle.OMatrix(S, sigma, K)
    with wt.build(sym, sigma, sample_k=K, layout=wt.LAYOUT_MATRIX) as t:
        inf = t.info()
        assert inf.layout == wt.LAYOUT_MATRIX and inf.levels == om.L
        for l in range(om.L):
            assert inf.level_size[l] == n and inf.level_ones[l] == n - om.zeros(l)
            for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
                assert np.array_equal(t.export(what, l), om.export(what, l)), (l, what)
        o1 = oracle.O1(S, sigma)
        rng = np.random.default_rng(n)
        q = 5000
        i = rng.integers(0, n, q).astype(np.uint64)
        i[:2] = [0, n - 1]
        assert np.array_equal(t.access(_dev(i, np.int64)).cpu().numpy().view(np.uint32), o1.access(i))
        c = rng.integers(0, sigma, q).astype(np.uint32)
        r = rng.integers(0, n + 1, q).astype(np.uint64)
        r[:2] = [0, n]
        assert np.array_equal(t.rank(_dev(c, np.int32), _dev(r, np.int64)).cpu().numpy().view(np.uint64),
                              o1.rank(c, r))
        counts = np.diff(o1.C)
        present = np.flatnonzero(counts)
        cs = present[rng.integers(0, present.size, q)].astype(np.uint32)
        j = (rng.random(q) * counts[cs]).astype(np.uint64) + 1
        j[0] = counts[cs[0]]
        assert np.array_equal(t.select(_dev(cs, np.int32), _dev(j, np.int64)).cpu().numpy().view(np.uint64),
                              o1.select(cs, j))
        assert t.status_sync() == wt.WT_OK


def test_matrix_invalid_queries_unsupported_parts_and_host_pipeline():
    n, sigma = 50000, 10
    sym = workloads.make_symbols(n, sigma, 1, "uniform", seed=4, device="cuda")
    S = sym.cpu().numpy()
    with wt.build(sym, sigma, layout=wt.LAYOUT_MATRIX) as t:
        assert t.access(_dev(np.array([n], np.uint64), np.int64)).cpu().numpy().view(np.uint32)[0] == U32MAX
        assert t.rank(_dev(np.array([sigma], np.uint32), np.int32),
                      _dev(np.array([0], np.uint64), np.int64)).cpu().numpy().view(np.uint64)[0] == U64MAX
        assert t.status_sync() == wt.WT_EQUERY
        with pytest.raises(wt.WTError) as e:
            t.train_select(wt.LEARN_PLA)
        assert e.value.status == wt.WT_EUNSUPPORTED
        with pytest.raises(wt.WTError):
            t.export(wt.EXPORT_NODES)
        # host-resident pipeline and a sorted large batch on the same layout
        o1 = oracle.O1(S, sigma)
        i = np.arange(0, n, 3, dtype=np.int64)
        out = t.query_host(0, torch.from_numpy(i).pin_memory(), chunk=1000)
        torch.cuda.synchronize()
        assert np.array_equal(out.numpy().view(np.uint32), o1.access(i.astype(np.uint64)))
        assert t.status_sync() == wt.WT_OK


def test_matrix_large_sorted_batches():
    w = workloads.WORKLOADS["text"]
    n = 1 << 27
    sym = workloads.make_symbols(n, w.sigma, 1, w.dist, w.zipf_s, seed=99, device="cuda")
    wl = workloads.Workload(w.name, w.index, n, w.sigma, 1, w.dist, w.zipf_s, {k: 1 << 17 for k in w.queries},
                            w.sample_k)
    q = workloads.make_queries(wl, sym, seed=98)
    with wt.build(sym, w.sigma) as tree, wt.build(sym, w.sigma, layout=wt.LAYOUT_MATRIX) as mat:
        assert mat.info().tree_bytes >= 64 << 20
        assert torch.equal(mat.access(q["access_i"]), tree.access(q["access_i"]))
        assert torch.equal(mat.rank(q["rank_c"], q["rank_i"]), tree.rank(q["rank_c"], q["rank_i"]))
        assert torch.equal(mat.select(q["select_c"], q["select_j"]), tree.select(q["select_c"], q["select_j"]))
        assert mat.status_sync() == wt.WT_OK and tree.status_sync() == wt.WT_OK
