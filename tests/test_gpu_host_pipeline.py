"""GPU parity of the host-resident query pipeline (wt_query_host): queries and
answers in host memory, pinned or pageable, split into chunks (ragged last
chunk, chunks large enough to be walked in sorted order, one chunk), against
the definitional oracle O1 and against the device entry points."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu

U64MAX = np.iinfo(np.uint64).max
U32MAX = np.iinfo(np.uint32).max


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _cpu(a, dtype, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dtype)
    return t.pin_memory() if pinned else t


def _queries(o1, n, sigma, q, rng):
    counts = np.diff(o1.C)
    present = np.nonzero(counts)[0]
    i = rng.integers(0, n + 1, q).astype(np.uint64)
    i[:3] = [n + 1, n + 7, 0]  # two out of range
    c = present[rng.integers(0, present.size, q)].astype(np.uint32)
    j = (rng.random(q) * counts[c]).astype(np.uint64) + 1
    j[:2] = [0, counts[c[1]] + 1]  # invalid ranks
    return i, c, j


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("chunk", [3000, 0, 1 << 20])
def test_query_host_matches_oracle(pinned, chunk):
    n, sigma = 300001, 96
    sym = workloads.make_symbols(n, sigma, 1, "zipf", 1.0, seed=77, device="cuda")
    S = sym.cpu().numpy()
    o1 = oracle.O1(S, sigma)
    rng = np.random.default_rng(78)
    q = 10007
    i, c, j = _queries(o1, n, sigma, q, rng)
    with wt.build(sym, sigma) as t:
        acc = t.query_host(0, _cpu(i.astype(np.int64), torch.int64, pinned), chunk=chunk,
                           out=_cpu(np.zeros(q, np.int32), torch.int32, pinned))
        rk = t.query_host(1, _cpu(i.astype(np.int64), torch.int64, pinned),
                          c=_cpu(c.astype(np.int32), torch.int32, pinned), chunk=chunk,
                          out=_cpu(np.zeros(q, np.int64), torch.int64, pinned))
        sl = t.query_host(2, _cpu(j.astype(np.int64), torch.int64, pinned),
                          c=_cpu(c.astype(np.int32), torch.int32, pinned), chunk=chunk,
                          out=_cpu(np.zeros(q, np.int64), torch.int64, pinned))
        kind = rng.integers(0, 3, q).astype(np.uint8)
        arg = np.where(kind == 2, j, np.minimum(i, n)).astype(np.uint64)
        mx = t.query_host(3, _cpu(arg.astype(np.int64), torch.int64, pinned),
                          c=_cpu(c.astype(np.int32), torch.int32, pinned),
                          kinds=_cpu(kind, torch.uint8, pinned), chunk=chunk,
                          out=_cpu(np.zeros(q, np.int64), torch.int64, pinned))
        torch.cuda.synchronize()
        assert t.status_sync() == wt.WT_EQUERY  # the invalid queries above
        want_a = np.full(q, U32MAX, np.uint32)
        ok = i < n
        want_a[ok] = o1.access(i[ok])
        assert np.array_equal(acc.numpy().view(np.uint32), want_a)
        want_r = np.full(q, U64MAX, np.uint64)
        ok = i <= n
        want_r[ok] = o1.rank(c[ok], i[ok])
        assert np.array_equal(rk.numpy().view(np.uint64), want_r)
        want_s = np.full(q, U64MAX, np.uint64)
        ok = (j >= 1) & (j <= np.diff(o1.C)[c])
        want_s[ok] = o1.select(c[ok], j[ok])
        assert np.array_equal(sl.numpy().view(np.uint64), want_s)
        want_m = np.full(q, U64MAX, np.uint64)
        for kd, f in ((0, lambda m: o1.access(arg[m]).astype(np.uint64)), (1, lambda m: o1.rank(c[m], arg[m]))):
            m = (kind == kd) & (arg < n)
            want_m[m] = f(m)
        m = (kind == 2) & ok
        want_m[m] = o1.select(c[m], arg[m])
        m = (kind == 1) & (arg == n)
        want_m[m] = o1.rank(c[m], arg[m])
        assert np.array_equal(mx.numpy().view(np.uint64), want_m)


def test_query_host_sorted_chunks_equal_device_calls():
    """Chunks of at least 2^16 queries on a tree above 64 MB go through the query
    ordering; the answers must equal the device entry points' answers slot by slot."""
    w = workloads.WORKLOADS["text"]
    n = 1 << 27
    w = workloads.Workload(w.name, w.index, n, w.sigma, w.symbol_bytes, w.dist, w.zipf_s,
                           {k: (1 << 17) + 5 for k in w.queries}, w.sample_k)
    sym = workloads.make_symbols(n, w.sigma, 1, w.dist, w.zipf_s, seed=5151, device="cuda")
    q = workloads.make_queries(w, sym, seed=5252)
    with wt.build(sym, w.sigma) as t:
        assert t.info().tree_bytes >= 64 << 20
        chunk = (1 << 16) + 3
        a = t.query_host(0, q["access_i"].cpu().pin_memory(), chunk=chunk)
        r = t.query_host(1, q["rank_i"].cpu().pin_memory(), c=q["rank_c"].cpu().pin_memory(), chunk=chunk)
        s = t.query_host(2, q["select_j"].cpu().pin_memory(), c=q["select_c"].cpu().pin_memory(), chunk=chunk)
        torch.cuda.synchronize()
        assert torch.equal(a, t.access(q["access_i"]).cpu())
        assert torch.equal(r, t.rank(q["rank_c"], q["rank_i"]).cpu())
        assert torch.equal(s, t.select(q["select_c"], q["select_j"]).cpu())
        # a sample against the definition
        S = sym.cpu().numpy()
        o1 = oracle.O1(S, w.sigma)
        k = np.arange(0, a.numel(), 997)
        assert np.array_equal(a.numpy().view(np.uint32)[k], o1.access(q["access_i"].cpu().numpy().view(np.uint64)[k]))
        assert t.status_sync() == wt.WT_OK


def test_query_host_rejects_device_memory():
    sym = workloads.make_symbols(5000, 10, 1, "uniform", seed=8, device="cuda")
    with wt.build(sym, 10) as t:
        L = wt.lib()
        d_arg = torch.zeros(16, dtype=torch.int64, device="cuda")
        h_arg = torch.zeros(16, dtype=torch.int64)
        h_out = torch.zeros(16, dtype=torch.int32)
        d_out = torch.zeros(16, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        assert L.wt_query_host(t._h, 0, None, None, d_arg.data_ptr(), h_out.data_ptr(), 16, 0, s) == wt.WT_EINVAL
        assert L.wt_query_host(t._h, 0, None, None, h_arg.data_ptr(), d_out.data_ptr(), 16, 0, s) == wt.WT_EINVAL
        assert L.wt_query_host(t._h, 1, None, None, h_arg.data_ptr(), h_out.data_ptr(), 16, 0, s) == wt.WT_EINVAL
        assert L.wt_query_host(t._h, 4, None, None, h_arg.data_ptr(), h_out.data_ptr(), 16, 0, s) == wt.WT_EINVAL
        assert L.wt_query_host(t._h, 0, None, None, h_arg.data_ptr(), h_out.data_ptr(), 0, 0, s) == wt.WT_OK
        assert L.wt_query_host(t._h, 0, None, None, h_arg.data_ptr(), h_out.data_ptr(), 16, 0, s) == wt.WT_OK
        torch.cuda.synchronize()
        assert h_out.numpy().view(np.uint32)[0] == sym[0].item()
        assert t.status_sync() == wt.WT_OK


@pytest.mark.parametrize("w,n,sigma,pinned", [(1, (1 << 27) + 12345, 96, True), (2, (1 << 25) + 7, 65536, False),
                                              (4, 3 * (1 << 24) + 4321, 5000, True), (4, 300001, 70000, True),
                                              (1, 1, 2, False)])
def test_build_from_host_memory_matches_oracle(w, n, sigma, pinned):
    """wt_build_host (64 MiB chunks copied while the histogram runs; the u32
    case has three whole chunks and a ragged fourth) against the naive oracle
    tree, every level's bits, counters and samples, C and the node table, and
    its answers against the definitions; also equal to wt_build's tree."""
    sym = workloads.make_symbols(n, sigma, w, "zipf" if sigma < 1000 else "uniform", 1.0, seed=n % 1000 + w,
                                 device="cuda")
    h = sym.cpu()
    if pinned:
        h = h.pin_memory()
    S = h.numpy().view({1: np.uint8, 2: np.uint16, 4: np.uint32}[w])
    o2 = oracle.O2Tree(S, sigma, K=4096)
    with wt.build(sym, sigma) as td, wt.build(h, sigma) as th:
        a, b = td.info(), th.info()
        assert a.levels == b.levels == o2.L
        for l in range(b.levels):
            assert b.level_size[l] == o2.level_size(l) and b.level_ones[l] == o2.level_ones(l)
            for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
                g = th.export(what, l)
                assert np.array_equal(g, o2.export(what, l)), (l, what)
                assert np.array_equal(g, td.export(what, l)), (l, what)
        assert np.array_equal(th.export(wt.EXPORT_C), o2.export(oracle.EXPORT_C))
        if o2.L:
            assert np.array_equal(th.export(wt.EXPORT_NODES), o2.export(oracle.EXPORT_NODES))
        o1 = oracle.O1(S, sigma)
        rng = np.random.default_rng(n)
        q = 20000
        i = rng.integers(0, n, q).astype(np.uint64)
        cnt = np.diff(o1.C).astype(np.int64)
        present = np.flatnonzero(cnt)
        c = present[rng.integers(0, present.size, q)].astype(np.uint32)
        j = (rng.random(q) * cnt[c]).astype(np.uint64) + 1
        di = torch.from_numpy(i.view(np.int64)).cuda()
        dc, dj = torch.from_numpy(c.view(np.int32)).cuda(), torch.from_numpy(j.view(np.int64)).cuda()
        assert np.array_equal(th.access(di).cpu().numpy().view(np.uint32), o1.access(i))
        assert np.array_equal(th.rank(dc, di).cpu().numpy().view(np.uint64), o1.rank(c, i))
        assert np.array_equal(th.select(dc, dj).cpu().numpy().view(np.uint64), o1.select(c, j))
        assert th.status_sync() == wt.WT_OK
