"""GPU parity: libwt (through the C ABI) against the CPU oracle, bit for bit.

Every exported structure (level bits, L1/L2 counters, select samples, C, codes,
node table) is compared with the naive oracle tree O2, and every query result
with the definitional oracle O1 (and O2 on the small cases).  Sizes span
several 32 KiB tiles, ragged tails, exact tile / L1-block ends, all three
symbol widths, power-of-two and reduced alphabets, and the degenerate cases.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402
from guard import guarded, intact  # noqa: E402

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


def _host(sym, w):
    return sym.cpu().numpy().view(NP_OF_W[w])


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _compare_structure(t, o2, sigma):
    inf = t.info()
    assert inf.levels == o2.L
    for l in range(o2.L):
        assert inf.level_size[l] == o2.level_size(l), l
        assert inf.level_ones[l] == o2.level_ones(l), l
        for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
            g = t.export(what, l)
            r = o2.export(what, l)
            assert g.shape == r.shape, (l, what)
            if not np.array_equal(g, r):
                bad = np.nonzero(g != r)[0]
                raise AssertionError(f"level {l} export {what}: {bad.size} mismatches, first at {bad[:5]}: "
                                     f"gpu {g[bad[:5]]} oracle {r[bad[:5]]}")
    assert np.array_equal(t.export(wt.EXPORT_C), o2.export(oracle.EXPORT_C))
    assert np.array_equal(t.export(wt.EXPORT_CODES), o2.export(oracle.EXPORT_CODES)[:sigma])
    assert np.array_equal(t.export(wt.EXPORT_LENS), o2.export(oracle.EXPORT_LENS)[:sigma])
    gn, rn = t.export(wt.EXPORT_NODES), o2.export(oracle.EXPORT_NODES)
    assert gn.shape == rn.shape
    assert np.array_equal(gn, rn)


def _edge_queries(n, counts, rng, q=4000):
    sigma = counts.size
    i_acc = np.concatenate([rng.integers(0, max(n, 1), q), [0, max(n - 1, 0)]]).astype(np.uint64)
    c_rank = rng.integers(0, sigma, q + 4).astype(np.uint32)
    i_rank = np.concatenate([rng.integers(0, n + 1, q), [0, n, n, 0]]).astype(np.uint64)
    present = np.nonzero(counts)[0]
    if present.size:
        c_sel = present[rng.integers(0, present.size, q)].astype(np.uint32)
        j_sel = (rng.random(q) * counts[c_sel]).astype(np.uint64) + 1
        # first and last occurrence of a few symbols
        extra = present[: min(8, present.size)]
        c_sel = np.concatenate([c_sel, extra, extra]).astype(np.uint32)
        j_sel = np.concatenate([j_sel, np.ones(extra.size, np.uint64), counts[extra].astype(np.uint64)])
    else:
        c_sel = np.zeros(0, np.uint32)
        j_sel = np.zeros(0, np.uint64)
    return i_acc, c_rank, i_rank, c_sel, j_sel


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def _run_queries(t, S, sigma, n, rng, o2=None):
    o1 = oracle.O1(S, sigma)
    counts = np.diff(o1.C).astype(np.int64)
    i_acc, c_rank, i_rank, c_sel, j_sel = _edge_queries(n, counts, rng)
    if n:
        out, full = guarded(i_acc.size, torch.int32)
        got = _u32(t.access(_dev(i_acc, np.int64), out=out))
        assert intact(full, i_acc.size), "access wrote outside its output"
        assert np.array_equal(got, o1.access(i_acc)), "access"
        if o2 is not None:
            assert np.array_equal(got, o2.access(i_acc))
    out, full = guarded(i_rank.size, torch.int64)
    got = _u64(t.rank(_dev(c_rank, np.int32), _dev(i_rank, np.int64), out=out))
    assert intact(full, i_rank.size), "rank wrote outside its output"
    want = o1.rank(c_rank, i_rank)
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0][:5]
        raise AssertionError(f"rank mismatch at {bad}: c={c_rank[bad]} i={i_rank[bad]} gpu={got[bad]} want={want[bad]}")
    if c_sel.size:
        out, full = guarded(c_sel.size, torch.int64)
        got = _u64(t.select(_dev(c_sel, np.int32), _dev(j_sel, np.int64), out=out))
        assert intact(full, c_sel.size), "select wrote outside its output"
        want = o1.select(c_sel, j_sel)
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0][:5]
            raise AssertionError(f"select mismatch at {bad}: c={c_sel[bad]} j={j_sel[bad]} gpu={got[bad]} want={want[bad]}")
    assert t.status_sync() == wt.WT_OK


# (n, sigma, symbol bytes, distribution, K)
CASES = [
    (1, 2, 1, "uniform", 256),
    (17, 3, 1, "uniform", 256),
    (1000, 4, 1, "uniform", 256),
    (32767, 6, 1, "uniform", 256),        # one partial u8 tile
    (32768, 25, 1, "uniform", 256),       # exactly one u8 tile
    (65536, 243, 1, "zipf", 256),         # exactly one L1 block
    (65537, 96, 1, "zipf", 4096),
    (131072, 2, 1, "uniform", 256),       # ends on an L1 boundary
    (200003, 256, 1, "uniform", 4096),    # several tiles + ragged tail
    (1 << 20, 256, 1, "uniform", 4096),   # the plain workload's shape
    (1 << 20, 96, 1, "zipf", 4096),
    (16384, 7, 2, "uniform", 256),        # exactly one u16 tile
    (100000, 1000, 2, "uniform", 256),
    (196608, 4097, 2, "uniform", 512),
    (300001, 65536, 2, "zipf", 4096),
    (8192, 3, 4, "uniform", 256),         # exactly one u32 tile
    (50000, 5, 4, "uniform", 256),
    (100001, (1 << 20) - 3, 4, "uniform", 1024),
    (262144, 1 << 20, 4, "uniform", 4096),
    # the level before the last also writes the last level's bits (its nodes
    # average 16 tiles or more): every width, level 0 re-encoding or not,
    # tiles that span two nodes, ragged ends
    (300001, 3, 1, "uniform", 256),       # u8, L = 2: level 0 re-encodes and folds
    (600001, 7, 1, "uniform", 256),       # u8, L = 3: folds at level 1
    (300001, 4, 2, "uniform", 256),       # u16, L = 2
    (300001, 6, 2, "uniform", 512),       # u16, L = 3
    (150001, 4, 4, "uniform", 256),       # u32, L = 2
    (200003, 6, 4, "uniform", 256),       # u32, L = 3
]


@pytest.mark.parametrize("n,sigma,w,dist,K", CASES)
def test_build_and_queries_match_oracle(n, sigma, w, dist, K):
    s = 1.2 if sigma == 65536 else 1.0
    sym = workloads.make_symbols(n, sigma, w, dist, s, seed=n * 31 + sigma, device="cuda")
    S = _host(sym, w)
    t = wt.build(sym, sigma, sample_k=K)
    o2 = oracle.O2Tree(S, sigma, K=K)
    _compare_structure(t, o2, sigma)
    _run_queries(t, S, sigma, n, np.random.default_rng(n + sigma), o2=o2 if n <= 300001 else None)
    t.close()


@pytest.mark.parametrize("name", ["plain", "text", "large_alphabet", "learned"])
def test_workload_shapes_reduced_n(name):
    """Each workload's distribution and alphabet at n = 2^21 (oracle compares everything)."""
    w0 = workloads.WORKLOADS[name]
    w, sym, q, counts = workloads.make_workload(name, device="cuda", n=1 << 21, scale_queries=0.01)
    S = _host(sym, w.symbol_bytes)
    t = wt.build(sym, w.sigma, sample_k=w0.sample_k)
    o2 = oracle.O2Tree(S, w.sigma, K=w0.sample_k)
    _compare_structure(t, o2, w.sigma)
    o1 = oracle.O1(S, w.sigma)
    if "access_i" in q:
        assert np.array_equal(_u32(t.access(q["access_i"])), o1.access(q["access_i"].cpu().numpy()))
    if "rank_c" in q:
        assert np.array_equal(_u64(t.rank(q["rank_c"], q["rank_i"])), o1.rank(q["rank_c"].cpu().numpy(), q["rank_i"].cpu().numpy()))
    if "select_c" in q:
        assert np.array_equal(_u64(t.select(q["select_c"], q["select_j"])),
                              o1.select(q["select_c"].cpu().numpy(), q["select_j"].cpu().numpy()))
    if "mixed_kind" in q:
        _check_mixed(t, q["mixed_kind"], q["mixed_c"], q["mixed_arg"], o1)
    assert t.status_sync() == wt.WT_OK
    t.close()


def _check_mixed(t, kind, c, arg, o1):
    got = _u64(t.query_mixed(kind, c, arg))
    k = kind.cpu().numpy()
    cc = c.cpu().numpy().view(np.uint32)
    aa = arg.cpu().numpy().view(np.uint64)
    want = np.full(k.size, U64MAX, np.uint64)
    m = k == 0
    want[m] = o1.access(aa[m]).astype(np.uint64)
    m = k == 1
    want[m] = o1.rank(cc[m], aa[m])
    m = k == 2
    want[m] = o1.select(cc[m], aa[m])
    assert np.array_equal(got, want)


def test_mixed_with_invalid_kind():
    n, sigma = 50000, 300
    sym = workloads.make_symbols(n, sigma, 2, "uniform", seed=5, device="cuda")
    S = _host(sym, 2)
    t = wt.build(sym, sigma)
    o1 = oracle.O1(S, sigma)
    rng = np.random.default_rng(9)
    q = 3000
    kind = rng.integers(0, 4, q).astype(np.uint8)  # 3 is not a query kind
    c = rng.integers(0, sigma, q).astype(np.uint32)
    counts = np.diff(o1.C)
    arg = np.where(kind == 2, (rng.random(q) * counts[c]).astype(np.uint64) + 1, rng.integers(0, n, q).astype(np.uint64))
    got = _u64(t.query_mixed(torch.from_numpy(kind).cuda(), _dev(c, np.int32), _dev(arg.astype(np.uint64), np.int64)))
    want = np.full(q, U64MAX, np.uint64)
    for kd, f in ((0, lambda m: o1.access(arg[m]).astype(np.uint64)), (1, lambda m: o1.rank(c[m], arg[m])),
                  (2, lambda m: o1.select(c[m], arg[m]))):
        m = kind == kd
        want[m] = f(m)
    assert np.array_equal(got, want)
    assert t.status_sync() == wt.WT_EQUERY  # the kind-3 queries
    assert t.status_sync() == wt.WT_OK      # sticky status was cleared
    t.close()


def test_invalid_queries_give_sentinels_and_status():
    n, sigma = 10000, 10
    sym = workloads.make_symbols(n, sigma, 1, "uniform", seed=3, device="cuda")
    S = _host(sym, 1)
    counts = np.bincount(S, minlength=sigma)
    t = wt.build(sym, sigma)
    assert _u32(t.access(_dev(np.array([n, n + 5], np.uint64), np.int64))).tolist() == [U32MAX, U32MAX]
    assert t.status_sync() == wt.WT_EQUERY
    r = _u64(t.rank(_dev(np.array([sigma, 0], np.uint32), np.int32), _dev(np.array([0, n + 1], np.uint64), np.int64)))
    assert r.tolist() == [U64MAX, U64MAX]
    assert t.status_sync() == wt.WT_EQUERY
    s = _u64(t.select(_dev(np.array([0, 1, sigma], np.uint32), np.int32),
                      _dev(np.array([0, counts[1] + 1, 1], np.uint64), np.int64)))
    assert s.tolist() == [U64MAX] * 3
    assert t.status_sync() == wt.WT_EQUERY
    # valid queries afterwards are unaffected
    assert _u32(t.access(_dev(np.array([0], np.uint64), np.int64)))[0] == S[0]
    assert t.status_sync() == wt.WT_OK
    t.close()


def test_symbol_out_of_range_is_reported():
    sym = torch.tensor([1, 2, 3, 9, 0, 1], dtype=torch.uint8, device="cuda")
    with pytest.raises(wt.WTError) as e:
        wt.build(sym, 5)
    assert e.value.status == wt.WT_ESYMBOL


def test_empty_and_single_symbol_alphabet():
    t = wt.build(torch.zeros(0, dtype=torch.uint8, device="cuda"), 7)
    r = _u64(t.rank(_dev(np.array([0, 3], np.uint32), np.int32), _dev(np.array([0, 0], np.uint64), np.int64)))
    assert r.tolist() == [0, 0]
    assert _u32(t.access(_dev(np.array([0], np.uint64), np.int64))).tolist() == [U32MAX]
    assert t.status_sync() == wt.WT_EQUERY
    t.close()
    n = 1000
    t = wt.build(torch.zeros(n, dtype=torch.uint8, device="cuda"), 1)
    assert t.levels == 0
    i = np.array([0, 5, n - 1], np.uint64)
    assert _u32(t.access(_dev(i, np.int64))).tolist() == [0, 0, 0]
    assert _u64(t.rank(_dev(np.zeros(3, np.uint32), np.int32), _dev(np.array([0, 7, n], np.uint64), np.int64))).tolist() == [0, 7, n]
    assert _u64(t.select(_dev(np.zeros(3, np.uint32), np.int32), _dev(np.array([1, 8, n], np.uint64), np.int64))).tolist() == [0, 7, n - 1]
    assert t.status_sync() == wt.WT_OK
    t.close()


def test_rejected_pointers():
    from paper_2505_03372_gb300.binding import Options, lib

    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    opt = Options(sample_k=4096)
    # misaligned device pointer
    assert lib().wt_build(buf.data_ptr() + 1, 32, 4, 1, ctypes.byref(opt), None, ctypes.byref(h)) == wt.WT_EINVAL
    # host pointer
    host = np.zeros(64, np.uint8)
    assert lib().wt_build(host.ctypes.data, 32, 4, 1, ctypes.byref(opt), None, ctypes.byref(h)) == wt.WT_EINVAL
    t = wt.build(buf, 4)
    out = np.zeros(4, np.uint32)
    idx = np.zeros(4, np.uint64)
    assert lib().wt_access(t._h, idx.ctypes.data, out.ctypes.data, 4, None) == wt.WT_EINVAL
    t.close()


def test_repeated_builds_and_profile_counts():
    wt.profile_reset()
    sym = workloads.make_symbols(100000, 96, 1, "zipf", seed=11, device="cuda")
    for _ in range(3):
        with wt.build(sym, 96) as t:
            t.access(torch.zeros(10, dtype=torch.int64, device="cuda"))
    rep = wt.profile_report()
    assert rep["access"]["launches"] == 3
    assert rep["level_pass_u8"]["launches"] == 3 * 7
    assert wt.profile_launches() >= 3 * 8


@pytest.mark.slow
@pytest.mark.parametrize("name", ["text", "large_alphabet", "learned"])
def test_full_size_workloads_match_oracle(name):
    """Full-size inputs (2^30 u8 Zipf over 96, 2^28 u32 over 2^20, 2^30 u16
    Zipf over 65536) in the bench's launch configuration: every level's bits,
    L1/L2 counters and samples, C and the node table against the naive oracle
    tree (built on the host cores, level by level), and sampled queries
    against the definitions."""
    w, sym, q, counts = workloads.make_workload(name, device="cuda", scale_queries=0.002)
    t = wt.build(sym, w.sigma, sample_k=w.sample_k)
    S = _host(sym, w.symbol_bytes)
    del sym
    o2 = oracle.O2Tree(S, w.sigma, K=w.sample_k)
    inf = t.info()
    assert inf.levels == o2.L
    for l in range(o2.L):
        assert inf.level_size[l] == o2.level_size(l) and inf.level_ones[l] == o2.level_ones(l), l
        for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
            g = t.export(what, l)
            r = o2.export(what, l)
            if not np.array_equal(g, r):
                bad = np.flatnonzero(g != r) if g.shape == r.shape else np.array([-1])
                raise AssertionError(f"{name} level {l} export {what}: {bad.size} mismatches, first at {bad[:5]}")
            del g, r
    assert np.array_equal(t.export(wt.EXPORT_C), o2.export(oracle.EXPORT_C))
    assert np.array_equal(t.export(wt.EXPORT_NODES), o2.export(oracle.EXPORT_NODES))
    del o2
    o1 = oracle.O1(S, w.sigma)
    for key, f in (("access_i", lambda: (_u32(t.access(q["access_i"])), o1.access(q["access_i"].cpu().numpy()))),
                   ("rank_c", lambda: (_u64(t.rank(q["rank_c"], q["rank_i"])), o1.rank(q["rank_c"].cpu().numpy(), q["rank_i"].cpu().numpy()))),
                   ("select_c", lambda: (_u64(t.select(q["select_c"], q["select_j"])), o1.select(q["select_c"].cpu().numpy(), q["select_j"].cpu().numpy())))):
        if key in q:
            g, r = f()
            assert np.array_equal(g, r), key
    if "mixed_kind" in q:
        _check_mixed(t, q["mixed_kind"], q["mixed_c"], q["mixed_arg"], o1)
    assert t.status_sync() == wt.WT_OK
    t.close()


def test_bounded_wait_times_out_and_context_survives():
    """A look-back whose predecessor never publishes gives up after its poll
    limit, reports WT_ETIMEOUT through the status word, and the GPU keeps
    working (a build right after it is still exact)."""
    from paper_2505_03372_gb300.binding import lib

    import time

    t0 = time.perf_counter()
    assert lib().wt_selftest_lookback_timeout(1 << 16, None) == wt.WT_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    sym = workloads.make_symbols(50000, 96, 1, "zipf", 1.0, seed=1, device="cuda")
    S = _host(sym, 1)
    with wt.build(sym, 96) as t:
        i = np.arange(0, 50000, 7, dtype=np.uint64)
        assert np.array_equal(_u32(t.access(_dev(i, np.int64))), S[i.astype(np.int64)].astype(np.uint32))
        assert t.status_sync() == wt.WT_OK


@pytest.mark.parametrize("name,n,nq", [("text", 1 << 27, 1 << 17), ("large_alphabet", 1 << 25, 1 << 17)])
def test_large_batches_in_walk_order(name, n, nq):
    """Batches of at least 2^16 queries on trees above 64 MB are walked in bucket
    order (by position, or by code prefix and position / rank); every answer must
    still land in its own slot and equal the definition, invalid queries included."""
    w = workloads.WORKLOADS[name]
    w = workloads.Workload(w.name, w.index, n, w.sigma, w.symbol_bytes, w.dist, w.zipf_s,
                           {k: nq for k in w.queries}, w.sample_k)
    sym = workloads.make_symbols(n, w.sigma, w.symbol_bytes, w.dist, w.zipf_s, seed=4242, device="cuda")
    q = workloads.make_queries(w, sym, seed=4343)
    S = _host(sym, w.symbol_bytes)
    o1 = oracle.O1(S, w.sigma)
    with wt.build(sym, w.sigma) as t:
        assert t.info().tree_bytes >= 64 << 20
        if "access_i" in q:
            i = q["access_i"].clone()
            i[:7] = n + torch.arange(7, device="cuda")  # out of range: sentinel in place
            g = _u32(t.access(i))
            ii = i.cpu().numpy()
            want = np.full(ii.size, np.uint32(0xFFFFFFFF), np.uint32)
            ok = ii < n
            want[ok] = o1.access(ii[ok])
            assert np.array_equal(g, want)
            assert t.status_sync() == wt.WT_EQUERY
            assert np.array_equal(_u64(t.rank(q["rank_c"], q["rank_i"])),
                                  o1.rank(q["rank_c"].cpu().numpy(), q["rank_i"].cpu().numpy()))
            assert np.array_equal(_u64(t.select(q["select_c"], q["select_j"])),
                                  o1.select(q["select_c"].cpu().numpy(), q["select_j"].cpu().numpy()))
        if "mixed_kind" in q:
            _check_mixed(t, q["mixed_kind"], q["mixed_c"], q["mixed_arg"], o1)
        assert t.status_sync() == wt.WT_OK


@pytest.mark.slow
def test_more_than_2_to_the_32_symbols():
    """A text longer than 2^32 symbols (u8 over sigma = 5, 3 levels): positions,
    L1 counters and samples pass 2^32, so every 64-bit path of the build and
    the walks is taken.  Every level against the naive oracle tree, queries
    (including positions and ranks near the end) against the definitions."""
    n = (1 << 32) + 12345
    sigma = 5
    sym = workloads.make_symbols(n, sigma, 1, "uniform", seed=2024, device="cuda")
    with wt.build(sym, sigma) as t:
        S = _host(sym, 1)
        del sym
        o2 = oracle.O2Tree(S, sigma, K=4096)
        inf = t.info()
        assert inf.levels == o2.L == 3
        for l in range(o2.L):
            assert inf.level_size[l] == o2.level_size(l) and inf.level_ones[l] == o2.level_ones(l), l
            for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
                assert np.array_equal(t.export(what, l), o2.export(what, l)), (l, what)
        assert int(t.export(wt.EXPORT_S0, 0)[-1]) > (1 << 32)  # sample positions past 2^32
        assert np.array_equal(t.export(wt.EXPORT_NODES), o2.export(oracle.EXPORT_NODES))
        del o2
        o1 = oracle.O1(S, sigma)
        counts = np.diff(o1.C).astype(np.int64)
        rng = np.random.default_rng(7)
        q = 20000
        i = np.concatenate([rng.integers(0, n, q), [0, n - 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 1]]).astype(np.uint64)
        c = rng.integers(0, sigma, i.size).astype(np.uint32)
        assert np.array_equal(_u32(t.access(_dev(i, np.int64))), o1.access(i))
        ir = i.copy()
        ir[-1] = n  # rank at the very end
        assert np.array_equal(_u64(t.rank(_dev(c, np.int32), _dev(ir, np.int64))), o1.rank(c, ir))
        j = (rng.random(i.size) * counts[c]).astype(np.uint64) + 1
        j[-5:] = counts[c[-5:]]  # last occurrences, far past 2^32
        got = _u64(t.select(_dev(c, np.int32), _dev(j, np.int64)))
        want = o1.select(c, j)
        assert np.array_equal(got, want)
        assert int(want.max()) > (1 << 32)
        assert t.status_sync() == wt.WT_OK


@pytest.mark.parametrize("n,sigma,w,nq", [
    (200003, 96, 1, 4001),         # 7 levels: one select per thread
    (200003, 1000, 2, 4001),       # 10 levels: two per thread, unsorted
    (1 << 27, 1000, 2, (1 << 17) + 1),  # two per thread, in walk order
])
def test_select_walk_pairs_with_odd_counts_and_invalid_queries(n, sigma, w, nq):
    """Deep trees walk their selects two per thread in lockstep.  An odd batch
    leaves the last thread one query; invalid queries (symbol out of range,
    j = 0, j past the count) sit next to valid ones in the same pairs.  Every
    valid answer equals the definition, every invalid one is the sentinel."""
    sym = workloads.make_symbols(n, sigma, w, "zipf", 1.0, seed=n + sigma, device="cuda")
    S = _host(sym, w)
    o1 = oracle.O1(S, sigma)
    counts = np.diff(o1.C).astype(np.int64)
    present = np.nonzero(counts)[0]
    rng = np.random.default_rng(nq)
    c = present[rng.integers(0, present.size, nq)].astype(np.uint32)
    j = (rng.random(nq) * counts[c]).astype(np.uint64) + 1
    bad = rng.random(nq) < 0.01
    kinds = rng.integers(0, 3, nq)
    c[bad & (kinds == 0)] = sigma + 5
    j[bad & (kinds == 1)] = 0
    jb = bad & (kinds == 2)
    j[jb] = counts[c[jb]].astype(np.uint64) + 1
    with wt.build(sym, sigma) as t:
        assert (t.info().levels >= 8) == (sigma >= 256)
        out, full = guarded(nq, torch.int64)
        got = _u64(t.select(_dev(c, np.int32), _dev(j, np.int64), out=out))
        assert intact(full, nq), "select wrote outside its output"
        want = np.full(nq, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64)
        ok = ~bad
        want[ok] = o1.select(c[ok], j[ok])
        assert np.array_equal(got, want)
        assert t.status_sync() == wt.WT_EQUERY
