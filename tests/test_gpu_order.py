"""Ordering as a step of its own: wt_order_queries on one stream while the
build's level passes run on another, then wt_walk_ordered.  The answers must
equal the one-step calls and the definitions (O1), invalid queries included,
on the unsorted path (small batch) and the sorted one (2^17 + 1 queries on a
2^27 tree)."""
import ctypes
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402
from guard import guarded, intact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _host(sym, w):
    return sym.cpu().numpy().view({1: np.uint8, 2: np.uint16, 4: np.uint32}[w])


def _u(t, bits):
    return t.cpu().numpy().view(np.uint32 if bits == 32 else np.uint64)


@pytest.mark.parametrize("n,sigma,w,nq", [(200003, 96, 1, 5001), (300001, 1000, 2, 4097), (1 << 27, 96, 1, (1 << 17) + 1)])
def test_order_on_a_side_stream_then_walk(n, sigma, w, nq):
    sym = workloads.make_symbols(n, sigma, w, "zipf", 1.0, seed=n + 3 * sigma, device="cuda")
    wl = workloads.Workload("ord", 91, n, sigma, w, "zipf", 1.0, queries={"access": nq, "rank": nq, "select": nq})
    q = workloads.make_queries(wl, sym, seed=11)
    q["access_i"][:3] = n + 5            # out of range
    q["rank_c"][3:5] = sigma + 2
    q["select_j"][5:7] = 0
    S = _host(sym, w)
    o1 = oracle.O1(S, sigma)
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    with wt.build(sym, sigma) as t:
        # the orders run on the side stream while the level passes run on main
        with torch.cuda.stream(side):
            oa = t.order(wt.ORDER_ACCESS, q["access_i"], stream=side)
            orank = t.order(wt.ORDER_RANK, q["rank_i"], c=q["rank_c"], stream=side)
            osel = t.order(wt.ORDER_SELECT, q["select_j"], c=q["select_c"], stream=side)
            kinds = (torch.arange(nq, device="cuda") % 3).to(torch.uint8)
            marg = torch.where(kinds == 0, q["access_i"], torch.where(kinds == 1, q["rank_i"], q["select_j"]))
            omix = t.order(wt.ORDER_MIXED, marg, c=q["rank_c"], kinds=kinds, stream=side)
        out_a, full_a = guarded(nq, torch.int32)
        out_r, full_r = guarded(nq, torch.int64)
        out_s, full_s = guarded(nq, torch.int64)
        out_m, full_m = guarded(nq, torch.int64)
        t.walk(oa, out=out_a, stream=main)
        t.walk(orank, out=out_r, stream=main)
        t.walk(osel, out=out_s, stream=main)
        t.walk(omix, out=out_m, stream=main)
        for o in (oa, orank, osel, omix):
            o.close(stream=main)
        assert t.status_sync() == wt.WT_EQUERY
        for full, cnt in ((full_a, nq), (full_r, nq), (full_s, nq), (full_m, nq)):
            assert intact(full, cnt)
        # the one-step calls on the same batch
        assert np.array_equal(_u(out_a, 32), _u(t.access(q["access_i"]), 32))
        assert np.array_equal(_u(out_r, 64), _u(t.rank(q["rank_c"], q["rank_i"]), 64))
        assert np.array_equal(_u(out_s, 64), _u(t.select(q["select_c"], q["select_j"]), 64))
        assert np.array_equal(_u(out_m, 64), _u(t.query_mixed(kinds, q["rank_c"], marg), 64))
        t.status_sync()
    # and the definitions
    ia = q["access_i"].cpu().numpy().astype(np.uint64)
    ok = ia < n
    want = np.full(nq, 0xFFFFFFFF, np.uint32)
    want[ok] = o1.access(ia[ok])
    assert np.array_equal(_u(out_a, 32), want)
    c, i = q["rank_c"].cpu().numpy().astype(np.uint32), q["rank_i"].cpu().numpy().astype(np.uint64)
    ok = c < sigma
    want = np.full(nq, np.uint64(2**64 - 1), np.uint64)
    want[ok] = o1.rank(c[ok], i[ok])
    assert np.array_equal(_u(out_r, 64), want)
    c, j = q["select_c"].cpu().numpy().astype(np.uint32), q["select_j"].cpu().numpy().astype(np.uint64)
    ok = j > 0
    want = np.full(nq, np.uint64(2**64 - 1), np.uint64)
    want[ok] = o1.select(c[ok], j[ok])
    assert np.array_equal(_u(out_s, 64), want)


def test_order_errors_and_empty_batch():
    sym = workloads.make_symbols(5000, 10, 1, "uniform", 1.0, seed=1, device="cuda")
    lib = wt.lib()
    with wt.build(sym, 10) as t, wt.build(sym, 10) as t2:
        i = torch.arange(100, dtype=torch.int64, device="cuda")
        h = ctypes.c_void_p()
        assert lib.wt_order_queries(t._h, 4, None, None, i.data_ptr(), 100, None, ctypes.byref(h)) == wt.WT_EINVAL
        assert h.value is None
        assert lib.wt_order_queries(t._h, wt.ORDER_RANK, None, None, i.data_ptr(), 100, None,
                                    ctypes.byref(h)) == wt.WT_EINVAL  # rank without c
        assert lib.wt_order_queries(t._h, wt.ORDER_ACCESS, None, None, i.data_ptr(), 100, None, None) == wt.WT_EINVAL
        o = t.order(wt.ORDER_ACCESS, i)
        out = torch.empty(100, dtype=torch.int32, device="cuda")
        # an order walks only on the tree it was made for
        assert lib.wt_walk_ordered(t2._h, o._h, out.data_ptr(), None) == wt.WT_EINVAL
        t.walk(o, out=out)
        assert np.array_equal(_u(out, 32), _u(t.access(i), 32))
        o.close()
        assert lib.wt_order_destroy(None, None) == wt.WT_EINVAL
        empty = t.order(wt.ORDER_SELECT, torch.empty(0, dtype=torch.int64, device="cuda"),
                        c=torch.empty(0, dtype=torch.int32, device="cuda"))
        assert t.walk(empty).numel() == 0
        empty.close()
        assert t.status_sync() == wt.WT_OK


def test_order_on_a_batch_tree_is_unsupported():
    views = [workloads.make_symbols(3000, 7, 2, "uniform", 1.0, seed=s, device="cuda") for s in (1, 2)]
    with wt.Batch(views, [7, 7]) as b:
        b.run()
        tv = b.tree(0)
        h = ctypes.c_void_p()
        i = torch.arange(10, dtype=torch.int64, device="cuda")
        assert wt.lib().wt_order_queries(tv._h, wt.ORDER_ACCESS, None, None, i.data_ptr(), 10, None,
                                         ctypes.byref(h)) == wt.WT_EUNSUPPORTED
