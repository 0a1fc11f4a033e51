"""Device memory from the caller's allocator (wt_options.allocator).

A counting allocator backed by PyTorch's caching allocator records every
block libwt takes and returns.  With it, the build, the ordered query walks,
the host query pipeline and learned-select training give the same answers as
with libwt's own pool, and every block is returned.  Then the k-th request is
refused, for every k up to the number the sequence makes: the call that asked
returns WT_ENOMEM, the blocks live after the failure are exactly those live
before the call (the tree's own, or none for a build), and destroying the tree
returns the rest.  The failure is made on the host, by the callback; no GPU
fault is involved.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


class CountingAllocator:
    """wt_allocator on torch's caching allocator that refuses request number fail_at (1-based)."""

    def __init__(self, fail_at=None):
        self.calls = 0
        self.live = {}
        self.fail_at = fail_at
        self.streams = set()

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.fail_at is not None and self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
            self.live[p] = (int(nbytes), int(stream or 0))
            self.streams.add(int(stream or 0))
            return p

        def _free(ptr, stream, ctx):
            nbytes, s = self.live.pop(ptr)
            assert int(stream or 0) == s  # released on the stream it was allocated on
            torch.cuda.caching_allocator_delete(ptr)

        self._fa, self._ff = wt._ALLOC_FN(_alloc), wt._FREE_FN(_free)
        self.struct = wt.Allocator(self._fa, self._ff, None)


N = 1 << 26  # a tree above 64 MiB of levels and query batches of 2^16: the walks order their queries
SIGMA = 4096


def _inputs():
    sym = workloads.make_symbols(N, SIGMA, 2, "zipf", 1.1, seed=71, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(72)
    q = 1 << 16
    i = torch.randint(0, N, (q,), generator=g, device="cuda", dtype=torch.int64)
    S = sym.cpu().numpy().view(np.uint16)
    o1 = oracle.O1(S, SIGMA)
    cnt = torch.from_numpy(np.diff(o1.C).astype(np.int64)).cuda()
    present = torch.nonzero(cnt).flatten()
    c = present[torch.randint(0, present.numel(), (q,), generator=g, device="cuda")]
    j = (torch.rand(q, generator=g, device="cuda", dtype=torch.float64) * cnt[c]).to(torch.int64) + 1
    return sym, S, o1, i, c.to(torch.int32), j


def _sequence(sym, i, c, j, allocator, stream):
    """Build, then an ordered access and select walk, a host-pipeline select and
    PLA training; yields after each step so the caller can check the live blocks."""
    t = wt.build(sym, SIGMA, allocator=allocator, stream=stream)
    yield "build", t
    a = t.access(i, stream=stream)
    yield "access", a
    s = t.select(c, j, stream=stream)
    yield "select", s
    h = t.query_host(2, j.cpu(), c=c.cpu(), stream=stream, chunk=(1 << 15) + 1)
    stream.synchronize()
    yield "select_host", h
    t.train_select(wt.LEARN_PLA, stream=stream)
    yield "train", t
    t.close()


def test_allocator_backs_every_allocation_and_answers_match():
    sym, S, o1, i, c, j = _inputs()
    ca = CountingAllocator()
    stream = torch.cuda.Stream()
    res = {}
    tree = None
    for name, val in _sequence(sym, i, c, j, ca.struct, stream):
        res[name] = val
        if name == "build":
            tree = val
            assert len(ca.live) == 2  # the tree's header and level memory; scratch already returned
    stream.synchronize()
    assert ca.calls >= 8 and not ca.live
    assert ca.streams == {stream.cuda_stream}  # every request on the caller's stream
    ii, cc, jj = i.cpu().numpy().view(np.uint64), c.cpu().numpy().view(np.uint32), j.cpu().numpy().view(np.uint64)
    assert np.array_equal(res["access"].cpu().numpy().view(np.uint32), o1.access(ii))
    want = o1.select(cc, jj)
    assert np.array_equal(res["select"].cpu().numpy().view(np.uint64), want)
    assert np.array_equal(res["select_host"].numpy().view(np.uint64), want)
    del tree
    # the default binding allocator (torch's caching allocator) and libwt's pool give the same tree
    with wt.build(sym, SIGMA) as ta, wt.build(sym, SIGMA, allocator=None) as tb:
        for l in range(ta.levels):
            for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0, wt.EXPORT_S1):
                assert np.array_equal(ta.export(what, l), tb.export(what, l))


def test_every_refused_allocation_gives_enomem_and_leaks_nothing():
    sym, S, o1, i, c, j = _inputs()
    probe = CountingAllocator()
    stream = torch.cuda.Stream()
    for _ in _sequence(sym, i, c, j, probe.struct, stream):
        pass
    stream.synchronize()
    total = probe.calls
    assert total >= 8
    for k in range(1, total + 1):
        ca = CountingAllocator(fail_at=k)
        tree = None
        failed = None
        seq = _sequence(sym, i, c, j, ca.struct, stream)
        before = {}
        while True:
            before = dict(ca.live)
            try:
                name, val = next(seq)
            except StopIteration:
                break
            except wt.WTError as e:
                failed = e
                break
            if name == "build":
                tree = val
        stream.synchronize()
        assert failed is not None and failed.status == wt.WT_ENOMEM, (k, failed)
        assert ca.live == before, (k, "blocks leaked by the failed call")
        if tree is not None:
            # the tree still answers after a failed query or training call
            got = tree.access(i[:1000], stream=stream)
            stream.synchronize()
            assert np.array_equal(got.cpu().numpy().view(np.uint32), o1.access(i[:1000].cpu().numpy().view(np.uint64)))
            tree.close()
        seq.close()
        stream.synchronize()
        assert not ca.live, k
