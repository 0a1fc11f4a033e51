"""wt_bitvector_support_static: the allocation-free entry point.

Callers that cannot allocate device memory (code running inside an allocator
or pool callback, loops that must avoid the driver's allocation path, hosts
that hand out only fixed buffers) get the rank counters and select samples of
a bitvector from this call, with every buffer supplied by them and the kernel's
scratch living in a static array inside libwt.

The test compares its output with what wt_build stores for the same bits: a
tree over the alphabet {0, 1} has a single level whose bits are the symbols,
so wt_export of that level is the reference; and with the oracle's counters
and samples, computed from prefix sums of the bits.  Each case calls the entry
point twice in a row (the static scratch keeps the previous call's contents
and must be cleared by the call itself).  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from guard import guarded, intact  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _reference(bits01, K):
    sym = torch.from_numpy(bits01.astype(np.uint8)).cuda()
    with wt.build(sym, 2, sample_k=K) as t:
        return {what: t.export(what, 0) for what in (wt.EXPORT_BITS, wt.EXPORT_L1, wt.EXPORT_L2, wt.EXPORT_S0,
                                                      wt.EXPORT_S1)}


def _call(words_dev, nbits, K, cap):
    """One call of the entry point through the C ABI; all buffers are allocated here, by the caller."""
    n1, n2 = nbits // 65536 + 1, nbits // 512 + 1
    l1, g1 = guarded(n1, torch.int64)
    l2, g2 = guarded(n2, torch.int16)
    s0, g3 = guarded(cap, torch.int64)
    s1, g4 = guarded(cap, torch.int64)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ones = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = wt.lib().wt_bitvector_support_static(words_dev.data_ptr(), nbits, K, l1.data_ptr(), l2.data_ptr(),
                                               s0.data_ptr(), s1.data_ptr(), cap, status.data_ptr(), ones.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream)
    assert st == wt.WT_OK, wt.status_str(st)
    torch.cuda.synchronize()
    assert status.item() == 0
    assert intact(g1, n1) and intact(g2, n2) and intact(g3, cap) and intact(g4, cap), "wrote outside an output"
    return (l1.cpu().numpy().view(np.uint64), l2.cpu().numpy().view(np.uint16), s0.cpu().numpy().view(np.uint64),
            s1.cpu().numpy().view(np.uint64), int(ones.item()))


@pytest.mark.parametrize("nbits,density,K", [
    (1, 0.5, 256),
    (1000, 0.5, 256),
    (65536, 0.5, 256),          # exactly one tile
    (65537, 0.1, 512),
    (131072, 0.9, 4096),        # ends on a tile boundary
    (200003, 0.5, 4096),
    ((1 << 22) + 12345, 0.016, 4096),
])
def test_matches_wt_build_twice(nbits, density, K):
    rng = np.random.default_rng(nbits)
    bits = (rng.random(nbits) < density).astype(np.uint8)
    ref = _reference(bits, K)
    words = torch.from_numpy(ref[wt.EXPORT_BITS].view(np.int64).copy()).cuda()
    cap = nbits // K + 2
    o_l1, o_l2, o_s0, o_s1 = oracle.bitvector_support(bits, K)
    for _ in range(2):
        l1, l2, s0, s1, ones = _call(words, nbits, K, cap)
        assert np.array_equal(l1, ref[wt.EXPORT_L1])
        assert np.array_equal(l2, ref[wt.EXPORT_L2])
        n0, n1 = ref[wt.EXPORT_S0].size, ref[wt.EXPORT_S1].size
        assert np.array_equal(s0[:n0], ref[wt.EXPORT_S0])
        assert np.array_equal(s1[:n1], ref[wt.EXPORT_S1])
        # and against the definition
        assert np.array_equal(l1, o_l1) and np.array_equal(l2, o_l2)
        assert np.array_equal(s0[:o_s0.size], o_s0) and np.array_equal(s1[:o_s1.size], o_s1)
        assert ones == int(bits.sum())


def test_rejects_inputs_beyond_the_static_scratch():
    words = torch.zeros(16, dtype=torch.int64, device="cuda")
    small = torch.zeros(16, dtype=torch.int64, device="cuda")
    l2 = torch.zeros(16, dtype=torch.int16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    too_big = (1 << 32) + 1
    st = wt.lib().wt_bitvector_support_static(words.data_ptr(), too_big, 4096, small.data_ptr(), l2.data_ptr(),
                                               small.data_ptr(), small.data_ptr(), too_big // 4096 + 2, None, None, s)
    assert st == wt.WT_EINVAL
    # a host buffer is refused before anything is enqueued
    host = np.zeros(16, np.uint64)
    st = wt.lib().wt_bitvector_support_static(host.ctypes.data, 64, 4096, small.data_ptr(), l2.data_ptr(),
                                               small.data_ptr(), small.data_ptr(), 2, None, None, s)
    assert st == wt.WT_EINVAL
    st = wt.lib().wt_bitvector_support_static(words.data_ptr(), 64, 4096, small.data_ptr(), l2.data_ptr(),
                                               small.data_ptr(), small.data_ptr(), 2, None, host.ctypes.data, s)
    assert st == wt.WT_EINVAL
