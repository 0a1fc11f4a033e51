"""GPU parity of the standalone binary rank / select (wt_bitvector_rank,
wt_bitvector_select) over bitvectors whose support wt_bitvector_support_static
built, against the oracle's definitions: sizes around 512-bit blocks and
65536-bit L1 blocks, empty and full bitvectors, the fills and layouts of the
bitvector benchmark, every boundary query and the out-of-range ones."""
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


def _bits(words, nbits):
    return np.unpackbits(words.cpu().numpy().view(np.uint8), bitorder="little")[:nbits]


CASES = [(1, 0.5, "uniform"), (511, 0.5, "uniform"), (512, 1.0, "uniform"), (513, 0.0, "uniform"),
         (65536 + 3, 0.1, "uniform"), (3 * 65536 + 777, 0.9, "uniform"), ((1 << 22) + 5, 0.5, "uniform"),
         ((1 << 22) + 5, 0.1, "adversarial"), ((1 << 22) + 5, 0.9, "adversarial"), (1 << 20, 1.0, "uniform")]


@pytest.mark.parametrize("nbits,fill,layout", CASES)
@pytest.mark.parametrize("K", [256, 4096])
def test_rank_select_match_oracle(nbits, fill, layout, K):
    words = workloads.make_bitvector(nbits, fill, layout, seed=1000 + nbits % 977, device="cuda")
    bits = _bits(words, nbits)
    bv = wt.Bitvector(words, nbits, sample_k=K)
    assert bv.ones == int(bits.sum())
    rng = np.random.default_rng(nbits)
    q = 20000
    i = rng.integers(0, nbits + 1, q).astype(np.int64)
    i[:4] = [0, nbits, nbits + 1, nbits + 100]
    out, full = guarded(q, torch.int64)
    got = bv.rank(torch.from_numpy(i).cuda(), out=out).cpu().numpy().view(np.uint64)
    assert intact(full, q), "rank wrote outside its output"
    want = np.full(q, U64MAX, np.uint64)
    ok = i <= nbits
    want[ok] = oracle.bv_rank(bits, i[ok])
    assert np.array_equal(got, want)
    assert bv.status_sync() == wt.WT_EQUERY
    for b in (0, 1):
        cnt = int((bits == b).sum())
        j = rng.integers(1, cnt + 1, q).astype(np.int64) if cnt else np.ones(q, np.int64)
        j[:3] = [0, cnt + 1, max(cnt, 1)]
        if cnt:
            j[3:3 + min(cnt, 50)] = np.arange(1, min(cnt, 50) + 1)  # the first b-bits
        out, full = guarded(q, torch.int64)
        got = bv.select(b, torch.from_numpy(j).cuda(), out=out).cpu().numpy().view(np.uint64)
        assert intact(full, q), "select wrote outside its output"
        want = np.full(q, U64MAX, np.uint64)
        ok = (j >= 1) & (j <= cnt)
        want[ok] = oracle.bv_select(bits, b, j[ok])
        assert np.array_equal(got, want), (b, np.flatnonzero(got != want)[:5])
        assert bv.status_sync() == wt.WT_EQUERY  # j = 0 and j = cnt + 1


def test_bitvector_argument_checks():
    words = workloads.make_bitvector(5000, 0.5, seed=3, device="cuda")
    bv = wt.Bitvector(words, 5000)
    L = wt.lib()
    s = torch.cuda.current_stream().cuda_stream
    i = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    h = torch.zeros(4, dtype=torch.int64)
    assert L.wt_bitvector_rank(bv.words.data_ptr(), 0, bv.l1.data_ptr(), bv.l2.data_ptr(), i.data_ptr(),
                               out.data_ptr(), 4, None, s) == wt.WT_EINVAL
    assert L.wt_bitvector_rank(bv.words.data_ptr(), 5000, bv.l1.data_ptr(), bv.l2.data_ptr(), h.data_ptr(),
                               out.data_ptr(), 4, None, s) == wt.WT_EINVAL
    assert L.wt_bitvector_select(bv.words.data_ptr(), 5000, bv.ones, 2, bv.l1.data_ptr(), bv.l2.data_ptr(),
                                 bv.s0.data_ptr(), bv.s1.data_ptr(), 4096, i.data_ptr(), out.data_ptr(), 4, None,
                                 s) == wt.WT_EINVAL
    assert L.wt_bitvector_select(bv.words.data_ptr(), 5000, bv.ones, 1, bv.l1.data_ptr(), bv.l2.data_ptr(),
                                 bv.s0.data_ptr(), bv.s1.data_ptr(), 1000, i.data_ptr(), out.data_ptr(), 4, None,
                                 s) == wt.WT_EINVAL
    assert L.wt_bitvector_select(bv.words.data_ptr() + 8, 5000, bv.ones, 1, bv.l1.data_ptr(), bv.l2.data_ptr(),
                                 bv.s0.data_ptr(), bv.s1.data_ptr(), 4096, i.data_ptr(), out.data_ptr(), 4, None,
                                 s) == wt.WT_EINVAL
