"""GPU parity of the minimal-alphabet extraction (wt_alphabet) against the
oracle's map: sparse and dense alphabets in all three widths, in place and
into a second array, one symbol, and a build on the extracted text."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402

pytestmark = pytest.mark.gpu

NP = {1: np.uint8, 2: np.uint16, 4: np.uint32}
TORCH = {1: torch.uint8, 2: torch.int16, 4: torch.int32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("w,n,k", [(1, 100003, 37), (1, 5000, 256), (2, 1 << 20, 3000), (2, 777, 1),
                                   (4, 1 << 20, 5000), (4, 123457, 70000)])
@pytest.mark.parametrize("inplace", [False, True])
def test_alphabet_matches_oracle(w, n, k, inplace):
    rng = np.random.default_rng(n + k + w)
    hi = 1 << (8 * w)
    pool = np.unique(rng.integers(0, hi, k, dtype=np.uint64)).astype(NP[w])  # k (or fewer) distinct values
    S = pool[rng.integers(0, pool.size, n)]
    S[0], S[-1] = pool[0], pool[-1]
    d = torch.from_numpy(S.view({1: np.uint8, 2: np.int16, 4: np.int32}[w]).copy()).cuda()
    out, vals, sigma = wt.alphabet(d, out=d if inplace else None)
    codes, values = oracle.alphabet_map(S)
    assert sigma == values.size
    assert np.array_equal(out.cpu().numpy().view(NP[w]).astype(np.int64), codes)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), values.astype(np.uint32))


def test_build_on_extracted_alphabet():
    rng = np.random.default_rng(9)
    values = np.array([3, 1000, 65535, 70000, 1 << 31], dtype=np.uint32)
    S = values[rng.integers(0, values.size, 200000)]
    d = torch.from_numpy(S.view(np.int32).copy()).cuda()
    codes, vals, sigma = wt.alphabet(d)
    assert sigma == 5
    with wt.build(codes, sigma) as t:
        i = torch.arange(0, 200000, 13, device="cuda", dtype=torch.int64)
        a = t.access(i).cpu().numpy().astype(np.int64)
        assert np.array_equal(vals.cpu().numpy().view(np.uint32)[a], S[i.cpu().numpy()])
        assert t.status_sync() == wt.WT_OK
