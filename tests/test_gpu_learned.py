"""Learned select on the GPU: gradients, exactness, bounds, and what training adds."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from paper_2505_03372_gb300 import binding as wt  # noqa: E402
from paper_2505_03372_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu
NP_OF_W = {1: np.uint8, 2: np.uint16, 4: np.uint32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _tensors(P):
    return P[:32], P[32:64], P[64:96], P[96:]


def test_mlp_gradient_matches_fp64_reference():
    rng = np.random.default_rng(5)
    for n in (1, 37, 4096, 16384):
        P = rng.normal(scale=0.5, size=omlp.NPARAM).astype(np.float32)
        u = rng.random(n).astype(np.float32)
        t = (u + 0.2 * rng.normal(size=n) + 0.1).astype(np.float32)
        g_gpu, loss_gpu = wt.mlp_gradient(P, u, t)
        loss_cpu, g_cpu = omlp.loss_and_grad(P.astype(np.float64), u.astype(np.float64), t.astype(np.float64))
        assert abs(loss_gpu - loss_cpu) <= 1e-4 * max(1.0, abs(loss_cpu))
        for a, b in zip(_tensors(g_gpu.astype(np.float64)), _tensors(g_cpu)):
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert rel <= 1e-4, (n, rel)


CASES = [
    # n, sigma, w, dist, s, K
    (200003, 96, 1, "zipf", 1.0, 256),
    (300001, 65536, 2, "zipf", 1.2, 4096),
    (1 << 20, 256, 1, "uniform", 1.0, 1024),
    (100001, (1 << 20) - 3, 4, "uniform", 1.0, 512),
    (70000, 2, 1, "uniform", 1.0, 256),
]


def _select_queries(counts, rng, q=20000):
    present = np.nonzero(counts)[0]
    c = present[rng.integers(0, present.size, q)].astype(np.uint32)
    j = (rng.random(q) * counts[c]).astype(np.uint64) + 1
    extra = present[: min(16, present.size)]
    c = np.concatenate([c, extra, extra]).astype(np.uint32)
    j = np.concatenate([j, np.ones(extra.size, np.uint64), counts[extra].astype(np.uint64)])
    return c, j


@pytest.mark.parametrize("mode", [wt.LEARN_PLA, wt.LEARN_MLP])
@pytest.mark.parametrize("n,sigma,w,dist,s,K", CASES)
def test_learned_select_is_exact(mode, n, sigma, w, dist, s, K):
    sym = workloads.make_symbols(n, sigma, w, dist, s, seed=n + 7 * sigma, device="cuda")
    S = sym.cpu().numpy().view(NP_OF_W[w])
    o1 = oracle.O1(S, sigma)
    counts = np.diff(o1.C).astype(np.int64)
    c, j = _select_queries(counts, np.random.default_rng(n))
    with wt.build(sym, sigma, sample_k=K) as t:
        with pytest.raises(wt.WTError):
            t.select_learned(torch.from_numpy(c.view(np.int32)).cuda(), torch.from_numpy(j.view(np.int64)).cuda())
        t.train_select(mode, steps=200)
        dc, dj = torch.from_numpy(c.view(np.int32)).cuda(), torch.from_numpy(j.view(np.int64)).cuda()
        got = t.select_learned(dc, dj).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, o1.select(c, j))
        assert np.array_equal(got, t.select(dc, dj).cpu().numpy().view(np.uint64))
        assert t.status_sync() == wt.WT_OK
        assert t.learned_info().fallbacks == 0


@pytest.mark.parametrize("mode", [wt.LEARN_PLA, wt.LEARN_MLP])
@pytest.mark.parametrize("n,sigma,K", [(150001, 300, 256), (1 << 22, 65536, 4096)])
def test_bounds_cover_every_error_the_cpu_recomputes(mode, n, sigma, K):
    """Every stored segment bound covers the error the CPU recomputes at every rank k of every level and bit."""
    sym = workloads.make_symbols(n, sigma, 2, "zipf", 1.2, seed=99, device="cuda")
    S = sym.cpu().numpy().view(np.uint16)
    o2 = oracle.O2Tree(S, sigma, K=K)
    with wt.build(sym, sigma, sample_k=K) as t:
        t.train_select(mode, steps=200)
        for l in range(o2.L):
            size, ones = o2.level_size(l), o2.level_ones(l)
            bits = o2.bits(l)
            P = t.export(wt.EXPORT_MLP, l)
            for b in (0, 1):
                total = ones if b else size - ones
                if total == 0:
                    continue
                pos = np.flatnonzero(bits == b).astype(np.int64)  # pos[k - 1] = select_b(l, k)
                assert pos.size == total
                samples = o2.export(oracle.EXPORT_S1 if b else oracle.EXPORT_S0, l)
                eps = t.export(wt.EXPORT_EPS1 if b else wt.EXPORT_EPS0, l).astype(np.int64)
                assert eps.size == total // K + 1
                k, m, k0, k1, x0, x1 = omlp.segment_knots_all(samples, total, size, K)
                if mode == wt.LEARN_PLA:
                    pred = omlp.predict_pla_all(k, k0, k1, x0, x1)
                else:
                    # the kernel's FP32 chain, every fused multiply-add rounded once
                    pred = omlp.predict_mlp_f32_all(k, k0, k1, x0, x1, P[b * 97:(b + 1) * 97])
                err = np.abs(pred - pos)
                bad = np.flatnonzero(err > eps[m])
                assert bad.size == 0, (l, b, int(k[bad[0]]), int(pred[bad[0]]), int(pos[bad[0]]), int(eps[m[bad[0]]]))
                # the bound is tight for PLA: some rank of every segment attains it
                if mode == wt.LEARN_PLA:
                    worst = np.zeros(eps.size, np.int64)
                    np.maximum.at(worst, m, err)
                    assert np.array_equal(worst, eps), (l, b)


def test_training_reduces_the_fitted_error():
    """What the trained network adds over linear interpolation between samples
    (its untrained starting point): the mean squared error of the predicted
    position fraction, recomputed on the CPU over a stride of every level's b-bits."""
    n, sigma, K = 400003, 65536, 4096
    sym = workloads.make_symbols(n, sigma, 2, "zipf", 1.2, seed=123, device="cuda")
    S = sym.cpu().numpy().view(np.uint16)
    o2 = oracle.O2Tree(S, sigma, K=K)
    with wt.build(sym, sigma, sample_k=K) as t:
        t.train_select(wt.LEARN_MLP, steps=400)
        inf_mlp = t.learned_info()
        mse_trained = mse_linear = 0.0
        npts = 0
        for l in range(o2.L):
            size, ones = o2.level_size(l), o2.level_ones(l)
            P = t.export(wt.EXPORT_MLP, l).astype(np.float64)
            for b in (0, 1):
                total = ones if b else size - ones
                if total < 2 * K:
                    continue
                samples = o2.export(oracle.EXPORT_S1 if b else oracle.EXPORT_S0, l)
                us, ts = [], []
                for k in range(1, total + 1, max(1, total // 2000)):
                    kn = omlp.knots(samples, total, size, k // K, K)
                    if k == kn[0]:
                        continue
                    us.append((k - kn[0]) / (kn[1] - kn[0]))
                    ts.append((o2.select_b(l, b, k) - kn[2]) / (kn[3] - kn[2]))
                us, ts = np.array(us), np.array(ts)
                y, _, _ = omlp.forward(P[b * 97:(b + 1) * 97], us)
                mse_trained += float(np.sum((us + y - ts) ** 2))
                mse_linear += float(np.sum((us - ts) ** 2))
                npts += us.size
        t.train_select(wt.LEARN_PLA)
        inf_pla = t.learned_info()
    assert npts > 0
    print(f"fraction MSE: linear {mse_linear / npts:.3e}, trained {mse_trained / npts:.3e}; "
          f"mean bound level 0 b=1: PLA {inf_pla.eps_mean[0][1]:.1f}, MLP {inf_mlp.eps_mean[0][1]:.1f}")
    assert mse_trained <= mse_linear * 1.001
