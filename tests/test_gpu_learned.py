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


def _level_model(t, o2, l, b, K, mode):
    """Ranks, their positions, segments and the model's predictions for level l,
    bit b, recomputed on the CPU from the exported model (None if no b-bits)."""
    size, ones = o2.level_size(l), o2.level_ones(l)
    total = ones if b else size - ones
    if total == 0:
        return None
    bits = o2.bits(l)
    pos = np.flatnonzero(bits == b).astype(np.int64)  # pos[k - 1] = select_b(l, k)
    samples = o2.export(oracle.EXPORT_S1 if b else oracle.EXPORT_S0, l)
    k, m, k0, k1, x0, x1 = omlp.segment_anchor_all(samples, total, size, K)
    eps = t.export(wt.EXPORT_EPS1 if b else wt.EXPORT_EPS0, l).astype(np.int64)
    nseg = total // (omlp.ANCHOR * K) + 1
    assert eps.size == nseg
    if mode == wt.LEARN_PLA:
        R = t.export(wt.EXPORT_RESID1 if b else wt.EXPORT_RESID0, l).astype(np.int64).reshape(nseg, 3)
        pred = omlp.predict_spline_all(k, k0, k1, x0, x1, R[m])
    else:
        R = None
        P = t.export(wt.EXPORT_MLP, l)
        # the kernel's FP32 chain, every fused multiply-add rounded once
        pred = omlp.predict_mlp_f32_all(k, k0, k1, x0, x1, P[b * 97:(b + 1) * 97])
    return dict(total=total, size=size, pos=pos, samples=samples, k=k, m=m, k0=k0, k1=k1, x0=x0, x1=x1, eps=eps,
                R=R, pred=pred, nseg=nseg)


def _unit(worst_max):
    """The bound's unit: the smallest 2^e with ceil(max / 2^e) <= 65535."""
    e = 0
    while (worst_max + (1 << e) - 1) >> e > 65535:
        e += 1
    return 1 << e


@pytest.mark.parametrize("mode", [wt.LEARN_PLA, wt.LEARN_MLP])
@pytest.mark.parametrize("n,sigma,K", [(150001, 300, 256), (1 << 22, 65536, 4096)])
def test_bounds_cover_every_error_the_cpu_recomputes(mode, n, sigma, K):
    """Every stored segment bound covers the error the CPU recomputes from the
    exported model at every rank k of every level and bit, and is the largest
    error rounded up to its unit; the fitted knots are non-decreasing and lie
    between the anchors."""
    sym = workloads.make_symbols(n, sigma, 2, "zipf", 1.2, seed=99, device="cuda")
    S = sym.cpu().numpy().view(np.uint16)
    o2 = oracle.O2Tree(S, sigma, K=K)
    with wt.build(sym, sigma, sample_k=K) as t:
        t.train_select(mode, steps=200)
        for l in range(o2.L):
            for b in (0, 1):
                d = _level_model(t, o2, l, b, K, mode)
                if d is None:
                    continue
                err = np.abs(d["pred"] - d["pos"])
                m, eps = d["m"], d["eps"]
                bad = np.flatnonzero(err > eps[m])
                assert bad.size == 0, (l, b, int(d["k"][bad[0]]), int(d["pred"][bad[0]]), int(d["pos"][bad[0]]),
                                       int(eps[m[bad[0]]]))
                worst = np.zeros(eps.size, np.int64)
                np.maximum.at(worst, m, err)
                unit = _unit(int(worst.max()))
                assert np.all(eps >= worst) and np.all(eps - worst < unit), (l, b)
                if mode == wt.LEARN_PLA:
                    for seg in range(d["nseg"]):
                        kn = omlp.anchor_knots(d["samples"], d["total"], d["size"], seg, K)
                        if kn[1] - kn[0] < 4:
                            continue
                        kap, xi = omlp.spline_knots(kn, d["R"][seg])
                        assert all(xi[i] <= xi[i + 1] for i in range(4)), (l, b, seg, xi)


def test_fitted_knots_match_the_least_squares_fit():
    """The GPU's knot residuals against the oracle's FP64 least-squares fit of
    the same segments (the GPU accumulates in FP32 and rounds to its residual
    unit; nearly every segment agrees within that)."""
    n, sigma, K = 1 << 21, 65536, 1024
    sym = workloads.make_symbols(n, sigma, 2, "zipf", 1.2, seed=31, device="cuda")
    S = sym.cpu().numpy().view(np.uint16)
    o2 = oracle.O2Tree(S, sigma, K=K)
    with wt.build(sym, sigma, sample_k=K) as t:
        t.train_select(wt.LEARN_PLA)
        checked = close = 0
        for l in (0, 1, 3):
            for b in (0, 1):
                d = _level_model(t, o2, l, b, K, wt.LEARN_PLA)
                if d is None:
                    continue
                unit = max(1, int(np.abs(d["R"]).max()) // 32767 + 1)
                for seg in range(0, d["nseg"], max(1, d["nseg"] // 40)):
                    kn = omlp.anchor_knots(d["samples"], d["total"], d["size"], seg, K)
                    if kn[1] - kn[0] < 4:
                        continue
                    sel = d["m"] == seg
                    ref = omlp.fit_spline_lsq(kn, d["k"][sel], d["pos"][d["k"][sel] - 1])
                    checked += 1
                    tol = 2 * unit + 2 + 1e-3 * np.abs(ref).max()
                    close += int(np.all(np.abs(d["R"][seg] - ref) <= tol))
        assert checked >= 40 and close >= 0.95 * checked, (close, checked)


def test_fitted_knots_narrow_the_window_over_the_untrained_line():
    """What training adds, on the learned-select workload's distribution (u16
    Zipf(1.2) over 65536, K = 4096): the mean window 2 eps + 1 of level 0 with
    fitted knots is at least 20 % narrower than with the untrained model (the
    line through the anchors), whose bounds the CPU computes."""
    n, sigma, K = 1 << 24, 65536, 4096
    sym = workloads.make_symbols(n, sigma, 2, "zipf", 1.2, seed=123, device="cuda")
    S = sym.cpu().numpy().view(np.uint16)
    o2 = oracle.O2Tree(S, sigma, K=K)
    with wt.build(sym, sigma, sample_k=K) as t:
        t.train_select(wt.LEARN_PLA)
        win_tr, win_un = [], []
        for b in (0, 1):
            d = _level_model(t, o2, 0, b, K, wt.LEARN_PLA)
            base = d["x0"] + ((d["k"] - d["k0"]) * (d["x1"] - d["x0"])) // (d["k1"] - d["k0"])
            worst = np.zeros(d["nseg"], np.int64)
            np.maximum.at(worst, d["m"], np.abs(base - d["pos"]))
            win_tr.append(2 * d["eps"] + 1)
            win_un.append(2 * worst + 1)
    tr, un = np.concatenate(win_tr).mean(), np.concatenate(win_un).mean()
    print(f"level 0 mean window: fitted knots {tr:.1f} bits, untrained line {un:.1f} bits")
    assert tr <= 0.8 * un


def test_training_the_network_does_not_worsen_the_fit():
    """The MLP (mode 2) on the same level data: the trained network's mean
    squared error of the position fraction is not above that of its starting
    point, the line through the anchors (g = 0).  On i.i.d. symbols the
    positions within a segment are a random walk around that line, so a model
    shared by all segments of a level has little to learn; the fitted knots of
    mode 1 are where the gain is."""
    n, sigma, K = 400003, 65536, 1024
    sym = workloads.make_symbols(n, sigma, 2, "zipf", 1.2, seed=123, device="cuda")
    S = sym.cpu().numpy().view(np.uint16)
    o2 = oracle.O2Tree(S, sigma, K=K)
    with wt.build(sym, sigma, sample_k=K) as t:
        t.train_select(wt.LEARN_MLP, steps=400)
        mse_trained = mse_linear = 0.0
        npts = 0
        for l in range(o2.L):
            P = t.export(wt.EXPORT_MLP, l).astype(np.float64)
            for b in (0, 1):
                size, ones = o2.level_size(l), o2.level_ones(l)
                total = ones if b else size - ones
                if total < 2 * omlp.ANCHOR * K:
                    continue
                samples = o2.export(oracle.EXPORT_S1 if b else oracle.EXPORT_S0, l)
                us, ts = [], []
                for k in range(1, total + 1, max(1, total // 2000)):
                    kn = omlp.anchor_knots(samples, total, size, k // (omlp.ANCHOR * K), K)
                    if k == kn[0]:
                        continue
                    us.append((k - kn[0]) / (kn[1] - kn[0]))
                    ts.append((o2.select_b(l, b, k) - kn[2]) / (kn[3] - kn[2]))
                us, ts = np.array(us), np.array(ts)
                y, _, _ = omlp.forward(P[b * 97:(b + 1) * 97], us)
                mse_trained += float(np.sum((us + y - ts) ** 2))
                mse_linear += float(np.sum((us - ts) ** 2))
                npts += us.size
    assert npts > 0
    print(f"fraction MSE: line {mse_linear / npts:.3e}, trained network {mse_trained / npts:.3e}")
    assert mse_trained <= mse_linear * 1.001
