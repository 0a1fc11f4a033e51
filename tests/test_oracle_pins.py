"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: the values the paper
prints for its worked example and for code counts, closed-form space
overheads, a pointer-based tree built by recursion on the sequence, pure-Python
definitions of access/rank/select, the textbook invariants, and a second
algorithm for the codes (Algorithm 3 against the recursive split).
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _ceil_lg(x):
    return 0 if x <= 1 else int(x - 1).bit_length()


# --------------------------------------------------------------------------
# codes (Section 5.1, Algorithm 3)
# --------------------------------------------------------------------------

def test_alg3_matches_recursive_split():
    for sigma in range(1, 5001):
        c1, l1, L1 = oracle.codes_split(sigma)
        c2, l2, L2 = oracle.codes_alg3(sigma)
        assert L1 == L2 == _ceil_lg(sigma), sigma
        assert np.array_equal(c1, c2), sigma
        assert np.array_equal(l1, l2), sigma


@pytest.mark.parametrize("sigma", list(range(1, 300)) + [1000, 4095, 4097, 65535, 65536, 96, (1 << 20) - 3])
def test_code_properties(sigma):
    code, ln, L = oracle.codes_split(sigma)
    code = code[:sigma].astype(object)
    ln = ln[:sigma].astype(int)
    assert L == _ceil_lg(sigma)
    if sigma == 1:
        assert ln[0] == 0
        return
    # lengths never increase with the symbol (Section 5.1)
    assert all(ln[s] >= ln[s + 1] for s in range(sigma - 1))
    # every internal node has two children: Kraft sum is exactly one
    assert sum(2 ** (L - int(x)) for x in ln) == 2 ** L
    # codes are strictly increasing and prefix-free as left-aligned values
    for s in range(sigma - 1):
        assert code[s] + 2 ** (L - ln[s]) <= code[s + 1]
    if sigma & (sigma - 1) == 0:
        assert all(int(code[s]) == s for s in range(sigma)) and all(x == L for x in ln)


def test_shorter_code_counts_from_paper():
    facts = _golden("paper_facts.json")["shorter_code_counts"]
    for k, expected in facts.items():
        if k.startswith("_"):
            continue
        sigma = int(k)
        _, ln, L = oracle.codes_split(sigma)
        assert int((ln[:sigma] < L).sum()) == expected, sigma


# --------------------------------------------------------------------------
# worked example of Sections 5.2-5.4
# --------------------------------------------------------------------------

def test_worked_example():
    g = _golden("worked_example.json")
    alpha = g["alphabet"]
    S = np.array([alpha.index(ch) for ch in g["text"]], np.uint8)
    sigma = len(alpha)
    t = oracle.O2Tree(S, sigma, K=2)
    o1 = oracle.O1(S, sigma)
    C = t.export(oracle.EXPORT_C)

    # levels equal the pointer-based tree concatenated level by level
    ref = brute.pointer_tree_levels(list(S), sigma)
    assert t.L == len(ref) == 2
    for l in range(t.L):
        assert list(t.bits(l)) == ref[l]

    a = g["access"]
    i = a["i"]
    assert t.access([i])[0] == alpha.index(a["answer"]) == o1.access([i])[0]
    assert t.bits(0)[i] == 1  # goes right at the root
    i1 = t.rank_b(0, 1, i) - t.rank_b(0, 1, int(C[0]))
    assert i1 == a["level1_index_in_node"]
    node1 = int(C[2])  # right child of the root starts at symbol c
    assert t.bits(1)[node1 + i1] == a["level1_bit"]

    r = g["rank"]
    c = alpha.index(r["c"])
    after0 = r["i"] - (t.rank_b(0, 0, r["i"]) - t.rank_b(0, 0, 0))
    assert after0 == r["after_level0"]
    res = t.rank_b(1, 0, node1 + after0) - t.rank_b(1, 0, node1)
    assert res == r["answer"] == t.rank([c], [r["i"]])[0] == o1.rank([c], [r["i"]])[0]

    s = g["select"]
    c = alpha.index(s["c"])
    k1 = t.rank_b(1, 0, node1) + s["j"]
    assert s["level1_select"] == {"bit": 0, "k": s["j"]}
    pos1 = t.select_b(1, 0, k1) - node1
    assert pos1 == s["level1_index_in_node"]
    k0 = t.rank_b(0, 1, 0) + pos1 + 1
    assert k0 == s["level0_select"]["k"]
    ans = t.select_b(0, 1, k0)
    assert ans == t.select([c], [s["j"]])[0] == o1.select([c], [s["j"]])[0] == brute.select(list(S), c, s["j"])


# --------------------------------------------------------------------------
# brute force on small inputs
# --------------------------------------------------------------------------

def _check_all_queries(S, sigma, K):
    Sl = [int(x) for x in S]
    n = len(Sl)
    t = oracle.O2Tree(S, sigma, K=K)
    o1 = oracle.O1(S, sigma)
    # access
    if n:
        idx = np.arange(n, dtype=np.uint64)
        want = np.array(Sl, np.uint32)
        assert np.array_equal(t.access(idx), want)
        assert np.array_equal(o1.access(idx), want)
    # rank for every (c, i)
    cs = np.repeat(np.arange(sigma, dtype=np.uint32), n + 1)
    ii = np.tile(np.arange(n + 1, dtype=np.uint64), sigma)
    want = np.array([brute.rank(Sl, int(c), int(i)) for c, i in zip(cs, ii)], np.uint64)
    assert np.array_equal(t.rank(cs, ii), want)
    assert np.array_equal(o1.rank(cs, ii), want)
    # select for every valid (c, j)
    pairs = [(c, j) for c in range(sigma) for j in range(1, Sl.count(c) + 1)]
    if pairs:
        cs = np.array([p[0] for p in pairs], np.uint32)
        js = np.array([p[1] for p in pairs], np.uint64)
        want = np.array([brute.select(Sl, c, j) for c, j in pairs], np.uint64)
        assert np.array_equal(t.select(cs, js), want)
        assert np.array_equal(o1.select(cs, js), want)
    # out-of-range queries report the sentinel
    assert t.access([n])[0] == np.iinfo(np.uint32).max
    assert t.rank([0], [n + 1])[0] == np.iinfo(np.uint64).max
    assert t.rank([sigma], [0])[0] == np.iinfo(np.uint64).max
    assert t.select([0], [0])[0] == np.iinfo(np.uint64).max
    assert t.select([0], [Sl.count(0) + 1])[0] == np.iinfo(np.uint64).max
    # level bits equal the pointer-based tree; counters and samples by counting
    ref = brute.pointer_tree_levels(Sl, sigma)
    assert t.L == (len(ref) if n else t.L)
    for l in range(t.L):
        bits = [int(x) for x in t.bits(l)]
        if n:
            assert bits == ref[l], (l, sigma)
        L1, L2, s0, s1 = brute.counters(bits, K)
        assert list(t.export(oracle.EXPORT_L1, l)) == L1
        assert list(t.export(oracle.EXPORT_L2, l)) == L2
        assert list(t.export(oracle.EXPORT_S0, l)) == s0
        assert list(t.export(oracle.EXPORT_S1, l)) == s1
    # node table: start = C[a], r0 = zeros before start, mid = C[a + prevPow2(b-a)]
    _check_nodes(t, Sl, sigma)
    return t


def _check_nodes(t, Sl, sigma):
    nodes = t.export(oracle.EXPORT_NODES)
    C = [0] * (sigma + 1)
    for s in Sl:
        C[s + 1] += 1
    for c in range(sigma):
        C[c + 1] += C[c]

    def pp2(x):
        p = 1
        while p * 2 < x:
            p *= 2
        return p

    seen = set()
    frontier = [(0, sigma, 0, 0)]
    while frontier:
        nxt = []
        for a, b, d, p in frontier:
            if b - a < 2:
                continue
            slot = (1 << d) - 1 + p
            seen.add(slot)
            start, r0, mid, valid = (int(x) for x in nodes[slot])
            assert valid == 1
            assert start == C[a]
            bits = [int(x) for x in t.bits(d)]
            assert r0 == bits[:start].count(0)
            m = a + pp2(b - a)
            assert mid == C[m]
            nxt += [(a, m, d + 1, 2 * p), (m, b, d + 1, 2 * p + 1)]
        frontier = nxt
    for slot in range(nodes.shape[0]):
        if slot not in seen:
            assert nodes[slot][3] == 0


@pytest.mark.parametrize("sigma", range(1, 9))
def test_brute_tiny_exhaustive_sizes(sigma):
    rng = np.random.default_rng(1000 + sigma)
    for n in range(0, 65):
        S = rng.integers(0, sigma, n).astype(np.uint8)
        _check_all_queries(S, sigma, K=3)


@pytest.mark.parametrize("sigma", [1, 2, 3, 5, 6, 7, 11, 25, 96, 100, 129, 200, 243, 255, 256, 257, 300])
def test_brute_random(sigma):
    rng = np.random.default_rng(sigma)
    for n in (1, 17, 500, 1500):
        dt = np.uint8 if sigma <= 256 else np.uint16
        S = rng.integers(0, sigma, n).astype(dt)
        _check_all_queries(S, sigma, K=7)


def test_invariants_medium():
    rng = np.random.default_rng(7)
    sigma = 96
    p = 1.0 / np.arange(1, sigma + 1)
    S = rng.choice(sigma, size=1 << 16, p=p / p.sum()).astype(np.uint8)
    n = S.size
    t = oracle.O2Tree(S, sigma, K=64)
    o1 = oracle.O1(S, sigma)
    C = o1.C.astype(np.int64)
    cs, js = [], []
    for c in range(sigma):
        cnt = int(C[c + 1] - C[c])
        if cnt:
            for j in sorted(set(rng.integers(1, cnt + 1, 20).tolist()) | {1, cnt}):
                cs.append(c)
                js.append(j)
    cs = np.array(cs, np.uint32)
    js = np.array(js, np.uint64)
    sel = t.select(cs, js)
    assert np.array_equal(sel, o1.select(cs, js))
    assert np.array_equal(S[sel.astype(np.int64)], cs.astype(np.uint8))
    # with the exclusive rank of Section 4: rank_c(select_c(j)) = j - 1 and rank_c(select_c(j) + 1) = j
    assert np.array_equal(t.rank(cs, sel), js - 1)
    assert np.array_equal(t.rank(cs, sel + 1), js)
    # sum over c of rank_c(i) = i
    ii = rng.integers(0, n + 1, 200).astype(np.uint64)
    tot = np.zeros(ii.size, np.uint64)
    for c in range(sigma):
        tot += t.rank(np.full(ii.size, c, np.uint32), ii)
    assert np.array_equal(tot, ii)
    # access(i) = S[i]
    idx = rng.integers(0, n, 5000).astype(np.uint64)
    assert np.array_equal(t.access(idx), S[idx.astype(np.int64)].astype(np.uint32))
    # total tree bits = sum over symbols of hist * code length
    _, ln, _ = oracle.codes_split(sigma)
    hist = np.diff(C)
    assert sum(t.level_size(l) for l in range(t.L)) == int((hist * ln[:sigma].astype(np.int64)).sum())


@pytest.mark.parametrize("sigma", [3, 96, 1000])
def test_threaded_build_matches_pointer_tree(sigma):
    """The O2 build split over several threads (more threads than the default
    rule gives a small input) against the pointer-based tree, level by level,
    and its counters and samples against the pure-Python counting."""
    rng = np.random.default_rng(77 + sigma)
    S = rng.integers(0, sigma, 3001).astype(np.uint16)
    for threads in (1, 3, 7):
        t = oracle.O2Tree(S, sigma, K=16, threads=threads)
        levels = brute.pointer_tree_levels([int(x) for x in S], sigma)
        assert t.L == len(levels)
        for l, bits in enumerate(levels):
            assert [int(x) for x in t.bits(l)] == bits, (threads, l)
            L1, L2, s0, s1 = brute.counters(bits, 16)
            assert t.export(oracle.EXPORT_L1, l).tolist() == L1
            assert t.export(oracle.EXPORT_L2, l).tolist() == L2
            assert t.export(oracle.EXPORT_S0, l).tolist() == s0
            assert t.export(oracle.EXPORT_S1, l).tolist() == s1


def test_threaded_build_and_queries_do_not_depend_on_threads():
    """A level larger than 2^16 bits (so the sample export is threaded too):
    one thread and several give the same tree; threaded query loops equal the
    definitional oracle."""
    rng = np.random.default_rng(5)
    sigma, n = 1000, 300001
    S = rng.integers(0, sigma, n).astype(np.uint16)
    t1 = oracle.O2Tree(S, sigma, K=256, threads=1)
    t5 = oracle.O2Tree(S, sigma, K=256, threads=5)
    for l in range(t1.L):
        for what in (oracle.EXPORT_BITS, oracle.EXPORT_L1, oracle.EXPORT_L2, oracle.EXPORT_S0, oracle.EXPORT_S1):
            assert np.array_equal(t1.export(what, l), t5.export(what, l)), (l, what)
    # samples of a large level against positions of the b-bits (numpy's flatnonzero)
    bits = t5.bits(0)
    for b, what in ((0, oracle.EXPORT_S0), (1, oracle.EXPORT_S1)):
        pos = np.flatnonzero(bits == b)
        want = np.concatenate([[0], pos[np.arange(256, pos.size + 1, 256) - 1]])
        assert np.array_equal(t5.export(what, 0), want.astype(np.uint64))
    o1 = oracle.O1(S, sigma)
    i = rng.integers(0, n, 5000).astype(np.uint64)
    c = rng.integers(0, sigma, 5000).astype(np.uint32)
    assert np.array_equal(t5.query_mt(0, i, threads=4), o1.access(i))
    assert np.array_equal(t5.query_mt(1, i, c, threads=3), o1.rank(c, i))
    cnt = np.diff(o1.C).astype(np.int64)
    j = (rng.random(5000) * cnt[c]).astype(np.uint64) + 1
    assert np.array_equal(t5.query_mt(2, j, c, threads=6), o1.select(c, j))


def test_node_start_alg8_matches_recursion():
    for sigma in list(range(2, 300)) + [1000, 4097, 5000]:
        t = oracle.O2Tree(np.zeros(1, np.uint16), sigma)
        code, ln, L = oracle.codes_split(sigma)

        def pp2(x):
            p = 1
            while p * 2 < x:
                p *= 2
            return p

        for c in range(sigma):
            starts = []  # start symbol of the node holding c at each depth
            a, b = 0, sigma
            while b - a >= 2:
                starts.append(a)
                m = a + pp2(b - a)
                if c < m:
                    b = m
                else:
                    a = m
            assert len(starts) == ln[c]
            start_symbol = c
            for l in range(int(ln[c]) - 1, -1, -1):
                if (int(code[c]) >> (L - 1 - l)) & 1:
                    start_symbol = t.node_start(start_symbol, l)
                assert start_symbol == starts[l], (sigma, c, l)


# --------------------------------------------------------------------------
# closed-form space overheads (Sections 4.1, 6.2, 6.3)
# --------------------------------------------------------------------------

def test_space_overheads_from_paper():
    facts = _golden("paper_facts.json")
    n = 1 << 24
    S = (np.random.default_rng(3).integers(0, 2, n)).astype(np.uint8)
    t = oracle.O2Tree(S, 2, K=16384)
    l1 = t.export(oracle.EXPORT_L1, 0).size
    l2 = t.export(oracle.EXPORT_L2, 0).size
    rank_pct = 100.0 * (l1 * 64 + l2 * 16) / n
    assert round(rank_pct, 2) == facts["rank_overhead"]["percent"]
    for row in facts["rank_select_overhead"]:
        t = oracle.O2Tree(S, 2, K=row["sample"])
        samples = t.export(oracle.EXPORT_S0, 0).size + t.export(oracle.EXPORT_S1, 0).size
        pct = 100.0 * (l1 * 64 + l2 * 16 + samples * 64) / n
        assert round(pct, 1) == row["percent"]


# --------------------------------------------------------------------------
# learned-select network (FP64 reference) against central differences
# --------------------------------------------------------------------------

def test_mlp_backward_matches_finite_differences():
    from oracle import mlp

    rng = np.random.default_rng(11)
    for trial in range(4):
        P = rng.normal(size=mlp.NPARAM)
        u = rng.random(300)
        t = u + 0.1 * rng.normal(size=300)
        loss, g = mlp.loss_and_grad(P, u, t)
        fd = mlp.finite_difference_grad(P, u, t)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-7), trial
        # the loss is the mean squared error of u + g(u) against t, recomputed directly
        y, _, _ = mlp.forward(P, u)
        assert abs(loss - float(np.mean((u + y - t) ** 2))) < 1e-12


def test_pla_predictor_hits_its_knots():
    from oracle import mlp

    samples = np.array([0, 7000, 15000, 21000], np.uint64)
    K, total, size = 4096, 3 * 4096 + 100, 22000
    for m in range(4):
        kn = mlp.knots(samples, total, size, m, K)
        assert mlp.predict_pla(kn, kn[0]) == kn[2]
        if m < 3:
            assert mlp.predict_pla(kn, kn[1]) == kn[3]


def test_vectorised_predictors_equal_the_scalar_ones():
    """The array forms used for all-rank bound checks give the scalar forms' values."""
    from oracle import mlp

    rng = np.random.default_rng(5)
    K, total, size = 256, 256 * 7 + 40, 5000
    samples = np.concatenate([[0], np.sort(rng.choice(np.arange(1, size), 7, replace=False))]).astype(np.uint64)
    k, m, k0, k1, x0, x1 = mlp.segment_knots_all(samples, total, size, K)
    P = (0.3 * rng.normal(size=mlp.NPARAM)).astype(np.float32)
    pla = mlp.predict_pla_all(k, k0, k1, x0, x1)
    net = mlp.predict_mlp_f32_all(k, k0, k1, x0, x1, P)
    for idx in list(range(0, total, 37)) + [total - 1]:
        kn = mlp.knots(samples, total, size, int(m[idx]), K)
        assert (int(k0[idx]), int(k1[idx]), int(x0[idx]), int(x1[idx])) == kn
        assert int(pla[idx]) == mlp.predict_pla(kn, int(k[idx]))
        assert int(net[idx]) == mlp.predict_mlp_f32(kn, int(k[idx]), P)


def _round_f32_exact(x):
    """Round the rational x to float32 (round to nearest, ties to even), from
    the definition of the format: 24 significant bits, exponents down to -126,
    subnormals spaced 2^-149 apart."""
    from fractions import Fraction

    if x == 0:
        return 0.0
    sgn = -1 if x < 0 else 1
    ax = abs(Fraction(x))
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    while Fraction(2) ** e > ax:
        e -= 1
    while Fraction(2) ** (e + 1) <= ax:
        e += 1
    ulp = Fraction(2) ** (max(e, -126) - 23)
    q, r = divmod(ax, ulp)
    if r * 2 > ulp or (r * 2 == ulp and q % 2 == 1):
        q += 1
    return sgn * float(q * ulp)


def test_fma_f32_rounds_once():
    """fma_f32 against exact rational arithmetic: random operands, and
    constructed sums that sit just below or above a float32 rounding midpoint
    (where rounding in float64 first, then to float32, goes the wrong way)."""
    from fractions import Fraction

    from oracle import mlp

    rng = np.random.default_rng(21)
    a = rng.normal(size=3000).astype(np.float32)
    b = (rng.normal(size=3000) * 10.0 ** rng.integers(-8, 8, 3000)).astype(np.float32)
    c = (rng.normal(size=3000) * 10.0 ** rng.integers(-8, 8, 3000)).astype(np.float32)
    f = np.float32
    one_p = f(1 + 2 ** -23)
    below_mid = f(2 ** -24 * (1 - 2 ** -23))  # (1 + 2^-23) * this = 2^-24 - 2^-70
    a = np.concatenate([a, [one_p, one_p, -one_p, one_p]]).astype(np.float32)
    b = np.concatenate([b, [below_mid, below_mid, below_mid, f(2 ** -24)]]).astype(np.float32)
    c = np.concatenate([c, [one_p, f(1.0), -one_p, one_p]]).astype(np.float32)
    got = mlp.fma_f32(a, b, c)
    for i in range(a.size):
        exact = Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i]))
        assert float(got[i]) == _round_f32_exact(exact), (i, a[i], b[i], c[i])
    # the constructed case: exact value 1 + 2^-23 + 2^-24 - 2^-70 rounds down to
    # 1 + 2^-23, while float64 first gives the midpoint and then 1 + 2^-22
    assert float(got[3000]) == 1 + 2 ** -23
    naive = (a[3000].astype(np.float64) * b[3000].astype(np.float64) + c[3000].astype(np.float64)).astype(np.float32)
    assert float(naive) == 1 + 2 ** -22


def test_mlp_forward_of_a_one_unit_network():
    """g(u) = b2 + sum_j w2_j relu(w1_j u + b1_j) with the packing {w1, b1, w2, b2},
    by hand for one active unit: w1 = 2, b1 = -0.5, w2 = 3, b2 = 0.25."""
    from oracle import mlp

    P = np.zeros(mlp.NPARAM)
    P[0], P[mlp.H], P[2 * mlp.H], P[3 * mlp.H] = 2.0, -0.5, 3.0, 0.25
    y, _, _ = mlp.forward(P, np.array([0.1, 0.25, 0.5, 1.0]))
    assert np.allclose(y, [0.25, 0.25, 1.75, 4.75], rtol=0, atol=1e-15)


def test_mlp_predictor_hand_values_and_edges():
    """predict_mlp_f32 for w1 = 1, b1 = 0, w2 = 0.5, b2 = 0 (h = 1.5 u, all
    values exact in float32), the clamp of h to [0, 1] on both sides, and the
    cap of the offset at the span when float32(span) rounds up."""
    from oracle import mlp

    P = np.zeros(mlp.NPARAM, np.float32)
    P[0], P[2 * mlp.H] = 1.0, 0.5
    kn = (0, 8, 100, 164)
    assert mlp.predict_mlp_f32(kn, 0, P) == 100
    assert mlp.predict_mlp_f32(kn, 2, P) == 124  # u = 0.25, h = 0.375, 64 * 0.375 = 24
    assert mlp.predict_mlp_f32(kn, 4, P) == 148  # u = 0.5, h = 0.75
    assert mlp.predict_mlp_f32(kn, 6, P) == 164  # u = 0.75, h = 1.125 -> 1
    P2 = P.copy()
    P2[3 * mlp.H] = -0.5  # h = 1.5 u - 0.5 < 0 below u = 1/3
    assert mlp.predict_mlp_f32(kn, 2, P2) == 100
    assert mlp.predict_mlp_f32(kn, 4, P2) == 116  # h = 0.25
    span = (1 << 25) - 1  # float32(span) = 2^25 > span
    assert mlp.predict_mlp_f32((0, 8, 7, 7 + span), 7, P) == 7 + span
    # the array form agrees on the same points
    k = np.array([0, 2, 4, 6], np.int64)
    z = np.zeros(4, np.int64)
    got = mlp.predict_mlp_f32_all(k, z, z + 8, z + 100, z + 164, P)
    assert got.tolist() == [100, 124, 148, 164]


def test_mlp_predictor_within_fp32_bound_of_fp64_forward():
    """The FP32 chain against the FP64 network on random parameters: |h32 - h64|
    stays within the forward error bound of 2 (H + 2) ulps of the magnitudes
    involved, and the position within span * that bound + 2."""
    from oracle import mlp

    rng = np.random.default_rng(33)
    u_max = 0.0
    for trial in range(20):
        P = (rng.normal(size=mlp.NPARAM) * 0.5).astype(np.float32)
        k0, span_k = 4096 * trial, int(rng.integers(2, 9000))
        x0, span_x = int(rng.integers(0, 1 << 30)), int(rng.integers(1, 1 << 24))
        kn = (k0, k0 + span_k, x0, x0 + span_x)
        for k in rng.integers(k0, k0 + span_k, 40):
            k = int(k)
            u32 = np.float32(np.float32(k - k0) / np.float32(span_k))
            u = float(u32)
            h32 = float(mlp._mlp_h_f32(u32, P))
            y64, _, _ = mlp.forward(P.astype(np.float64), np.array([u]))
            h64 = u + float(y64[0])
            w1, b1, w2, b2 = mlp.unpack(P.astype(np.float64))
            mag = abs(u) + abs(b2) + float(np.sum(np.abs(w2) * (np.abs(w1) * abs(u) + np.abs(b1))))
            bound = 2.0 * (mlp.H + 2) * 2.0 ** -24 * mag
            assert abs(h32 - h64) <= bound, (trial, k, h32, h64, bound)
            pos = mlp.predict_mlp_f32(kn, k, P)
            ref = x0 + min(span_x, int(np.floor(span_x * min(max(h64, 0.0), 1.0))))
            assert abs(pos - ref) <= span_x * bound + 2 * span_x * 2.0 ** -24 + 2, (trial, k, pos, ref)
            u_max = max(u_max, u)
    assert u_max > 0.9


def test_spline_predictor_by_hand_and_brute_force():
    """The fitted-knot model's prediction: by hand on one segment, and the
    array form against the scalar form over every rank of a random level."""
    from oracle import mlp

    # segment (k0, k1, x0, x1) = (0, 16, 0, 160): untrained knots at (0, 0), (4, 40), ..., (16, 160)
    kn = (0, 16, 0, 160)
    R = [5, -10, 0]  # knots at positions 0, 45, 70, 120, 160
    kap, xi = mlp.spline_knots(kn, R)
    assert kap == [0, 4, 8, 12, 16] and xi == [0, 45, 70, 120, 160]
    assert mlp.predict_spline(kn, R, 2) == 22    # slope 45 / 4 = 11.25, 2 * 11.25 = 22.5 -> 22
    assert mlp.predict_spline(kn, R, 4) == 45
    assert mlp.predict_spline(kn, R, 6) == 57    # 45 + trunc(2 * 6.25)
    assert mlp.predict_spline(kn, R, 13) == 130
    assert mlp.predict_spline((0, 3, 10, 16), [99, 99, 99], 2) == 14  # short segment: the anchors only
    # exact integer interpolation: floor of the rational, no float rounding
    assert mlp.interp(0, 3, 0, 1, 2) == 0            # 2 / 3 -> 0
    assert mlp.interp(0, 3, 100, 103, 2) == 102
    assert mlp.interp(0, 4096, 0, 1 << 40, 4095) == (1 << 40) - (1 << 28)  # float32 would round this
    assert mlp.interp(7, 10, 50, 50, 9) == 50        # flat knots
    rng = np.random.default_rng(3)
    bits = (rng.random(20000) < 0.3).astype(np.uint8)
    pos = np.flatnonzero(bits)
    K = 64
    total, size = pos.size, bits.size
    samples = np.concatenate([[0], pos[np.arange(K, total + 1, K) - 1]])
    k, m, k0, k1, x0, x1 = mlp.segment_anchor_all(samples, total, size, K)
    nseg = total // (mlp.ANCHOR * K) + 1
    Rs = rng.integers(-3, 4, (nseg, 3))
    pred = mlp.predict_spline_all(k, k0, k1, x0, x1, Rs[m])
    for idx in list(range(0, total, 97)) + [total - 1]:
        kn = mlp.anchor_knots(samples, total, size, int(m[idx]), K)
        assert (int(k0[idx]), int(k1[idx]), int(x0[idx]), int(x1[idx])) == kn
        assert int(pred[idx]) == mlp.predict_spline(kn, Rs[m[idx]], int(k[idx]))


def test_spline_fit_is_the_least_squares_solution():
    """fit_spline_lsq (normal equations on hat functions) against
    numpy.linalg.lstsq on the explicit design matrix, and a noiseless
    piecewise-linear curve through the knots is recovered exactly."""
    from oracle import mlp

    rng = np.random.default_rng(8)
    kn = (1000, 1400, 50000, 58000)
    ks = np.arange(1001, 1400)
    pos = 50000 + (ks - 1000) * 20 + rng.normal(0, 40, ks.size).cumsum() * 0.1
    R = mlp.fit_spline_lsq(kn, ks, pos)
    kap = [1000 + t * 100 for t in range(5)]
    X = np.zeros((ks.size, 3))
    for t in (1, 2, 3):
        X[:, t - 1] = np.clip(np.minimum((ks - kap[t - 1]) / 100.0, (kap[t + 1] - ks) / 100.0), 0, None)
    base = 50000 + (ks - 1000) * 20.0
    ref = np.linalg.lstsq(X, pos - base, rcond=None)[0]
    assert np.allclose(R, ref, rtol=1e-9, atol=1e-6)
    true = np.array([30.0, -55.0, 12.0])
    knots_y = np.concatenate([[0.0], true, [0.0]])
    exact = base + np.interp(ks, kap, knots_y)
    assert np.allclose(mlp.fit_spline_lsq(kn, ks, exact), true, atol=1e-6)


def test_bitvector_rank_select_by_brute_force():
    """The oracle's binary rank/select against one-position-at-a-time loops, plus
    the invariants rank_1(select_1(j)) = j - 1, B[select_b(j)] = b and
    rank_1(i) + rank_0(i) = i."""
    from oracle import brute

    rng = np.random.default_rng(31)
    for n, p in ((1, 0.5), (7, 0.0), (9, 1.0), (64, 0.3), (513, 0.5), (1000, 0.9)):
        bits = (rng.random(n) < p).astype(np.uint8)
        i = np.arange(n + 1)
        want = np.array([brute.bv_rank(bits, k) for k in i], dtype=np.uint64)
        assert np.array_equal(oracle.bv_rank(bits, i), want)
        for b in (0, 1):
            cnt = int((bits == b).sum())
            j = np.arange(1, cnt + 1)
            sel = oracle.bv_select(bits, b, j)
            assert sel.tolist() == [brute.bv_select(bits, b, int(x)) for x in j]
            assert np.all(bits[sel.astype(np.int64)] == b)
            if b == 1 and cnt:
                assert np.array_equal(oracle.bv_rank(bits, sel.astype(np.int64)), (j - 1).astype(np.uint64))
        assert np.array_equal(oracle.bv_rank(bits, i) + oracle.bv_rank(1 - bits, i), i.astype(np.uint64))


def test_bitvector_support_by_brute_force():
    """oracle.bitvector_support against the pure-Python counting, over sizes
    around the 512- and 65536-bit blocks and all-zero / all-one vectors."""
    rng = np.random.default_rng(17)
    for n, fill, K in ((1, 0.5, 4), (511, 0.5, 8), (512, 1.0, 16), (513, 0.0, 16), (65536, 0.3, 256),
                       (65536 * 2 + 700, 0.7, 512), (200003, 0.02, 64)):
        bits = (rng.random(n) < fill).astype(np.uint8)
        L1, L2, s0, s1 = brute.counters(bits.tolist(), K)
        g = oracle.bitvector_support(bits, K)
        assert g[0].tolist() == L1 and g[1].tolist() == L2 and g[2].tolist() == s0 and g[3].tolist() == s1, n


def test_alphabet_map_by_brute_force():
    """The oracle's minimal-alphabet map against a set/sort over Python ints."""
    rng = np.random.default_rng(5)
    for n, hi in ((1, 10), (50, 7), (1000, 1 << 20), (300, 256)):
        S = rng.integers(0, hi, n)
        codes, values = oracle.alphabet_map(S)
        want_vals = sorted(set(int(x) for x in S))
        assert values.tolist() == want_vals
        rank = {v: k for k, v in enumerate(want_vals)}
        assert codes.tolist() == [rank[int(x)] for x in S]


def test_wavelet_matrix_oracle_by_brute_force():
    """The oracle's wavelet matrix levels against list-based stable partitions,
    its counters and samples against counting, and the matrix identity that
    level l+1 is level l's zeros followed by its ones."""
    rng = np.random.default_rng(12)
    for n, sigma, K in ((1, 2, 256), (37, 5, 256), (2000, 96, 256), (5000, 1000, 256), (70000, 3, 256)):
        S = rng.integers(0, sigma, n)
        om = oracle.OMatrix(S, sigma, K)
        bl = brute.matrix_levels(S, sigma)
        assert len(om.levels) == len(bl)
        for l, bits in enumerate(bl):
            assert om.levels[l].tolist() == bits
            L1, L2, s0, s1 = brute.counters(bits, K)
            assert om.export(1, l).tolist() == L1
            assert om.export(2, l).tolist() == L2
            assert om.export(3, l).tolist() == s0
            assert om.export(4, l).tolist() == s1
            words = om.export(0, l)
            assert np.unpackbits(words.view(np.uint8), bitorder="little")[:n].tolist() == bits
            assert om.zeros(l) == bits.count(0)


def test_bitvector_generator_layouts():
    """The bitvector inputs have the stated fills and layouts: uniform ones at the
    fill rate; adversarial ones 99 % within the last min(1, 0.99 fill / 0.95) of
    the positions.  (Sampling only; checked on the CPU with a small vector.)"""
    torch = pytest.importorskip("torch")
    from paper_2505_03372_gb300 import workloads

    n = 400_003
    for fill in workloads.BITVECTOR_FILLS:
        u = workloads.make_bitvector(n, fill, "uniform", seed=7, device="cpu")
        bits = np.unpackbits(u.numpy().view(np.uint8), bitorder="little")
        assert bits[n:].sum() == 0
        assert abs(bits[:n].mean() - fill) < 0.01
        a = workloads.make_bitvector(n, fill, "adversarial", seed=7, device="cpu")
        bits = np.unpackbits(a.numpy().view(np.uint8), bitorder="little")[:n]
        k = min(1.0, 0.99 * fill / 0.95)
        tail = bits[int(n * (1 - k)):]
        assert abs(bits.mean() - fill) < 0.01
        assert tail.sum() >= 0.985 * bits.sum()
