"""Seeded synthetic workloads (symbols and query batches).

This module is shared by the GPU tests, the benchmark and the oracle checks.
It holds random-number generation and sampling only -- none of the wavelet
tree's arithmetic.  To draw valid select queries (j in [1, count(c)]) it needs
per-symbol counts, which it takes from torch.bincount, a library routine.

The inputs stand in for the paper's uniform random texts and its real texts
(Section 6.1), which are not available here: uniform symbols over sigma, or a
Zipf law P(k) proportional to 1/(k+1)^s over [0, sigma) for text-like inputs.
Random draws are made with a torch.Generator seeded per workload (Philox on
CUDA), so a workload is reproducible on a given device type and torch version.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

SEED_BASE = 0x5EED0000


@dataclass
class Workload:
    name: str
    index: int
    n: int
    sigma: int
    symbol_bytes: int
    dist: str            # "uniform" or "zipf"
    zipf_s: float = 0.0
    queries: dict = field(default_factory=dict)  # kind -> count; "mixed" = thirds of access/rank/select
    sample_k: int = 4096

    @property
    def dtype(self):
        return {1: torch.uint8, 2: torch.int16, 4: torch.int32}[self.symbol_bytes]

    def describe(self) -> str:
        d = "uniform" if self.dist == "uniform" else f"Zipf(s={self.zipf_s})"
        q = ", ".join(f"{v} {k}" for k, v in self.queries.items())
        return f"n={self.n} u{8 * self.symbol_bytes} {d} over sigma={self.sigma}; queries: {q}"


# The five workload shapes: plain, text-like, large alphabet, batched, learned select.
WORKLOADS = {
    "plain": Workload("plain", 0, 1 << 20, 256, 1, "uniform", queries={"access": 100_000, "rank": 100_000, "select": 100_000}),
    "text": Workload("text", 1, 1 << 30, 96, 1, "zipf", 1.0, queries={"access": 10_000_000, "rank": 10_000_000, "select": 10_000_000}),
    "large_alphabet": Workload("large_alphabet", 2, 1 << 28, 1 << 20, 4, "uniform", queries={"mixed": 20_000_000}),
    "learned": Workload("learned", 4, 1 << 30, 65536, 2, "zipf", 1.2, queries={"select": 100_000_000}),
}


def generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def zipf_cdf(sigma: int, s: float, device) -> torch.Tensor:
    k = torch.arange(1, sigma + 1, dtype=torch.float64, device=device)
    p = k.pow(-s)
    c = torch.cumsum(p, 0)
    return c / c[-1]


def _from_cdf(cdf: torch.Tensor, count: int, g: torch.Generator, device) -> torch.Tensor:
    u = torch.rand(count, dtype=torch.float64, generator=g, device=device)
    idx = torch.searchsorted(cdf, u, right=True)
    return idx.clamp_(max=cdf.numel() - 1)


def make_symbols(n: int, sigma: int, symbol_bytes: int, dist: str = "uniform", zipf_s: float = 1.0,
                 seed: int = SEED_BASE, device="cuda", chunk: int = 1 << 26) -> torch.Tensor:
    """n symbols in [0, sigma) stored in 1, 2 or 4 bytes (u16/u32 as int16/int32 bit patterns)."""
    dtype = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[symbol_bytes]
    out = torch.empty(n, dtype=dtype, device=device)
    g = generator(seed, device)
    cdf = zipf_cdf(sigma, zipf_s, device) if dist == "zipf" else None
    for a in range(0, n, chunk):
        m = min(chunk, n - a)
        if cdf is None:
            v = torch.randint(0, sigma, (m,), generator=g, device=device, dtype=torch.int64)
        else:
            v = _from_cdf(cdf, m, g, device)
        if symbol_bytes == 2:
            v = torch.where(v >= 32768, v - 65536, v)
        out[a:a + m] = v.to(dtype)
    return out


def symbols_as_int64(sym: torch.Tensor) -> torch.Tensor:
    """Unsigned symbol values of a symbol tensor (u16/u32 stored as int16/int32)."""
    if sym.dtype == torch.int16:
        return sym.to(torch.int64) & 0xFFFF
    if sym.dtype == torch.int32:
        return sym.to(torch.int64) & 0xFFFFFFFF
    return sym.to(torch.int64)


def symbol_counts(sym: torch.Tensor, sigma: int, chunk: int = 1 << 26) -> torch.Tensor:
    cnt = torch.zeros(sigma, dtype=torch.int64, device=sym.device)
    for a in range(0, sym.numel(), chunk):
        cnt += torch.bincount(symbols_as_int64(sym[a:a + chunk]), minlength=sigma)[:sigma]
    return cnt


def make_queries(w: Workload, sym: torch.Tensor, seed: int = None, counts: torch.Tensor = None,
                 scale: float = 1.0) -> dict:
    """Query batches of a workload; ``scale`` shrinks the counts (for quick runs).

    access: i uniform in [0, n).  rank: c uniform (or from the Zipf law), i
    uniform in [0, n).  select: c drawn like rank's c but only among symbols
    that occur, j uniform in [1, count(c)].  mixed: each query independently
    access, rank or select with probability 1/3.
    """
    device = sym.device
    n, sigma = sym.numel(), w.sigma
    g = generator(SEED_BASE + 0x100 + w.index if seed is None else seed, device)
    if counts is None:
        counts = symbol_counts(sym, sigma)
    base = zipf_cdf(sigma, w.zipf_s, device) if w.dist == "zipf" else None

    def draw_c(q):
        if base is None:
            return torch.randint(0, sigma, (q,), generator=g, device=device, dtype=torch.int64)
        return _from_cdf(base, q, g, device)

    present = (counts > 0).to(torch.float64)
    if base is None:
        wsel = present
    else:
        pdf = torch.diff(base, prepend=torch.zeros(1, dtype=torch.float64, device=device))
        wsel = pdf * present
    csel = torch.cumsum(wsel, 0)
    csel = csel / csel[-1] if csel[-1] > 0 else csel

    def draw_select(q):
        c = _from_cdf(csel, q, g, device)
        u = torch.rand(q, dtype=torch.float64, generator=g, device=device)
        j = (u * counts[c].to(torch.float64)).to(torch.int64) + 1
        j = torch.minimum(j, counts[c]).clamp_(min=1)
        return c, j

    out = {}
    for kind, q in w.queries.items():
        q = max(1, int(q * scale))
        if kind == "access":
            out["access_i"] = torch.randint(0, max(n, 1), (q,), generator=g, device=device, dtype=torch.int64)
        elif kind == "rank":
            out["rank_c"] = draw_c(q).to(torch.int32)
            out["rank_i"] = torch.randint(0, max(n, 1), (q,), generator=g, device=device, dtype=torch.int64)
        elif kind == "select":
            c, j = draw_select(q)
            out["select_c"] = c.to(torch.int32)
            out["select_j"] = j
        elif kind == "mixed":
            k = torch.randint(0, 3, (q,), generator=g, device=device, dtype=torch.int64)
            c_r = draw_c(q)
            c_s, j_s = draw_select(q)
            i_a = torch.randint(0, max(n, 1), (q,), generator=g, device=device, dtype=torch.int64)
            c = torch.where(k == 1, c_r, torch.where(k == 2, c_s, torch.zeros_like(c_r)))
            arg = torch.where(k == 2, j_s, i_a)
            out["mixed_kind"] = k.to(torch.uint8)
            out["mixed_c"] = c.to(torch.int32)
            out["mixed_arg"] = arg
    return out


def make_workload(name: str, device="cuda", n: int = None, scale_queries: float = 1.0):
    """Symbols and queries of a named workload (optionally with a smaller n)."""
    w = WORKLOADS[name]
    if n is not None and n != w.n:
        w = Workload(w.name, w.index, n, w.sigma, w.symbol_bytes, w.dist, w.zipf_s, dict(w.queries), w.sample_k)
    sym = make_symbols(w.n, w.sigma, w.symbol_bytes, w.dist, w.zipf_s, SEED_BASE + w.index, device)
    counts = symbol_counts(sym, w.sigma)
    q = make_queries(w, sym, counts=counts, scale=scale_queries)
    return w, sym, q, counts


# --------------------------------------------------------------------------
# batched workload: thousands of independent trees
# --------------------------------------------------------------------------

BATCH_SIGMAS = (4, 256, 65536)


def make_batch(ntrees: int = 4096, seed: int = SEED_BASE + 3, device="cuda", log_n=(10, 24), log_q=(4, 16),
               sigmas=BATCH_SIGMAS, symbol_bytes: int = 2):
    """Symbols and mixed queries of a batch of independent trees.

    Tree i has n_i = floor(2^U(log_n)) symbols drawn uniformly from [0, sigma_i),
    sigma_i drawn uniformly from `sigmas`, and floor(2^U(log_q)) queries, each
    access, rank or select with probability 1/3 (arguments as in make_queries;
    select's symbol is drawn uniformly among the symbols that occur in the tree).
    All symbols live in one buffer; each tree starts on a 16-byte boundary.
    Returns (buffer, per-tree views, sigmas, queries dict with tree/kind/c/arg).
    """
    g = generator(seed, device)
    gh = torch.Generator()
    gh.manual_seed(seed)
    u = torch.rand(ntrees, generator=gh, dtype=torch.float64)
    ns = torch.floor(2.0 ** (log_n[0] + u * (log_n[1] - log_n[0]))).to(torch.int64).tolist()
    sg = [sigmas[i] for i in torch.randint(0, len(sigmas), (ntrees,), generator=gh).tolist()]
    uq = torch.rand(ntrees, generator=gh, dtype=torch.float64)
    qs = torch.floor(2.0 ** (log_q[0] + uq * (log_q[1] - log_q[0]))).to(torch.int64).tolist()
    align = 16 // symbol_bytes
    offs, tot = [], 0
    for n in ns:
        offs.append(tot)
        tot += (n + align - 1) // align * align
    dtype = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[symbol_bytes]
    buf = torch.zeros(max(tot, 1), dtype=dtype, device=device)
    views = []
    qt, qk, qc, qa = [], [], [], []
    for i, (n, s, q, o) in enumerate(zip(ns, sg, qs, offs)):
        v = torch.randint(0, s, (n,), generator=g, device=device, dtype=torch.int64)
        cnt = torch.bincount(v, minlength=s)
        if symbol_bytes == 2:
            v = torch.where(v >= 32768, v - 65536, v)
        buf[o:o + n] = v.to(dtype)
        views.append(buf[o:o + n])
        kind = torch.randint(0, 3, (q,), generator=g, device=device, dtype=torch.int64)
        pos = torch.randint(0, max(n, 1), (q,), generator=g, device=device, dtype=torch.int64)
        c_r = torch.randint(0, s, (q,), generator=g, device=device, dtype=torch.int64)
        present = torch.nonzero(cnt).flatten()
        c_s = present[torch.randint(0, max(present.numel(), 1), (q,), generator=g, device=device)] if present.numel() \
            else torch.zeros(q, dtype=torch.int64, device=device)
        cs_cnt = cnt[c_s] if present.numel() else torch.ones(q, dtype=torch.int64, device=device)
        j = (torch.rand(q, generator=g, device=device, dtype=torch.float64) * cs_cnt).to(torch.int64) + 1
        j = torch.minimum(j, cs_cnt)
        qt.append(torch.full((q,), i, dtype=torch.int32, device=device))
        qk.append(kind.to(torch.uint8))
        qc.append(torch.where(kind == 1, c_r, torch.where(kind == 2, c_s, torch.zeros_like(c_r))).to(torch.int32))
        qa.append(torch.where(kind == 2, j, pos))
    queries = {"tree": torch.cat(qt), "kind": torch.cat(qk), "c": torch.cat(qc), "arg": torch.cat(qa)}
    return buf, views, sg, queries


def batch_subset(views, sigmas, q, lo: int, hi: int):
    """Trees [lo, hi) of a batch with their queries (tree ids renumbered from
    0), the symbols copied into a buffer of their own with every tree on a
    16-byte boundary.  Returns (buffer, views, sigmas, queries) like make_batch."""
    sel = list(views[lo:hi])
    w = sel[0].element_size() if sel else 2
    align = 16 // w
    offs, tot = [], 0
    for v in sel:
        offs.append(tot)
        tot += (v.numel() + align - 1) // align * align
    device = q["tree"].device
    dtype = sel[0].dtype if sel else torch.int16
    buf = torch.zeros(max(tot, 1), dtype=dtype, device=device)
    out_views = []
    for v, o in zip(sel, offs):
        buf[o:o + v.numel()] = v
        out_views.append(buf[o:o + v.numel()])
    m = (q["tree"] >= lo) & (q["tree"] < hi)
    sub = {"tree": (q["tree"][m] - lo).to(torch.int32), "kind": q["kind"][m], "c": q["c"][m], "arg": q["arg"][m]}
    return buf, out_views, list(sigmas[lo:hi]), sub


# --------------------------------------------------------------------------
# standalone bitvectors (the paper's binary rank/select experiments, whose
# bitvectors follow Kurpicz's generator: a fill of 10, 50 or 90 %, ones either
# uniform or concentrated at the end)
# --------------------------------------------------------------------------

BITVECTOR_FILLS = (0.1, 0.5, 0.9)


def make_bitvector(nbits: int, fill: float, layout: str = "uniform", seed: int = SEED_BASE + 5,
                   device="cuda", chunk: int = 1 << 28) -> torch.Tensor:
    """int64 words (LSB-first) of an nbits-bit vector.  "uniform": every bit is 1
    with probability `fill`.  "adversarial": 99 % of the ones fall in the last
    k·nbits positions, k = min(1, 0.99·fill / 0.95) (95 % ones there); the
    remaining 1 % of the ones are spread uniformly over the rest.  Bits are drawn
    chunk by chunk (a byte per bit) and packed 8 at a time."""
    g = generator(seed, device)
    nw = (nbits + 63) // 64
    out = torch.zeros(nw * 8, dtype=torch.uint8, device=device)
    weights = torch.tensor([1, 2, 4, 8, 16, 32, 64, 128], dtype=torch.int16, device=device)
    tail0 = nbits
    p_head = p_tail = fill
    if layout == "adversarial":
        k = min(1.0, 0.99 * fill / 0.95)
        tail0 = int(nbits * (1.0 - k))
        p_tail = min(1.0, 0.99 * fill / k) if k > 0 else 0.0
        p_head = (0.01 * fill * nbits) / max(tail0, 1)
    elif layout != "uniform":
        raise ValueError(layout)
    for s in range(0, nbits, chunk):
        e = min(nbits, s + chunk)
        pos = torch.arange(s, e, device=device)
        thr = torch.where(pos < tail0, torch.full_like(pos, int(p_head * 65536)), torch.full_like(pos, int(p_tail * 65536)))
        r = torch.randint(0, 65536, (e - s,), generator=g, device=device, dtype=torch.int64)
        bits = (r < thr).to(torch.int16)
        pad = (-bits.numel()) % 8
        if pad:
            bits = torch.cat([bits, torch.zeros(pad, dtype=torch.int16, device=device)])
        packed = (bits.view(-1, 8) * weights).sum(1).to(torch.uint8)
        out[s // 8: s // 8 + packed.numel()] = packed
    return out.view(torch.int64)
