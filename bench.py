#!/usr/bin/env python
"""Benchmark: wavelet-tree build + batched access/rank/select on one GB300.

A step is one pass of the whole hot path over one synthetic input: build the
tree of the text workload (n = 2^30 uint8 symbols, Zipf(s=1.0) over sigma = 96,
7 levels with reduced codes), then 10M access, 10M rank and 10M select
queries, then free the tree.  ``value`` is queries per second over whole steps
(build time included), in Mqueries/s; the per-phase rates (build GB/s,
access/rank/select Mq/s) are reported under "phases".

  python bench.py [--steps K] [--warmup W] [--workload text|plain|large_alphabet|learned]
  python bench.py --impl reference      # the CPU oracle on a bounded sample

Under torchrun (N > 1) every rank builds the same tree (the build does not
shard: replicas) and answers its own query batch (queries shard with no
collective), so the scaling is weak in queries.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "access/rank/select Mqueries/s, build GB/s; learned vs sampled select"
UNIT = "Mqueries/s"
PEAK_FALLBACK_GBS = 6800.0


# --------------------------------------------------------------------------
# multi-rank bookkeeping (torchrun, one process per GPU): every rank builds the
# same tree from the same seed and answers its own query batch; the step time
# is the slowest rank's, the value counts every rank's queries
# --------------------------------------------------------------------------

def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's own query batch (rank 0 keeps the single-GPU seed)."""
    return base + 7919 * rank


def job_ms(ms: float, dist) -> float:
    """The step time of the job: the maximum over ranks (all ranks return it)."""
    if dist is None:
        return ms
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(world: int, q_per_rank: int, ms: float) -> float:
    """Whole-job throughput in Mqueries/s: every rank's queries over the job's step time."""
    return world * q_per_rank / (ms * 1e-3) / 1e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="text")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-sampled select comparison")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' records")
    ap.add_argument("--n", type=int, default=None, help="override the workload's n (small profiling cases)")
    ap.add_argument("--query-scale", type=float, default=1.0, help="scale the query counts (small profiling cases)")
    ap.add_argument("--overlap", action="store_true",
                    help="sort the query batches on a second stream while the level passes run (measured: no "
                         "gain on one GB300, the level pass already fills the SMs)")
    ap.add_argument("--layout", default="tree", choices=["tree", "matrix"],
                    help="level-wise wavelet tree (the paper's) or the wavelet matrix variant")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if shutil.which("nvidia-smi"):
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# algorithmic traffic models
# --------------------------------------------------------------------------

def level_pass_bytes(sizes, w, K):
    """Bytes one level pass must move: read T_l, write bits, counters and
    samples, write T_{l+1} (none at the last level)."""
    out = []
    L = len(sizes)
    for l, sz in enumerate(sizes):
        b = sz * w + (sz + 7) // 8 + (sz // 65536 + 1) * 8 + (sz // 512 + 1) * 2 + (sz // K + 2) * 8
        if l + 1 < L:
            b += sizes[l + 1] * w
        out.append(b)
    return out


def build_bytes(n, w, sizes, K):
    """Algorithmic bytes of the level-wise build: histogram read + every level pass."""
    return n * w + sum(level_pass_bytes(sizes, w, K))


def query_sectors(kind, L, mean_len):
    """32-byte DRAM sectors per query (counters, node tables and C cache-resident):
    per level one L2-counter sector and on average 1.5 word sectors for a rank;
    access reads a single bit at its last level; a sampled select reads about
    one sample, four L2-search and 1.5 word sectors per level."""
    if kind == "rank":
        return 2.5 * mean_len
    if kind == "access":
        return 2.5 * (L - 1) + 1
    return 6.5 * mean_len


# --------------------------------------------------------------------------
# the CPU oracle as baseline (threaded over the host cores, bounded sample,
# median of several runs, scaled to the metric's unit)
# --------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample_rate(wl, n_sample=1 << 24, q_sample=200_000, runs=3, seed_off=0):
    """The oracle on the host cores: the naive level-wise build (O2, its
    counting sorts split over threads) on n_sample symbols of the workload's
    distribution, then q_sample each of access / rank / select tree walks
    split over threads; median of `runs` repetitions, build time scaled by
    n / n_sample and query time by the workload's query count."""
    import numpy as np
    import oracle
    from paper_2505_03372_gb300 import workloads

    sym = workloads.make_symbols(n_sample, wl.sigma, wl.symbol_bytes, wl.dist, wl.zipf_s,
                                 seed=workloads.SEED_BASE + wl.index + seed_off, device="cpu")
    S = sym.numpy().view({1: np.uint8, 2: np.uint16, 4: np.uint32}[wl.symbol_bytes])
    w2 = workloads.Workload(wl.name, wl.index, n_sample, wl.sigma, wl.symbol_bytes, wl.dist, wl.zipf_s,
                            {"access": q_sample, "rank": q_sample, "select": q_sample}, wl.sample_k)
    q = workloads.make_queries(w2, sym)
    ai = q["access_i"].numpy().view(np.uint64)
    rc, ri = q["rank_c"].numpy().view(np.uint32), q["rank_i"].numpy().view(np.uint64)
    sc, sj = q["select_c"].numpy().view(np.uint32), q["select_j"].numpy().view(np.uint64)
    tb, tq = [], []
    for _ in range(runs):
        t0 = time.perf_counter()
        tree = oracle.O2Tree(S, wl.sigma, K=wl.sample_k)
        t1 = time.perf_counter()
        tree.query_mt(0, ai)
        tree.query_mt(1, ri, rc)
        tree.query_mt(2, sj, sc)
        t2 = time.perf_counter()
        del tree
        tb.append(t1 - t0)
        tq.append(t2 - t1)
    b, qt = statistics.median(tb), statistics.median(tq)
    Q = sum(wl.queries.values())
    t_full = b * (wl.n / n_sample) + qt * (Q / (3 * q_sample))
    return {"value": Q / t_full / 1e6, "unit": UNIT, "cores": oracle.default_threads(), "cpu_model": cpu_model(),
            "kind": "oracle", "runs": runs,
            "sample": (f"naive level-wise tree (Algorithms 3-8, counting sorts split over the host threads) built on "
                       f"{n_sample} symbols of the same distribution plus {q_sample} each of access/rank/select tree "
                       f"walks split over the host threads; median of {runs} runs; build time scaled by n/{n_sample}, "
                       f"query time by {Q}/{3 * q_sample}"),
            "build_s_sample": b, "query_s_sample": qt}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2505_03372_gb300 import workloads

    oracle.build()
    wl = workloads.WORKLOADS[args.workload if args.workload in workloads.WORKLOADS else "text"]
    vals, info = [], None
    for s in range(args.warmup + args.steps):
        info = oracle_sample_rate(wl, n_sample=1 << 23, q_sample=100_000, runs=1, seed_off=s)
        if s >= args.warmup:
            vals.append(info["value"])
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8" if wl.symbol_bytes == 1 else f"u{8 * wl.symbol_bytes}",
        "data": "synthetic", "config": {"workload": wl.describe(), "sample_k": wl.sample_k},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": info["cores"], "cpu_model": info["cpu_model"],
                         "kind": "oracle", "sample": info["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

OUT_KEYS = {"access_i": "access", "rank_i": "rank", "select_j": "select", "mixed_arg": "mixed"}


def prepare(wl, rank):
    """Symbols, counts, queries and output buffers of a workload on the current GPU."""
    import torch
    from paper_2505_03372_gb300 import workloads

    sym = workloads.make_symbols(wl.n, wl.sigma, wl.symbol_bytes, wl.dist, wl.zipf_s,
                                 seed=workloads.SEED_BASE + wl.index, device="cuda")
    counts = workloads.symbol_counts(sym, wl.sigma)
    q = workloads.make_queries(wl, sym, seed=rank_seed(workloads.SEED_BASE + 0x100 + wl.index, rank), counts=counts)
    outs = {}
    for k, v in q.items():
        if k in OUT_KEYS:
            outs[OUT_KEYS[k]] = torch.empty(v.numel(), dtype=torch.int32 if k == "access_i" else torch.int64,
                                            device="cuda")
    Q = sum(v.numel() for k, v in q.items() if k in OUT_KEYS)
    return sym, counts, q, outs, Q


def make_step(wt, wl, layout, overlap=False):
    """One step: build, then every query batch.  With `overlap`, the batches are
    sorted by walk key (wt_order_queries) on a second stream while the build's
    level passes run, and walked (wt_walk_ordered) on the build's stream after
    it.  wt_build returns only after the histogram and C are done (it reads
    the level sizes back), so all of the previous step's work has finished by
    then and the orders never overlap another step."""
    side = None
    if overlap:
        import torch

        side = torch.cuda.Stream(priority=-1)  # the orders' CTAs go ahead of waiting level-pass CTAs

    def step_overlap(sym_dev, qd, od):
        import torch

        t = wt.build(sym_dev, wl.sigma, sample_k=wl.sample_k, layout=layout)
        main = torch.cuda.current_stream()
        jobs = []
        with torch.cuda.stream(side):
            if "access_i" in qd:
                jobs.append((t.order(wt.ORDER_ACCESS, qd["access_i"], stream=side), od["access"]))
            if "rank_i" in qd:
                jobs.append((t.order(wt.ORDER_RANK, qd["rank_i"], c=qd["rank_c"], stream=side), od["rank"]))
            if "select_j" in qd:
                jobs.append((t.order(wt.ORDER_SELECT, qd["select_j"], c=qd["select_c"], stream=side), od["select"]))
            if "mixed_arg" in qd:
                jobs.append((t.order(wt.ORDER_MIXED, qd["mixed_arg"], c=qd["mixed_c"], kinds=qd["mixed_kind"],
                                     stream=side), od["mixed"]))
        for o, out in jobs:
            t.walk(o, out=out, stream=main)
        for o, _ in jobs:
            o.close(stream=main)
        return t

    def step(sym_dev, qd, od):
        t = wt.build(sym_dev, wl.sigma, sample_k=wl.sample_k, layout=layout)
        if "access_i" in qd:
            t.access(qd["access_i"], out=od["access"])
        if "rank_i" in qd:
            t.rank(qd["rank_c"], qd["rank_i"], out=od["rank"])
        if "select_j" in qd:
            t.select(qd["select_c"], qd["select_j"], out=od["select"])
        if "mixed_arg" in qd:
            t.query_mixed(qd["mixed_kind"], qd["mixed_c"], qd["mixed_arg"], out=od["mixed"])
        return t
    return step_overlap if overlap else step


def measure(wt, wl, sym, q, outs, steps, warmup, layout, barrier=lambda: None, clocks_gpu=None, overlap=False):
    """Warm-up steps, then `steps` timed steps (build + every query batch) with
    CUDA events on the launching stream; per-kernel times from libwt's
    launch events.  Returns the step time, launches, kernel report and the
    level sizes."""
    import torch

    step = make_step(wt, wl, layout, overlap)
    inf = None
    for _ in range(max(warmup, 3)):
        t = step(sym, q, outs)
        st = t.status_sync()
        if st != wt.WT_OK:
            raise RuntimeError("device status after warm-up: " + wt.status_str(st))
        inf = t.info()
        lens = t.export(wt.EXPORT_LENS) if inf.levels and layout == wt.LAYOUT_TREE else None
        t.close()
    sizes = [inf.level_size[l] for l in range(inf.levels)]
    wt.profile_reset()
    wt.profile_enable(True)
    clocks = ClockSampler(clocks_gpu) if clocks_gpu is not None else None
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        t = step(sym, q, outs)
        t.close()
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    rep = wt.profile_report()
    launches = wt.profile_launches()
    wt.profile_enable(False)
    return {"ms": ev0.elapsed_time(ev1) / steps, "launches": launches, "kern": rep, "sizes": sizes, "clk": clk,
            "lens": lens}


def analyse(wl, q, m, steps):
    """Phases, the level pass against the copy bandwidth and the queries against
    measured DRAM bytes per query."""
    import numpy as np

    peak, peak_kind = peaks()
    w, sizes, kern = wl.symbol_bytes, m["sizes"], {k: dict(v) for k, v in m["kern"].items()}
    lp_bytes = level_pass_bytes(sizes, w, wl.sample_k)
    b_build = build_bytes(wl.n, w, sizes, wl.sample_k)
    qkern = ("access", "rank", "select", "mixed", "order_hist", "order_scan", "order_scatter")
    build_ms = sum(v["ms"] for k, v in kern.items() if k not in qkern) / steps
    phases = {"build_ms": build_ms, "build_GBps": b_build / (build_ms * 1e-3) / 1e9,
              "build_input_GBps": wl.n * w / (build_ms * 1e-3) / 1e9,
              "query_order_ms": sum(v["ms"] for k, v in kern.items() if k.startswith("order_")) / steps}
    qk_of = {"access": "access_i", "rank": "rank_i", "select": "select_j", "mixed": "mixed_arg"}
    for kind, qk in qk_of.items():
        if kind in kern and kern[kind]["launches"]:
            ms = kern[kind]["ms"] / kern[kind]["launches"]
            phases[f"{kind}_ms"] = ms
            phases[f"{kind}_Mqps"] = q[qk].numel() / (ms * 1e-3) / 1e6
    lp_name = {1: "level_pass_u8", 2: "level_pass_u16", 4: "level_pass_u32"}[w]
    tot = max(sum(v["ms"] for v in kern.values()), 1e-9)
    for k in kern:
        kern[k]["share"] = kern[k]["ms"] / tot
    cands = [(kern[k]["ms"], k) for k in [lp_name, "access", "rank", "select", "mixed"] if k in kern]
    dom_ms, dom = max(cands)
    nlaunch = kern[dom]["launches"]
    lens = m.get("lens")
    code_len = 0.0
    cs = [q[k].cpu().numpy().view(np.uint32) for k in ("rank_c", "select_c", "mixed_c") if k in q]
    if lens is not None and cs:
        code_len = float(lens[np.concatenate(cs)].astype(np.float64).mean())
    L = len(sizes)
    qroof = {}
    for kind, qk in qk_of.items():
        if kind in kern and kern[kind]["launches"]:
            ms = kern[kind]["ms"] / kern[kind]["launches"]
            nq = q[qk].numel()
            rec = _query_traffic(kind)
            r = {"model_sectors_per_query": (query_sectors(kind, L, code_len) if kind != "mixed" else statistics.mean(
                [query_sectors(k, L, code_len) for k in ("access", "rank", "select")]))}
            r["model_frac"] = nq * r["model_sectors_per_query"] * 32 / (ms * 1e-3) / 1e9 / peak
            if rec is not None:
                r["dram_bytes_per_query"] = rec
                r["achieved_GBps"] = nq * rec / (ms * 1e-3) / 1e9
                r["frac"] = r["achieved_GBps"] / peak
            else:
                r["frac"] = None
            qroof[kind] = r
    if dom == lp_name:
        per_launch = sum(lp_bytes) / len(lp_bytes)
        achieved = sum(lp_bytes) * steps / (dom_ms * 1e-3) / 1e9
        traffic = _measured_traffic(dom, sum(sizes) / max(len(sizes), 1))
    else:
        qk = qk_of[dom]
        rec = _query_traffic(dom)
        per_launch = q[qk].numel() * (rec if rec is not None else 0.0)
        achieved = per_launch * nlaunch / (dom_ms * 1e-3) / 1e9
        traffic = per_launch if rec is not None else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": per_launch, "avg_launch_ms": dom_ms / nlaunch,
            "traffic": traffic, "queries": qroof}
    if lp_name in kern:
        roof["level_pass_frac"] = (sum(lp_bytes) * steps / (kern[lp_name]["ms"] * 1e-3) / 1e9) / peak
    return phases, roof, kern


def definitional_check(wl, sym, q, outs, nsample=64, seed=1):
    """Sampled answers of the last timed step against the definitions of
    Section 1, evaluated with torch on the input symbols on the GPU: access(i)
    = S[i]; rank_c(i) = #{j < i : S[j] = c}; select_c(j) = p with S[p] = c and
    #{q < p : S[q] = c} = j - 1.  Independent of libwt's code."""
    import torch
    from paper_2505_03372_gb300 import workloads

    S = workloads.symbols_as_int64(sym) if sym.dtype != torch.uint8 else sym.to(torch.int64)
    g = torch.Generator()
    g.manual_seed(seed)
    bad = checked = 0

    def pick(n):
        return torch.randint(0, n, (min(nsample, n),), generator=g).tolist()

    def rank_def(c, i):
        return int((S[:i] == c).sum().item())

    if "access_i" in q:
        ks = pick(q["access_i"].numel())
        ii = q["access_i"][ks].cpu().tolist()
        got = outs["access"][ks].cpu().to(torch.int64).tolist()
        for i, gv in zip(ii, got):
            checked += 1
            bad += int(S[i].item() != (gv & 0xFFFFFFFF))
    if "rank_i" in q:
        for k in pick(q["rank_i"].numel()):
            c, i, gv = int(q["rank_c"][k]) & 0xFFFFFFFF, int(q["rank_i"][k]), int(outs["rank"][k])
            checked += 1
            bad += int(rank_def(c, i) != gv)
    if "select_j" in q:
        for k in pick(q["select_j"].numel()):
            c, j, p = int(q["select_c"][k]) & 0xFFFFFFFF, int(q["select_j"][k]), int(outs["select"][k])
            checked += 1
            bad += int(not (0 <= p < S.numel() and int(S[p]) == c and rank_def(c, p) == j - 1))
    if "mixed_arg" in q:
        for k in pick(q["mixed_arg"].numel()):
            kd, c, x, gv = int(q["mixed_kind"][k]), int(q["mixed_c"][k]) & 0xFFFFFFFF, int(q["mixed_arg"][k]), \
                int(outs["mixed"][k])
            checked += 1
            if kd == 0:
                bad += int(int(S[x]) != gv)
            elif kd == 1:
                bad += int(rank_def(c, x) != gv)
            else:
                bad += int(not (0 <= gv < S.numel() and int(S[gv]) == c and rank_def(c, gv) == x - 1))
    return {"checked": checked, "ok": bad == 0, "mismatches": bad,
            "how": "sampled answers of the timed run against the definitions (access = S[i]; rank = count of c in "
                   "S[0, i); select: S[p] = c and count of c in S[0, p) = j - 1) evaluated with torch on the input"}


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_03372_gb300 import binding as wt
    from paper_2505_03372_gb300 import workloads

    wl = workloads.WORKLOADS[args.workload]
    if args.n is not None or args.query_scale != 1.0:
        qs = {k: max(1, int(v * args.query_scale)) for k, v in wl.queries.items()}
        wl = workloads.Workload(wl.name, wl.index, args.n or wl.n, wl.sigma, wl.symbol_bytes, wl.dist, wl.zipf_s, qs,
                                wl.sample_k)
    layout = wt.LAYOUT_MATRIX if args.layout == "matrix" else wt.LAYOUT_TREE

    def barrier():
        if dist is not None:
            dist.barrier()

    sym, counts, q, outs, Q = prepare(wl, rank)
    m = measure(wt, wl, sym, q, outs, args.steps, args.warmup, layout, barrier, local if rank == 0 else None,
                overlap=args.overlap)
    ms_step = job_ms(m["ms"], dist)
    value = job_value(world, Q, ms_step)
    phases, roof, kern = analyse(wl, q, m, args.steps)
    w = wl.symbol_bytes
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8" if w == 1 else f"u{8 * w}", "data": "synthetic", "impl": "ours",
        "config": {"workload": wl.describe() + ("; wavelet matrix layout" if args.layout == "matrix" else ""),
                   "queries_per_step_per_gpu": Q, "sample_k": wl.sample_k,
                   "l2_flush": "inputs larger than L2 (1 GiB symbols, ~0.9 GiB tree, 0.5 GiB queries)",
                   "parallelism": "replicated build, sharded queries" if world > 1 else "1 GPU",
                   "query_order": "second stream, overlapping the level passes (wt_order_queries)" if args.overlap
                   else "build's stream, after the build"},
        "phases": phases, "roofline": roof, "kernels": kern, "gpu_launches": m["launches"], "clocks": m["clk"],
        "parity": definitional_check(wl, sym, q, outs),
    }

    # ---- end to end: host buffers, copies inside the timed region ----
    if not args.no_e2e:
        line["e2e"] = _e2e(args, wl, sym, q, outs, make_step(wt, wl, layout), barrier, dist, world, Q)
    # ---- learned vs sampled select on this workload's select queries ----
    if ("select_j" in q or "mixed_arg" in q) and not args.no_learned:
        line["learned_select"] = learned_compare(wt, wl, sym, q)
    del sym, q, outs
    # ---- the other workloads, each timed the same way (rank 0, N = 1) ----
    if world == 1 and not args.no_configs and args.workload == "text" and args.n is None:
        line["configs"] = config_records(args, wt, workloads)
    # ---- CPU oracle baseline (rank 0, N = 1) ----
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        cb = oracle_sample_rate(wl)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "cpu_model", "kind", "sample", "runs")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def config_records(args, wt, workloads):
    """Every other workload measured in the same run: ms per step, Mqueries/s,
    build GB/s, the level pass against the copy bandwidth and a sampled
    definitional check; the learned-select workload also compares learned and
    sampled select; the batched workload runs its graph."""
    recs = {}
    for name in ("plain", "large_alphabet", "learned"):
        wl = workloads.WORKLOADS[name]
        sym, counts, q, outs, Q = prepare(wl, 0)
        m = measure(wt, wl, sym, q, outs, max(3, min(args.steps, 5)), 3, wt.LAYOUT_TREE, overlap=args.overlap)
        phases, roof, kern = analyse(wl, q, m, max(3, min(args.steps, 5)))
        rec = {"workload": wl.describe(), "ms_per_step": m["ms"], "Mqps": Q / (m["ms"] * 1e-3) / 1e6,
               "queries_per_step": Q, "build_ms": phases["build_ms"], "build_GBps": phases["build_GBps"],
               "level_pass_frac": roof.get("level_pass_frac"), "phases": phases, "queries_roofline": roof["queries"],
               "parity": definitional_check(wl, sym, q, outs)}
        if name == "learned":
            rec["learned_select"] = learned_compare(wt, wl, sym, q, reps=5)
        recs[name] = rec
        del sym, q, outs, counts
    try:
        recs["batched"] = batched_record(args, wt, workloads, 4096, max(3, min(args.steps, 5)), 0, 1, None,
                                         with_e2e=False)
    except Exception as e:  # reported, not hidden
        recs["batched"] = {"error": repr(e)}
    return recs


def learned_compare(wt, wl, sym, q, reps=5):
    """Sampled select against learned select (PLA, then the trained MLP) on the
    workload's select queries, same tree and GPU; median of `reps` timed
    repeats per arm (CUDA events); answers must be identical."""
    import numpy as np
    import torch

    if "select_j" in q:
        c, j = q["select_c"], q["select_j"]
    else:
        msk = q["mixed_kind"] == 2
        c, j = q["mixed_c"][msk].contiguous(), q["mixed_arg"][msk].contiguous()
    out = torch.empty(j.numel(), dtype=torch.int64, device="cuda")
    ref = torch.empty_like(out)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), ts

    res = {"queries": int(j.numel()), "reps": reps}
    with wt.build(sym, wl.sigma, sample_k=wl.sample_k) as t:
        ms, ts = timed(lambda: t.select(c, j, out=ref))
        inf = t.info()
        sample_bytes = sum(((inf.level_size[l] - inf.level_ones[l]) // wl.sample_k + 1
                            + inf.level_ones[l] // wl.sample_k + 1) * 8 for l in range(inf.levels))
        res["sampled"] = {"ms": ms, "ms_runs": ts, "Mqps": j.numel() / (ms * 1e-3) / 1e6, "bytes": sample_bytes}
        for name, mode in (("pla", wt.LEARN_PLA), ("mlp", wt.LEARN_MLP)):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            t.train_select(mode)
            e1.record()
            torch.cuda.synchronize()
            train_ms = e0.elapsed_time(e1)
            ms, ts = timed(lambda: t.select_learned(c, j, out=out))
            li = t.learned_info()
            epsm = [li.eps_mean[l][b] for l in range(inf.levels) for b in (0, 1)]
            res[name] = {"ms": ms, "ms_runs": ts, "Mqps": j.numel() / (ms * 1e-3) / 1e6, "train_ms": train_ms,
                         "identical_to_sampled": bool(torch.equal(out, ref)), "fallbacks": int(li.fallbacks),
                         "mean_window_bits": 2 * float(np.mean(epsm)) + 1, "model_bytes": int(li.model_bytes),
                         "speedup_vs_sampled": res["sampled"]["ms"] / ms}
    return res


def _query_traffic(kind):
    """Measured DRAM bytes per query of a walk kernel (profiles/traffic.json,
    from a one-kernel ncu capture), or None if absent or the source changed."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)["queries"][kind]
        for fn, sha in rec["sources"].items():
            with open(os.path.join(ROOT, fn), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest()[:16] != sha:
                    return None
    except Exception:
        return None
    return float(rec["dram_bytes_per_query"])


def _measured_traffic(kernel, symbols_per_launch):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json),
    scaled by the symbols one launch processes; None if the kernel source changed
    since the counters were taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["file"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except Exception:
        return None
    if sha != rec["source_sha256_16"]:
        return None
    return rec["dram_bytes_per_symbol"] * symbols_per_launch


def _e2e(args, wl, sym, q, outs, step, barrier, dist, world, Q):
    import torch
    from paper_2505_03372_gb300 import binding as wt

    h_sym = sym.cpu().pin_memory()
    h_q = {k: v.cpu().pin_memory() for k, v in q.items()}
    h_out = {k: torch.empty(v.numel(), dtype=v.dtype, pin_memory=True) for k, v in outs.items()}
    h2d = h_sym.numel() * h_sym.element_size() + sum(v.numel() * v.element_size() for v in h_q.values())
    d2h = sum(v.numel() * v.element_size() for v in h_out.values())

    def run(nsteps):
        # Everything through the host-memory entry points.  wt_build_host copies
        # the symbols in chunks on its own copy stream, which does not wait for
        # the work already queued, so step k+1's copy overlaps step k's level
        # passes and walks; every step's inputs are still copied in, and its
        # answers copied out, inside the timed region.
        for k in range(nsteps):
            t = wt.build(h_sym, wl.sigma, sample_k=wl.sample_k, allocator=None,
                         layout=wt.LAYOUT_MATRIX if args.layout == "matrix" else wt.LAYOUT_TREE)
            # queries and answers: the host query pipeline (wt_query_host), whose
            # copies overlap the build and the other batches' walks
            if "access_i" in h_q:
                t.query_host(0, h_q["access_i"], out=h_out["access"])
            if "rank_i" in h_q:
                t.query_host(1, h_q["rank_i"], c=h_q["rank_c"], out=h_out["rank"])
            if "select_j" in h_q:
                t.query_host(2, h_q["select_j"], c=h_q["select_c"], out=h_out["select"])
            if "mixed_arg" in h_q:
                t.query_host(3, h_q["mixed_arg"], c=h_q["mixed_c"], kinds=h_q["mixed_kind"], out=h_out["mixed"])
            t.close()

    run(max(args.warmup, 3))
    # three windows of the timed steps, the median reported: the host side of
    # this leg varies between windows far more than the device work does
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(args.steps)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        runs.append(job_ms(e0.elapsed_time(e1) / args.steps, dist))
    ms = statistics.median(runs)
    # the answers of the last step, checked against the device-resident run
    for k in h_out:
        if not torch.equal(h_out[k], outs[k].cpu()):
            raise RuntimeError(f"e2e answers differ from the device-resident run ({k})")
    return {"value": job_value(world, Q, ms), "unit": UNIT, "ms_per_step": ms, "ms_per_step_windows": runs,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "path": "pinned host symbols -> wt_build_host (64 MiB chunks copied while the histogram runs; the "
                    "next step's copy overlaps this step's passes) ; pinned host queries -> wt_query_host (chunked "
                    "H2D, walk, D2H on two copy streams) -> pinned host answers"}


def batched_record(args, wt, workloads, ntrees, steps, rank, world, dist, with_e2e=True):
    """4096 independent trees (n log-uniform in [2^10, 2^24] uint16, sigma from
    {4, 256, 65536}) built and queried (log-uniform [16, 2^16] mixed queries per
    tree) by one CUDA-graph launch per step; K and the query CTA size come from
    the autotuner (timed on a calibration subset before the timed region).
    Under torchrun the trees are split across the ranks (contiguous ranges of
    the drawn batch, no collective); each rank builds and queries its share."""
    import numpy as np
    import torch
    from paper_2505_03372_gb300 import autotune

    buf, views, sigmas, q = workloads.make_batch(ntrees=ntrees, seed=workloads.SEED_BASE + 3)
    lo, hi = shard_range(len(views), rank, world)
    if world > 1:
        buf, views, sigmas, q = workloads.batch_subset(views, sigmas, q, lo, hi)
    t0 = time.perf_counter()
    opts = autotune.tune_batch(views, sigmas, q)
    tune_s = time.perf_counter() - t0
    Q = q["arg"].numel()
    nsym = sum(v.numel() for v in views)
    local = torch.cuda.current_device()
    with wt.Batch(views, sigmas, **opts) as b:
        out = b.set_queries(q["tree"], q["kind"], q["c"], q["arg"])
        for _ in range(max(args.warmup, 3)):
            b.run()
        st = b.status_sync()
        if st != wt.WT_OK:
            raise RuntimeError("batch status: " + wt.status_str(st))
        launches0 = wt.profile_launches()
        clocks = ClockSampler(local) if (rank == 0 and with_e2e) else None
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            b.run()
        e1.record()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        launches = wt.profile_launches() - launches0
        ms = job_ms(e0.elapsed_time(e1) / steps, dist)
        # algorithmic bytes of one step: every tree's level-wise build plus the query sectors
        K = opts["sample_k"]
        bbytes = 0
        kinds = q["kind"].cpu().numpy()
        trees = q["tree"].cpu().numpy()
        Ls = []
        for v, sg in zip(views, sigmas):
            L = max(1, int(math.ceil(math.log2(sg)))) if sg > 1 else 0
            Ls.append(L)
            bbytes += build_bytes(v.numel(), 2, [v.numel()] * L, K)
        Lq = np.array(Ls)[trees]
        secs = np.where(kinds == 0, 2.5 * (Lq - 1) + 1, np.where(kinds == 1, 2.5 * Lq, 6.5 * Lq))
        qbytes = float(secs.sum()) * 32
        peak, peak_kind = peaks()
        achieved = (bbytes + qbytes) / (ms * 1e-3) / 1e9
        # a sampled check of the answers against their definitions, tree by tree
        outs_np = out.cpu().numpy().view(np.uint64)
        g = np.random.default_rng(7)
        bad = checked = 0
        for k in g.integers(0, Q, min(200, Q)):
            tr, kd, c, x = int(trees[k]), int(kinds[k]), int(q["c"][k]) & 0xFFFFFFFF, int(q["arg"][k])
            S = workloads.symbols_as_int64(views[tr])
            gv = int(outs_np[k])
            checked += 1
            if kd == 0:
                bad += int(int(S[x]) != gv)
            elif kd == 1:
                bad += int(int((S[:x] == c).sum()) != gv)
            else:
                bad += int(not (0 <= gv < S.numel() and int(S[gv]) == c and int((S[:gv] == c).sum()) == x - 1))
        rec = {"workload": f"{ntrees} trees, n log-uniform [2^10, 2^24] uint16, sigma from {{4, 256, 65536}}, "
                           f"uniform symbols; log-uniform [16, 2^16] mixed queries per tree",
               "trees_this_rank": len(views), "symbols": nsym, "queries_per_step": Q, "ms_per_step": ms,
               "Mqps": job_value(world, Q, ms), "build_input_GBps": nsym * 2 / (ms * 1e-3) / 1e9,
               "options": opts, "tune_s": tune_s, "device_bytes": b.nbytes(), "gpu_launches": launches,
               "graph_kernels": None, "clocks": clk,
               "roofline": {"bound": "hbm", "kernel": "whole graph (build + queries)", "achieved": achieved,
                            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                            "algorithmic_bytes_per_launch": bbytes + qbytes, "avg_launch_ms": ms,
                            "peak_source": f"{peak_kind} copy bandwidth"},
               "parity": {"checked": checked, "ok": bad == 0, "mismatches": bad,
                          "how": "sampled answers against their definitions on each tree's symbols (torch)"}}
        if with_e2e:
            # end to end: symbols and queries from pinned host memory, results back
            h_buf = buf.cpu().pin_memory()
            h_q = {k: v.cpu().pin_memory() for k, v in q.items()}
            h_out = torch.empty(Q, dtype=torch.int64, pin_memory=True)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record()
            for _ in range(steps):
                buf.copy_(h_buf, non_blocking=True)
                for k in q:
                    q[k].copy_(h_q[k], non_blocking=True)
                b.run()
                h_out.copy_(out, non_blocking=True)
            f1.record()
            torch.cuda.synchronize()
            e2e_ms = job_ms(f0.elapsed_time(f1) / steps, dist)
            h2d = h_buf.numel() * h_buf.element_size() + sum(v.numel() * v.element_size() for v in h_q.values())
            rec["e2e"] = {"value": job_value(world, Q, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                          "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": Q * 8,
                          "path": "pinned host symbols and queries -> H2D -> wt_batch_run (graph) -> D2H results"}
    return rec


def shard_range(ntrees, rank, world):
    """Contiguous range [lo, hi) of the batch's trees that a rank builds and queries."""
    per, extra = divmod(ntrees, world)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def run_batched(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_03372_gb300 import binding as wt, workloads

    ntrees = int(args.n) if args.n else 4096
    rec = batched_record(args, wt, workloads, ntrees, args.steps, rank, world, dist, with_e2e=True)
    line = {
        "metric": METRIC, "value": rec["Mqps"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic", "impl": "ours",
        "config": {"workload": rec["workload"], "trees_per_rank": rec["trees_this_rank"], "options": rec["options"],
                   "tune_s": rec["tune_s"], "device_bytes": rec["device_bytes"],
                   "parallelism": "trees split across ranks" if world > 1 else "1 GPU",
                   "l2_flush": "inputs larger than L2 (symbols and trees tens of GB)"},
        "phases": {"step_ms": rec["ms_per_step"], "build_input_GBps": rec["build_input_GBps"]},
        "roofline": rec["roofline"], "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
        "parity": rec["parity"], "e2e": rec.get("e2e"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_bitvector(args):
    """The paper's standalone binary rank / select experiment on synthetic
    Kurpicz-style bitvectors: 2^32 bits with a fill of 10, 50 or 90 %, ones
    uniform or 99 % at the end; per bitvector 1e8 rank, 1e8 select_0 and 1e8
    select_1 queries (uniform positions / ranks), one thread per query.  A step
    answers all of them on all six bitvectors."""
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_03372_gb300 import binding as wt, workloads

    nbits = int(args.n) if args.n else 1 << 32
    q = max(1, int(1e8 * args.query_scale))
    K = 4096
    g = workloads.generator(workloads.SEED_BASE + 6 + 7919 * rank, "cuda")
    cases = []
    for layout in ("uniform", "adversarial"):
        for fill in workloads.BITVECTOR_FILLS:
            words = workloads.make_bitvector(nbits, fill, layout, seed=workloads.SEED_BASE + 5 + int(fill * 100),
                                             device="cuda")
            bv = wt.Bitvector(words, nbits, sample_k=K)
            del words
            # the support kernel alone (counters, samples and the ones count), timed again
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bv.support()
            e1.record()
            torch.cuda.synchronize()
            i = torch.randint(0, nbits + 1, (q,), generator=g, device="cuda", dtype=torch.int64)
            cnt = {1: bv.ones, 0: nbits - bv.ones}
            j = {b: (torch.rand(q, generator=g, device="cuda", dtype=torch.float64) * cnt[b]).to(torch.int64) + 1
                 for b in (0, 1)}
            cases.append({"name": f"{layout} {int(fill * 100)} %", "bv": bv, "i": i, "j": j,
                          "support_ms": e0.elapsed_time(e1), "out": torch.empty(q, dtype=torch.int64, device="cuda")})

    def step():
        for c in cases:
            c["bv"].rank(c["i"], out=c["out"])
            c["bv"].select(0, c["j"][0], out=c["out"])
            c["bv"].select(1, c["j"][1], out=c["out"])

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    for c in cases:
        if c["bv"].status_sync() != wt.WT_OK:
            raise RuntimeError("bitvector status after warm-up")
    launches0 = wt.profile_launches()
    clocks = ClockSampler(local) if rank == 0 else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    launches = wt.profile_launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    Q = 3 * q * len(cases)
    # per-kind times, measured again call by call (outside the timed region)
    peak, peak_kind = peaks()
    phases, qroof = {}, {}
    tot = {"rank": 0.0, "select": 0.0}
    for c in cases:
        row = {"support_ms": c["support_ms"], "ones": c["bv"].ones}
        for kind, fn in (("rank", lambda: c["bv"].rank(c["i"], out=c["out"])),
                         ("select0", lambda: c["bv"].select(0, c["j"][0], out=c["out"])),
                         ("select1", lambda: c["bv"].select(1, c["j"][1], out=c["out"]))):
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record()
            fn()
            f1.record()
            torch.cuda.synchronize()
            t = f0.elapsed_time(f1)
            row[f"{kind}_Mqps"] = q / (t * 1e-3) / 1e6
            tot["rank" if kind == "rank" else "select"] += t
        phases[c["name"]] = row
    for kind, sec in (("rank", 2.5), ("select", 6.5)):
        nq = q * len(cases) * (1 if kind == "rank" else 2)
        gsec = nq * sec / (tot[kind] * 1e-3) / 1e9
        qroof[kind] = {"sectors_per_query": sec, "achieved_Gsectors_s": gsec, "peak_Gsectors_s": peak / 32,
                       "frac": gsec / (peak / 32)}
    dom = max(qroof, key=lambda k: tot[k])
    line = {
        "metric": METRIC, "value": world * Q / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "ours",
        "config": {"workload": f"bitvector: {nbits} bits, fill 10/50/90 %, uniform and adversarial (99 % of the "
                               f"ones at the end); {q} rank, {q} select_0 and {q} select_1 each; K = {K}",
                   "queries_per_step_per_gpu": Q,
                   "l2_flush": "inputs larger than L2 (six 512 MiB bitvectors, 2.4 GB of queries)"},
        "phases": phases,
        "roofline": {"bound": "hbm", "kernel": f"bv_{dom}", "achieved": qroof[dom]["achieved_Gsectors_s"] * 32,
                     "peak": peak, "unit": "GB/s", "frac": qroof[dom]["frac"], "traffic": None,
                     "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "queries": qroof},
        "gpu_launches": launches, "clocks": clk, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "bitvector":
        run_bitvector(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
