"""Autotuner for batched trees: picks the select sample interval K and the
query kernel's CTA size by timing candidates on a calibration subset of the
batch, and caches the choice in a JSON file keyed by GPU and workload shape.

    from paper_2505_03372_gb300 import autotune
    opts = autotune.tune_batch(views, sigmas, queries)   # {"sample_k": ..., "query_threads": ...}
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import binding as wt

DEFAULT_CACHE = os.environ.get("WT_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                             ".tune_cache.json"))
CANDIDATES = [{"sample_k": k, "query_threads": t} for k in (2048, 4096, 8192) for t in (128, 256, 512)]


def shape_key(views, sigmas, queries) -> str:
    n = [v.numel() for v in views]
    return "|".join([
        torch.cuda.get_device_name(),
        f"w{views[0].element_size()}",
        "sigma" + ",".join(str(s) for s in sorted(set(int(x) for x in sigmas))),
        f"logn{round(math.log2(max(1, sum(n) / len(n))))}",
        f"trees{len(views)}",
        f"q{round(math.log2(max(1, queries['arg'].numel())))}",
    ])


def _time(b, reps):
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(views, sigmas, queries, cache_path: str = DEFAULT_CACHE, stride: int = 16, reps: int = 3,
               candidates=CANDIDATES, force: bool = False) -> dict:
    """Best options for this batch shape; timed on every `stride`-th tree and its queries."""
    key = shape_key(views, sigmas, queries)
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if key in cache and not force:
        return cache[key]["best"]
    idx = list(range(0, len(views), stride))
    sub_v = [views[i] for i in idx]
    sub_s = [sigmas[i] for i in idx]
    remap = torch.full((len(views),), -1, dtype=torch.int64, device=queries["tree"].device)
    remap[torch.tensor(idx, device=remap.device)] = torch.arange(len(idx), device=remap.device)
    keep = remap[queries["tree"].long()] >= 0
    sq = {k: v[keep].contiguous() for k, v in queries.items()}
    sq["tree"] = remap[sq["tree"].long()].to(torch.int32).contiguous()
    results = []
    for cand in candidates:
        with wt.Batch(sub_v, sub_s, sample_k=cand["sample_k"], query_threads=cand["query_threads"]) as b:
            b.set_queries(sq["tree"], sq["kind"], sq["c"], sq["arg"])
            results.append((_time(b, reps), cand))
    best = min(results, key=lambda r: r[0])[1]
    cache[key] = {"best": best, "timings_ms": [[r[0], r[1]] for r in results]}
    try:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best
