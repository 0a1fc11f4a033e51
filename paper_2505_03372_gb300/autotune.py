"""Autotuner for batched trees: picks the select sample interval K, the query
kernel's CTA size and the persistent level pass's CTAs per SM by timing
candidates on a calibration subset of the batch, and caches the choice in a
JSON file keyed by GPU and workload shape.

The search is staged: first the level-pass grid and the query CTA size at
K = 4096 (nine candidates), then K with the best of those (three), so twelve
graph builds instead of twenty-seven.

    from paper_2505_03372_gb300 import autotune
    opts = autotune.tune_batch(views, sigmas, queries)
    # {"sample_k": ..., "query_threads": ..., "lp_ctas_per_sm": ...}
"""
from __future__ import annotations

import json
import math
import os

from . import binding as wt

DEFAULT_CACHE = os.environ.get("WT_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                             ".tune_cache.json"))
SAMPLE_K = (2048, 4096, 8192)
QUERY_THREADS = (128, 256, 512)
LP_CTAS = (2, 4, 6)


def stage1_candidates():
    return [{"sample_k": 4096, "query_threads": t, "lp_ctas_per_sm": c} for c in LP_CTAS for t in QUERY_THREADS]


def stage2_candidates(best):
    return [dict(best, sample_k=k) for k in SAMPLE_K if k != best["sample_k"]]


def shape_key(views, sigmas, queries, device_name=None) -> str:
    """Cache key: GPU name, symbol width, the set of alphabet sizes, the rounded
    log2 of the mean tree size, the tree count and the rounded log2 of the
    query count."""
    if device_name is None:
        import torch

        device_name = torch.cuda.get_device_name()
    n = [v.numel() for v in views]
    return "|".join([
        device_name,
        f"w{views[0].element_size()}",
        "sigma" + ",".join(str(s) for s in sorted(set(int(x) for x in sigmas))),
        f"logn{round(math.log2(max(1, sum(n) / len(n))))}",
        f"trees{len(views)}",
        f"q{round(math.log2(max(1, queries['arg'].numel())))}",
    ])


def load_cache(path):
    """The cache file's contents, or {} if it is missing or unreadable."""
    try:
        with open(path) as f:
            c = json.load(f)
        return c if isinstance(c, dict) else {}
    except (OSError, ValueError):
        return {}


def calibration_subset(views, sigmas, queries, stride):
    """Every stride-th tree and its queries, tree ids renumbered."""
    import torch

    idx = list(range(0, len(views), stride))
    sub_v = [views[i] for i in idx]
    sub_s = [sigmas[i] for i in idx]
    remap = torch.full((len(views),), -1, dtype=torch.int64, device=queries["tree"].device)
    remap[torch.tensor(idx, device=remap.device)] = torch.arange(len(idx), device=remap.device)
    keep = remap[queries["tree"].long()] >= 0
    sq = {k: v[keep].contiguous() for k, v in queries.items()}
    sq["tree"] = remap[sq["tree"].long()].to(torch.int32).contiguous()
    return sub_v, sub_s, sq


def time_graph(views, sigmas, queries, cand, reps=3):
    """Mean ms of one graph launch (build + queries) with the candidate's options."""
    import torch

    with wt.Batch(views, sigmas, **cand) as b:
        b.set_queries(queries["tree"], queries["kind"], queries["c"], queries["arg"])
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
               force: bool = False, timer=None, device_name=None) -> dict:
    """Best options for this batch shape, timed on every `stride`-th tree and
    its queries (`timer(views, sigmas, queries, candidate) -> ms`, default
    time_graph), cached under shape_key."""
    key = shape_key(views, sigmas, queries, device_name)
    cache = load_cache(cache_path)
    if key in cache and not force:
        return dict(cache[key]["best"])
    if timer is None:
        sub = calibration_subset(views, sigmas, queries, stride)

        def timer(v, s, q, cand):
            return time_graph(*sub, cand, reps)
    results = [(timer(views, sigmas, queries, c), c) for c in stage1_candidates()]
    best = min(results, key=lambda r: r[0])[1]
    results += [(timer(views, sigmas, queries, c), c) for c in stage2_candidates(best)]
    best = min(results, key=lambda r: r[0])[1]
    cache[key] = {"best": best, "timings_ms": [[r[0], r[1]] for r in results]}
    try:
        tmp = cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    except OSError:
        pass
    return dict(best)
