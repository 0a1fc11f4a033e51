"""The debug library (libwt_debug.so: every load of a query walk checked
against its array's length, WT_EBOUNDS on a failure).  It stands in for
compute-sanitizer, which is closed on this machine.

A child process runs the same query workload twice: once with the release
library and once with the debug one.  Trees of every width, reduced and
power-of-two alphabets, the wavelet matrix, both learned models, a batch of
trees and standalone bitvectors are covered, with invalid queries mixed in.
The debug run must report no failed check, and its answers and status codes
must equal the release run's.  A planted select sample that points past the
bitvector's end (into padding that the test allocates, so the access stays
inside memory even unchecked) must be caught as WT_EBOUNDS by the debug
library.  The planted case runs with the debug library only.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CHILD = r'''
import hashlib, json, os, sys
sys.path.insert(0, os.environ["WT_TEST_ROOT"])
import torch
from paper_2505_03372_gb300 import binding as wt, workloads

def h(*ts):
    m = hashlib.sha256()
    for t in ts:
        m.update(t.detach().cpu().contiguous().numpy().tobytes())
    return m.hexdigest()[:16]

def invalid(q, n, sigma):
    q = {k: v.clone() for k, v in q.items()}
    if "access_i" in q:
        q["access_i"][:3] = n + 7
        q["rank_c"][:2] = sigma + 1
        q["rank_i"][2:4] = n + 1
        q["select_j"][:2] = 0
        q["select_c"][2:4] = sigma + 3
    return q

res = {}
shapes = [(200003, 96, 1, "zipf", 1.0), (300001, 65536, 2, "zipf", 1.2), (100001, (1 << 20) - 3, 4, "uniform", 1.0),
          (65536, 243, 1, "zipf", 1.0), (131072, 256, 1, "uniform", 1.0)]
for n, sigma, w, dist, s in shapes:
    sym = workloads.make_symbols(n, sigma, w, dist, s, seed=n + sigma, device="cuda")
    wl = workloads.Workload("dbg", 90, n, sigma, w, dist, s, queries={"access": 3001, "rank": 3001, "select": 3001})
    q = invalid(workloads.make_queries(wl, sym, seed=7), n, sigma)
    for layout in (wt.LAYOUT_TREE, wt.LAYOUT_MATRIX):
        with wt.build(sym, sigma, layout=layout) as t:
            a = t.access(q["access_i"])
            r = t.rank(q["rank_c"], q["rank_i"])
            sl = t.select(q["select_c"], q["select_j"])
            st = t.status_sync()
            kinds = (torch.arange(3001, device="cuda") % 3).to(torch.uint8)
            mx = t.query_mixed(kinds, q["rank_c"], torch.where(kinds == 0, q["access_i"],
                               torch.where(kinds == 1, q["rank_i"], q["select_j"])))
            st2 = t.status_sync()
            key = f"{n}_{sigma}_{layout}"
            res[key] = [h(a, r, sl, mx), st, st2]
            if layout == wt.LAYOUT_TREE and sigma == 65536:
                for mode in (wt.LEARN_PLA, wt.LEARN_MLP):
                    t.train_select(mode)
                    ls = t.select_learned(q["select_c"], q["select_j"])
                    res[key + f"_learned{mode}"] = [h(ls), t.status_sync(), int(t.learned_info().fallbacks)]
'''
CHILD += r'''
# a batch of trees with their queries
views, sigmas = [], []
for i, (n, sigma) in enumerate(((5000, 4), (70000, 256), (120001, 65536), (33, 7), (65537, 1000))):
    views.append(workloads.make_symbols(n, sigma, 2, "uniform", 1.0, seed=300 + i, device="cuda"))
    sigmas.append(sigma)
tree = torch.tensor([i % 5 for i in range(4000)], dtype=torch.int32, device="cuda")
kind = (torch.arange(4000, device="cuda") % 3).to(torch.uint8)
c = torch.tensor([[3, 200, 60000, 5, 999][i % 5] for i in range(4000)], dtype=torch.int32, device="cuda")
arg = torch.tensor([1 + (i * 7919) % 30 for i in range(4000)], dtype=torch.int64, device="cuda")
with wt.Batch(views, sigmas) as b:
    out = b.set_queries(tree, kind, c, arg)
    b.run()
    res["batch"] = [h(out), b.status_sync()]
# standalone bitvectors
g = torch.Generator(device="cuda"); g.manual_seed(5)
for nbits, fill in ((4096, 0.3), (1 << 20, 0.9), (70001, 0.5)):
    bits = (torch.rand(nbits, generator=g, device="cuda") < fill)
    words = torch.zeros((nbits + 63) // 64 * 64, dtype=torch.bool, device="cuda")
    words[:nbits] = bits
    wv = (words.view(-1, 64).to(torch.int64) << torch.arange(64, device="cuda")).sum(1)
    bv = wt.Bitvector(wv, nbits, sample_k=256)
    i = torch.randint(0, nbits + 1, (5000,), generator=g, device="cuda")
    j1 = torch.randint(1, max(bv.ones, 1) + 1, (5000,), generator=g, device="cuda")
    j0 = torch.randint(1, max(nbits - bv.ones, 1) + 1, (5000,), generator=g, device="cuda")
    res[f"bv_{nbits}"] = [h(bv.rank(i), bv.select(1, j1), bv.select(0, j0)), bv.status_sync()]
if os.environ.get("WT_LIB_VARIANT") == "debug":
    # planted: sample 1 of the ones points past nbits; words and L2 counters
    # are re-allocated far larger than nbits needs, so the access that the
    # check stops would still land inside them
    nbits = 4096
    bits = torch.rand(nbits, generator=g, device="cuda") < 0.4
    wv = (bits.view(-1, 64).to(torch.int64) << torch.arange(64, device="cuda")).sum(1)
    bv = wt.Bitvector(wv, nbits, sample_k=256)
    big_w = torch.zeros(4096, dtype=torch.int64, device="cuda")
    big_w[:bv.words.numel()] = bv.words
    big_l2 = torch.zeros(1024, dtype=torch.int16, device="cuda")
    big_l2[:bv.l2.numel()] = bv.l2
    bv.words, bv.l2 = big_w, big_l2
    bv.select(1, torch.tensor([100], dtype=torch.int64, device="cuda"))
    res["planted_clean"] = bv.status_sync()
    bv.s1[1] = 32768
    bv.select(1, torch.tensor([300], dtype=torch.int64, device="cuda"))
    res["planted"] = bv.status_sync()
torch.cuda.synchronize()
print("RESULT " + json.dumps(res), flush=True)
'''


def _run(variant):
    env = dict(os.environ, WT_TEST_ROOT=ROOT)
    env.pop("WT_LIB_VARIANT", None)
    if variant == "debug":
        env["WT_LIB_VARIANT"] = "debug"
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_library_checks_every_walk_load_and_changes_no_answer():
    from paper_2505_03372_gb300 import binding as wt

    if not os.path.exists(os.path.join(ROOT, "paper_2505_03372_gb300", "libwt_debug.so")):
        pytest.fail("libwt_debug.so missing: __graft_entry__.build() builds it")
    rel = _run("release")
    dbg = _run("debug")
    assert dbg.pop("planted_clean") == wt.WT_OK
    assert dbg.pop("planted") == wt.WT_EBOUNDS
    assert set(rel) == set(dbg)
    for k in rel:
        assert dbg[k] == rel[k], (k, rel[k], dbg[k])
        assert wt.WT_EBOUNDS not in dbg[k][1:], k
    # the invalid queries were seen (and only as such)
    assert any(v[1] == wt.WT_EQUERY for k, v in rel.items() if not k.startswith(("bv_", "batch")))
