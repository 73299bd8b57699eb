"""Autotuner: pick launch parameters per size class of the sieved ranges.

A size class is (range start band, width band).  For each class a seeded set
of representative intervals is sieved with every candidate parameter set
(segment bytes, small-prime limit, threads per CTA, bucket limit, chunk size)
and the fastest is kept.  The table is JSON:

    {"device": "...", "classes": {"<lo band>/<w band>": {"segment_bytes": ..., ...}}}

``plan_for(table, lo, hi)`` returns the parameters for one range, and
``Sieve.apply_plan`` / ``batch_count_tuned`` in the package use them.

  python -m paper_1205_4883_gb300.autotune [--out tuned.json] [--quick]
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import time
from typing import Dict, List, Sequence, Tuple

from .workloads import SplitMix64, log_uniform_int

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuned.json")

# band edges (log10): start of the range and its width
LO_BANDS = [(0, 10), (10, 13), (13, 19)]
W_BANDS = [(0, 5), (5, 7), (7, 9), (9, 19)]

PARAM_KEYS = {"segment_bytes": 1, "threads": 2, "small_limit": 3, "ctas_per_sm": 4,
              "chunk_segments": 5, "bucket_limit": 6, "cursor_mb": 7, "mid_limit": 9}


def band(x: int, bands) -> int:
    lx = math.log10(x) if x > 0 else 0.0
    for i, (a, b) in enumerate(bands):
        if a <= lx < b:
            return i
    return len(bands) - 1


def class_key(lo: int, hi: int) -> str:
    return f"{band(max(lo, 1), LO_BANDS)}/{band(max(hi - lo, 1), W_BANDS)}"


def plan_for(table: dict, lo: int, hi: int) -> Dict[str, int]:
    return dict(table.get("classes", {}).get(class_key(lo, hi), {}))


def load_table(path: str = DEFAULT_TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {"classes": {}}


def sample_class(lo_band, w_band, n: int, seed: int, hi_max: int) -> Tuple[List[int], List[int]]:
    rng = SplitMix64(seed)
    los, his = [], []
    for _ in range(n):
        lo = log_uniform_int(rng, *lo_band)
        w = log_uniform_int(rng, *w_band)
        lo = min(lo, hi_max - w - 1)
        los.append(max(lo, 0))
        his.append(max(lo, 0) + w)
    return los, his


def candidates(quick: bool):
    segs = [65536, 229376] if quick else [32768, 65536, 131072, 229376]
    smalls = [448] if quick else [256, 448, 896]
    threads = [1024] if quick else [512, 1024]
    buckets = [1 << 62, 0]
    chunks = [16]
    for seg, small, thr, bl, ch in itertools.product(segs, smalls, threads, buckets, chunks):
        yield {"segment_bytes": seg, "small_limit": small, "threads": thr, "bucket_limit": bl,
               "chunk_segments": ch, "ctas_per_sm": 1}


def tune(out: str = DEFAULT_TABLE, quick: bool = False, budget_s: float = 240.0) -> dict:
    import torch

    from . import Sieve
    t_start = time.time()
    hi_cap = 10**14 + 10**9 + 1
    sv = Sieve(hi_cap)
    table = {"device": torch.cuda.get_device_name(0), "classes": {}, "timing_ms": {}}
    cands = list(candidates(quick))
    for (li, lb), (wi, wb) in itertools.product(enumerate(LO_BANDS), enumerate(W_BANDS)):
        lb_c = (lb[0], min(lb[1], 14))
        wb_c = (wb[0], min(wb[1], 9 if li < 2 else 8))
        if lb_c[0] >= lb_c[1] or wb_c[0] >= wb_c[1]:
            continue
        n = 64 if wb_c[1] <= 7 else 8
        los, his = sample_class(lb_c, wb_c, n, seed=1205 + 17 * li + wi, hi_max=hi_cap)
        best, best_ms, timings = None, float("inf"), {}
        for c in cands:
            if time.time() - t_start > budget_s:
                break
            for k, v in c.items():
                sv.set_param(PARAM_KEYS[k], v)
            sv.batch_count(los, his)  # warm-up (and graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                sv.batch_count(los, his)
            ms = (time.perf_counter() - t0) / 3 * 1e3
            timings[json.dumps(c, sort_keys=True)] = ms
            if ms < best_ms:
                best, best_ms = c, ms
        if best is not None:
            key = f"{li}/{wi}"
            table["classes"][key] = best
            table["timing_ms"][key] = {"best": best_ms, "integers": sum(h - l for l, h in zip(los, his)),
                                       "candidates": len(timings)}
    sv.close()
    with open(out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--budget-s", type=float, default=240.0)
    a = ap.parse_args()
    t = tune(a.out, a.quick, a.budget_s)
    print(json.dumps(t["classes"], indent=1))
