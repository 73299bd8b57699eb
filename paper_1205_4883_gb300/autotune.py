"""Autotuner: launch parameters per size class of the sieved ranges.

The paper's Algorithm 1 picks how a block is sieved from its size (one core
for a short last block, two from both ends otherwise).  The GPU form is a
table from a range's size class -- the band of its start and the band of its
width -- to launch parameters: segment bytes, wheel (mod 30 or mod 210),
bucket limit, the per-phase tier's limit and the Miller-Rabin threshold.
``sieve_batch_count_params`` applies them per range inside one batched
launch, so a batch mixing all classes is still one graph launch.

The objective is the time of a whole mixed batch: a seeded batch drawn from the
same distribution as the 4096-interval workload (lo log-uniform in
[10^6, 10^14], width log-uniform in [10^3, 10^8]) but from another seed, so
that the workload itself is held out.  Timing a class on its own would
mislead: one launch sizes shared memory for its largest segment, so a class
that gains from a small segment alone (a larger L1 share) does not gain in
the mix.  The search is coordinate-wise: starting from the context's
defaults, for each class (heaviest first) and each parameter in turn, the
candidate value that makes the batch fastest is kept if it wins by a clear
margin; two passes.  The defaults are always a candidate, so the tuned table
is never slower than the defaults on the tuning batch.  The table is JSON:

    {"device": "...", "classes": {"<lo band>/<w band>": {"seg_bytes": ..., ...}},
     "timing_ms": {...}}

  python -m paper_1205_4883_gb300.autotune [--out tuned.json] [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from typing import Dict, List, Sequence, Tuple

from .workloads import SplitMix64, log_uniform_int

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuned.json")

# band edges (log10): start of the range and its width
LO_BANDS = [(0, 8), (8, 10), (10, 12), (12, 13), (13, 19)]
W_BANDS = [(0, 4), (4, 5), (5, 6), (6, 7), (7, 19)]

MR_NEVER = 0xFFFFFFFF
BUCKETS_OFF = 1 << 62
# candidates per parameter (0 = the context's default for that field)
CANDIDATES = {
    "seg_bytes": [0, 32768, 65536, 131072],
    "wheel": [0, 210],
    "bucket_limit": [0, 229376, 1 << 20],
    "mid_limit": [0, 4096, 16384],
    "mr_percent": [0, 5, 25, 100],
}
FIELDS = tuple(CANDIDATES)
# a candidate replaces the current choice only if it is this much faster
MIN_GAIN = 0.01


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


def range_params(table: dict, lo: Sequence[int], hi: Sequence[int]) -> List[Dict[str, int]]:
    """The per-range launch parameters (sieve_range_params fields) for a batch."""
    classes = table.get("classes", {})
    return [{k: v for k, v in classes.get(class_key(a, b), {}).items() if k in FIELDS} for a, b in zip(lo, hi)]


def range_params_array(table: dict, lo: Sequence[int], hi: Sequence[int]):
    """range_params as a sieve_range_params array, built with numpy (one table row
    per size class, gathered by each range's class index)."""
    import numpy as np

    from . import range_params_array as to_array
    lo_a = np.asarray(lo, dtype=np.float64)
    w_a = np.asarray(hi, dtype=np.float64) - lo_a

    def bands_of(x, bands):
        lx = np.log10(np.maximum(x, 1.0))
        idx = np.full(len(x), len(bands) - 1, dtype=np.int64)
        for i in range(len(bands) - 1, -1, -1):
            a, b = bands[i]
            idx[(lx >= a) & (lx < b)] = i
        return idx

    li, wi = bands_of(lo_a, LO_BANDS), bands_of(w_a, W_BANDS)
    rows = [{k: v for k, v in table.get("classes", {}).get(f"{a}/{b}", {}).items() if k in FIELDS}
            for a in range(len(LO_BANDS)) for b in range(len(W_BANDS))]
    per_class = to_array(rows)
    out = per_class[li * len(W_BANDS) + wi] if len(lo) else per_class[:0]
    return np.ascontiguousarray(out)


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


def _time_mixed(sv, los, his, table, reps: int) -> float:
    """Median host time (ms) of the batch with the table's per-range parameters."""
    import torch
    pa = range_params_array(table, los, his)
    sv.batch_count_params(los, his, pa)  # warm-up (and graph capture)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        sv.batch_count_params(los, his, pa)
        ts.append(time.perf_counter() - t0)
    return sorted(ts)[len(ts) // 2] * 1e3


def tune(out: str = DEFAULT_TABLE, quick: bool = False, budget_s: float = 300.0, hi_cap: int = 10**14 + 10**9 + 1,
         passes: int = 2, m: int = 4096, seed: int = 7) -> dict:
    import torch

    from . import Sieve
    from .workloads import batch_intervals
    t_start = time.time()
    sv = Sieve(hi_cap)
    los, his = batch_intervals(m, seed=seed)
    reps = 3 if quick else 7
    # classes present in the tuning batch, heaviest (most integers) first
    weight: Dict[str, int] = {}
    for a, b in zip(los, his):
        weight[class_key(a, b)] = weight.get(class_key(a, b), 0) + (b - a)
    classes = sorted(weight, key=lambda k: -weight[k])
    table = {"device": torch.cuda.get_device_name(0), "classes": {}, "timing_ms": {},
             "method": f"coordinate search on a mixed batch of {m} intervals (seed {seed}), {passes} passes, "
                       f"median of {reps} timed calls, a change kept only if {MIN_GAIN:.0%} faster"}
    base_ms = _time_mixed(sv, los, his, table, reps)
    best_ms, tried = base_ms, 1
    for _ in range(passes):
        for key in classes:
            for f in FIELDS:
                if time.time() - t_start > budget_s:
                    break
                cur = table["classes"].get(key, {})
                if cur.get("wheel") == 210 and f in ("bucket_limit", "mr_percent"):
                    continue
                for v in CANDIDATES[f]:
                    if v == cur.get(f, 0):
                        continue
                    trial = dict(cur, **{f: v})
                    trial = {k: x for k, x in trial.items() if x}
                    t2 = dict(table, classes=dict(table["classes"], **{key: trial}))
                    ms = _time_mixed(sv, los, his, t2, reps)
                    tried += 1
                    if ms < best_ms * (1 - MIN_GAIN):  # a clear win, not timing noise
                        best_ms, table = ms, t2
    table["classes"] = {k: v for k, v in table["classes"].items() if v}
    table["timing_ms"] = {"defaults": base_ms, "tuned": best_ms, "intervals": m, "seed": seed,
                          "candidates": tried}
    sv.close()
    table["budget_s_used"] = time.time() - t_start
    with open(out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--budget-s", type=float, default=300.0)
    a = ap.parse_args()
    t = tune(a.out, a.quick, a.budget_s)
    print(json.dumps(t["classes"], indent=1))
    print(json.dumps(t["timing_ms"], indent=1))
