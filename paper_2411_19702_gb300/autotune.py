"""Autotuner for the tensor-core Gram: tile width, kernel and sample split per (m, n) bucket.

The Gram runs either single-CTA tiles of 128 x tile_n (tile_n in {64, 128,
256}; 240 with FP4 operands) or CTA-pair tiles of 256 x 256 (256 x 240 with
FP4) on clusters of two SMs.  Narrow tiles waste less padding when n is
small; wide tiles and CTA pairs stream fewer operand bytes per pair but need
enough tiles to fill the GPU.  ``tune`` measures, for one representative
shape per (m, n) bucket (floor(log2 m), floor(2 log2 n) -- the buckets the
native table uses), the device time of the fused kernel for every candidate
(each single-CTA width, and CTA pairs) through the library's event profiler,
keeps the fastest, and installs the choice: the bucket's single-CTA width
(``gbmi_tuner_set``) and whether it runs on CTA pairs
(``gbmi_tuner_set_pair``).  For buckets narrow enough that a call may have
fewer tiles than the GPU runs at once, it then times the sample split with
that kernel (the cost model's choice, no split, or 2-32 sample ranges) and
installs the fastest (``gbmi_tuner_set_split``).  Single calls, batches and
servers then follow the table.  Tables are saved and loaded as JSON.
"""
from __future__ import annotations

import json
import math

from . import gbmi

CANDIDATES = (("single", 64), ("single", 128), ("single", 256), ("pair", 0))
# sample splits timed per bucket: 0 = the cost model, 1 = none, S = S ranges
SPLITS = (0, 1, 2, 4, 8, 16, 32)
# widest n whose calls can have fewer tiles than concurrent slots (a wider
# all-pairs call fills the GPU and never splits)
SPLIT_MAX_N = 3000


def bucket(m: int, n: int) -> tuple[int, int]:
    return int(math.floor(math.log2(max(m, 1)))), int(math.floor(2.0 * math.log2(max(n, 1))))


def _time_calls(X, reps: int) -> float:
    """Device time of the Gram launches of one fused call under the current settings."""
    import torch
    n = X.shape[1]
    out = torch.empty((n, n), dtype=torch.float32, device=X.device)
    gbmi.mi_all_pairs(X, out=out, path="fused")
    gbmi.sync()
    gbmi.profile(enable=True, reset=True)
    for _ in range(reps):
        gbmi.mi_all_pairs(X, out=out, path="fused")
    prof = gbmi.profile(enable=False)
    # the Gram launches of the call (one fused launch, or the sample split's
    # counts launch and the MI kernel that sums its parts)
    ms = sum(v["ms"] for k, v in prof.items() if k.startswith("gram_tc") or k == "mi_from_counts")
    calls = max((v["launches"] for k, v in prof.items() if k.startswith("gram_tc")), default=0)
    return ms / calls if calls else float("inf")


def _time_candidate(X, kind: str, tile_n: int, reps: int) -> float:
    gbmi.set_option(gbmi.OPT_PAIR, 2 if kind == "pair" else 0)
    gbmi.set_option(gbmi.OPT_TILE_N, tile_n)
    try:
        return _time_calls(X, reps)
    finally:
        gbmi.set_option(gbmi.OPT_TILE_N, 0)
        gbmi.set_option(gbmi.OPT_PAIR, 1)


def _name(kind: str, tile_n: int) -> str:
    return "pair" if kind == "pair" else f"single{tile_n}"


def tune(shapes, candidates=CANDIDATES, reps: int = 3, density: float = 0.1, seed: int = 0,
         device: str = "cuda", install: bool = True) -> dict:
    """Measure each candidate on one random problem per bucket of ``shapes``.

    Returns {"mb,nb": {"m": m, "n": n, "tile_n": best single-CTA width,
    "pair": 0 or 1, "split": sample ranges (0 = the cost model, 1 = none),
    "ms": {candidate: ms}, "ms_split": {ranges: ms}}} (no "ms_split" for
    buckets wider than SPLIT_MAX_N).
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    reps_by_bucket = {}
    for m, n in shapes:
        reps_by_bucket.setdefault(bucket(int(m), int(n)), (int(m), int(n)))
    table = {}
    for key, (m, n) in sorted(reps_by_bucket.items()):
        X = (torch.rand((m, n), generator=g, device=device) < density).to(torch.uint8)
        times = {_name(k, w): _time_candidate(X, k, w, reps) for k, w in candidates}
        singles = {w: times[_name("single", w)] for k, w in candidates if k == "single"}
        best_w = min(singles, key=lambda w: (singles[w], -w)) if singles else 256
        best = min(times, key=lambda c: times[c])
        entry = {"m": m, "n": n, "tile_n": best_w, "pair": 1 if best == "pair" else 0,
                 "split": 0, "ms": times}
        if n <= SPLIT_MAX_N:
            # the sample split with the bucket's kernel and width (forced by
            # options, so the table is left as it was)
            gbmi.set_option(gbmi.OPT_PAIR, 2 if entry["pair"] else 0)
            gbmi.set_option(gbmi.OPT_TILE_N, 0 if entry["pair"] else best_w)
            split_ms = {}
            try:
                for parts in SPLITS:
                    gbmi.tuner_set_split(m, n, parts)
                    split_ms[str(parts)] = _time_calls(X, reps)
            finally:
                gbmi.tuner_set_split(m, n, 0)
                gbmi.set_option(gbmi.OPT_TILE_N, 0)
                gbmi.set_option(gbmi.OPT_PAIR, 1)
            # ties keep the cost model (0), then the fewest ranges
            entry["split"] = int(min(split_ms, key=lambda p: (split_ms[p], p != "0", int(p))))
            entry["ms_split"] = split_ms
        table[f"{key[0]},{key[1]}"] = entry
        del X
    if install:
        apply(table)
    return table


def tune_batch(Xs, Ys=None, table: dict | None = None, reps: int = 3) -> dict:
    """Choose the kernel assignment of a grouped batch by timing the whole batch.

    Candidates: the built-in rule (jobs whose both sides span >= 768 variables
    on CTA pairs), the per-bucket ``table`` (if given), every job on
    single-CTA tiles, every job on CTA pairs.  Each is built as a batch plan
    (one CUDA graph) and timed with CUDA events over ``reps`` replays; the
    fastest setting is left installed (GBMI_OPT_PAIR and the tuner table) and
    returned with all times: {"best": name, "ms": {name: ms}}.
    """
    import torch

    def timed(setup):
        setup()
        plan = gbmi.Batch(Xs, Ys)
        try:
            plan.run()
            gbmi.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan.run()
            e1.record()
            e1.synchronize()
            gbmi.sync()
            return e0.elapsed_time(e1) / reps
        finally:
            plan.close()

    def rule():
        gbmi.tuner_clear()
        gbmi.set_option(gbmi.OPT_PAIR, 1)

    def with_table():
        rule()
        apply(table)

    def single():
        gbmi.tuner_clear()
        gbmi.set_option(gbmi.OPT_PAIR, 0)

    def pairs():
        gbmi.tuner_clear()
        gbmi.set_option(gbmi.OPT_PAIR, 2)

    setups = {"rule": rule, "single": single, "pairs": pairs}
    if table:
        setups["table"] = with_table
    times = {name: timed(f) for name, f in setups.items()}
    best = min(times, key=lambda k: times[k])
    setups[best]()
    return {"best": best, "ms": times}


def apply(table: dict):
    """Install a table's choices in the library."""
    for entry in table.values():
        gbmi.tuner_set(entry["m"], entry["n"], entry["tile_n"])
        if "pair" in entry:
            gbmi.tuner_set_pair(entry["m"], entry["n"], entry["pair"])
        if "split" in entry:
            gbmi.tuner_set_split(entry["m"], entry["n"], entry["split"])


def save(table: dict, path: str):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path: str, install: bool = True) -> dict:
    with open(path) as f:
        table = json.load(f)
    if install:
        apply(table)
    return table
