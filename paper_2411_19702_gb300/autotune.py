"""Tile-width autotuner for the tensor-core Gram.

The Gram works on 128 x tile_n output tiles with tile_n in {64, 128, 256}.
Narrow tiles waste less padding when n is small; wide tiles stream fewer
operand bytes per pair.  ``tune`` measures, for one representative shape per
(m, n) bucket (floor(log2 m), floor(2 log2 n) -- the buckets the native table
uses), the device time of the fused kernel with each width through the
library's event profiler, keeps the fastest, and installs the choices with
``gbmi_tuner_set``.  Tables are saved and loaded as JSON.
"""
from __future__ import annotations

import json
import math

from . import gbmi

CANDIDATES = (64, 128, 256)


def bucket(m: int, n: int) -> tuple[int, int]:
    return int(math.floor(math.log2(max(m, 1)))), int(math.floor(2.0 * math.log2(max(n, 1))))


def _time_width(X, tile_n: int, reps: int) -> float:
    import torch
    n = X.shape[1]
    out = torch.empty((n, n), dtype=torch.float32, device=X.device)
    gbmi.set_option(gbmi.OPT_TILE_N, tile_n)
    try:
        gbmi.mi_all_pairs(X, out=out, path="fused")
        gbmi.sync()
        gbmi.profile(enable=True, reset=True)
        for _ in range(reps):
            gbmi.mi_all_pairs(X, out=out, path="fused")
        prof = gbmi.profile(enable=False)
    finally:
        gbmi.set_option(gbmi.OPT_TILE_N, 0)
    g = prof.get("gram_tc_fused_mi")
    return g["ms"] / max(g["launches"], 1) if g else float("inf")


def tune(shapes, candidates=CANDIDATES, reps: int = 3, density: float = 0.1, seed: int = 0,
         device: str = "cuda", install: bool = True) -> dict:
    """Measure each candidate width on one random problem per bucket of ``shapes``.

    Returns {"m,n-bucket": {"m": m, "n": n, "tile_n": best, "ms": {width: ms}}}.
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
        times = {w: _time_width(X, w, reps) for w in candidates}
        best = min(times, key=lambda w: (times[w], -w))
        table[f"{key[0]},{key[1]}"] = {"m": m, "n": n, "tile_n": best,
                                       "ms": {str(w): t for w, t in times.items()}}
        del X
    if install:
        apply(table)
    return table


def apply(table: dict):
    """Install a table's choices in the library."""
    for entry in table.values():
        gbmi.tuner_set(entry["m"], entry["n"], entry["tile_n"])


def save(table: dict, path: str):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path: str, install: bool = True) -> dict:
    with open(path) as f:
        table = json.load(f)
    if install:
        apply(table)
    return table
