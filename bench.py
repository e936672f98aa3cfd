"""Benchmark: all-pairs binary MI throughput (pairs/s) at the paper scale.

Workload: m = 100,000 samples x n = 10,000 variables, p_j ~ Beta(0.5, 5)
(about 91% zeros, standing in for the paper's 90%-sparse simulated data),
1% of the columns planted as noisy copies of others.  One step = one
mi_all_pairs call through the C ABI (pack to FP4 + column terms + fused
tcgen05 block-scaled FP4 Gram with the MI epilogue), X already resident in
HBM.  The input (1.0 GB) and
the output (0.4 GB) are both larger than L2, so no flush is needed between
steps.  Pairs per step = n(n-1)/2 (distinct unordered pairs; the diagonal is
computed too but not counted).

The JSON line also carries the plain unfused path (Gram -> int32 counts in
HBM -> elementwise MI), the fused path with FP8 operands and the popcount
path on the same input, the roofline
of the dominant kernel, SM clocks sampled during the timed region, an
end-to-end figure through the host-buffer C-ABI call, the FP64 oracle
timed on the host cores on a bounded sample of pairs, the batching workload
(512 uneven datasets in one grouped graph vs separate calls) and the serving
workload (Poisson arrivals at 200 req/s of mixed all-pairs / cross requests
through the native server under a 40 GB budget: p50/p99 latency, a sweep of
offered rates up to saturation, requests whose inputs are uploaded from pinned
host memory, and the capacity of a burst of requests under continuous
batching), the out-of-core
output (n = 50,000 in row panels to host memory), the sparse (CSR) path at
99-99.9% zeros, cross MI between X and a second matrix of the same shape,
and the precision configuration (2^20 samples x 2^14 variables: throughput
and the largest error on sampled pairs against the FP64 oracle).

--impl reference times the FP64 oracle (the only reference this method has:
the paper ships no GPU code) on the host cores, each step a bounded sample of
the same workload's pairs.

Multi-GPU (torchrun): by default every rank runs its own replica of the
workload (weak scaling, no collective on the data path); value = all ranks'
pairs / max time.  --scaling strong splits the one workload instead: rank r
computes shard r of N of the fused Gram's tile list (gbmi_mi_all_pairs_shard,
no collective either); value = the workload's pairs / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PAPER_OPT_T_S = 5.6      # Opt-T (PyTorch, Apple M2 CPU) at 100000 x 10000, Fig. 2 text
METRIC = "MI pairs/s"
UNIT = "pairs/s"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of weakly scaled replicas: all ranks' units / slowest rank's time."""
    return world * units_per_rank / seconds_max


def strong_rate(units_total: float, seconds_max: float) -> float:
    """Whole-job throughput of one problem split over the ranks: its units / slowest time."""
    return units_total / seconds_max


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica: every rank solves its own independent problem."""
    return base + rank


def workload_seed(base: int, rank: int, strong: bool) -> int:
    """Strong scaling splits one problem (the same input on every rank); weak scaling
    gives every rank its own replica."""
    return base if strong else replica_seed(base, rank)


def _workload(m, n):
    return {"workload": f"paper-scale all-pairs MI, m={m} samples x n={n} variables, "
                        "p_j~Beta(0.5,5), 1% planted noisy copies",
            "m": m, "n": n, "pairs_per_step": n * (n - 1) // 2,
            "l2": "inputs larger than L2 (X 1.0 GB, out 0.4 GB per step); no flush",
            "parallelism": "replicas (one independent problem per GPU)"}


POPC_PER_CLK_PER_SM = 16   # 32-bit population counts per clock per SM (integer pipe)
FP4_OVER_BF16 = 6.0        # nominal dense tensor rates: FP4 13.5, BF16 2.25 PFLOP/s


def _fp8_gemm_tflops(dev, size=8192, reps=10):
    """cuBLASLt FP8 E4M3 GEMM rate (torch._scaled_mm, best of `reps`): context only."""
    import torch
    try:
        a = torch.randn(size, size, device=dev).to(torch.float8_e4m3fn)
        b = torch.randn(size, size, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        f = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            f()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1))
        del a, b
        return 2.0 * size ** 3 / (best * 1e-3) / 1e12
    except Exception:
        return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", 0.0)),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "source": "fallback"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons in a background process."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t is not None:
                self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- profile summary
def _source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_19702_gb300", "csrc")
    for f in ("gram_tc.cu", "ptx.cuh", "mi_device.cuh", "internal.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per launch of the fused Gram kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "gram_tc_fused_mi_paper_scale.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None, None
    src = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    tr = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not src or not tr:
        return None, None
    if src.group(1) != _source_digest():
        return None, "stale"
    return float(tr.group(1)), "ncu"


# --------------------------------------------------------------- oracle timing
def _oracle_rate(XT, n, seconds, seed=11, min_pairs=2048):
    """Oracle pairs/s on seeded pairs of the transposed data, about `seconds` of work."""
    import oracle
    import simdata
    pi, pj = simdata.sample_pairs(n, n, min_pairs, seed)
    t0 = time.perf_counter()
    oracle.mi_pairs_t(XT, XT, pi, pj)
    dt = max(time.perf_counter() - t0, 1e-6)
    rate = min_pairs / dt
    k = int(max(min_pairs, rate * seconds))
    pi, pj = simdata.sample_pairs(n, n, k, seed + 1)
    t0 = time.perf_counter()
    oracle.mi_pairs_t(XT, XT, pi, pj)
    dt = time.perf_counter() - t0
    return k / dt, k, dt


def run_reference(args):
    """The FP64 oracle as the reference arm, on the host cores."""
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    if rank != 0:
        return 0
    import oracle
    import simdata
    m, n = args.m, args.n
    X, _ = simdata.make(m, n, simdata.PAPER.seed, "beta", 0.01, 0.05, device="cpu")
    XT = oracle.transpose(X)
    del X
    cores = oracle.max_threads()
    # size each step so the whole run stays within about a minute
    rate, _, _ = _oracle_rate(XT, n, 0.5)
    steps = args.steps + args.warmup
    per_step = int(max(32, min(rate * 60.0 / max(steps, 1), rate * 2.0)))
    total_pairs, total_t = 0, 0.0
    for s in range(steps):
        pi, pj = simdata.sample_pairs(n, n, per_step, 1000 + s)
        t0 = time.perf_counter()
        oracle.mi_pairs_t(XT, XT, pi, pj)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            total_pairs += per_step
            total_t += dt
    value = total_pairs / total_t
    ms_per_step = 1000.0 * total_t / max(args.steps, 1)
    sample = (f"{per_step} seeded pairs of the m={m} x n={n} workload per step "
              f"(each pair walks all {m} samples); transposition of X excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / (n * (n - 1) / 2 / PAPER_OPT_T_S), "dtype": "f64",
            "data": "synthetic", "config": _workload(m, n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- library comparator
def measure_library_plain(X, m, n, fused_out, reps=5):
    """The same two steps on library calls, for context: the transposed FP8 operand by torch
    ops, N11 by cuBLASLt's FP8 GEMM (torch._scaled_mm, FP32 output), then this library's
    elementwise MI kernel on the counts."""
    import torch

    from paper_2411_19702_gb300 import gbmi
    dev = X.device
    try:
        one = torch.ones((), device=dev)

        def step():
            Xt = X.t().contiguous().to(torch.float8_e4m3fn)          # pack: transpose + FP8
            N = torch._scaled_mm(Xt, Xt.t(), scale_a=one, scale_b=one, out_dtype=torch.float32)
            N11 = N.to(torch.int32)
            v = torch.diagonal(N11).contiguous()
            return gbmi.mi_from_counts(N11, v, v, m)
        out = step()
        gbmi.sync()
        rows = torch.arange(0, n, 97, device=dev)
        same = bool(torch.equal(out[rows], fused_out[rows]))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = step()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        del out
        torch.cuda.empty_cache()
        return {"ms_per_step": ms, "value": n * (n - 1) / 2 / (ms * 1e-3),
                "steps": "torch transpose + FP8 cast, cuBLASLt FP8 GEMM (FP32 out), int32 cast, "
                         "elementwise MI kernel (both triangles)",
                "sampled_rows_bit_identical_to_fused": same}
    except Exception as e:  # a torch build without FP8 GEMM on this device
        return {"unavailable": str(e).splitlines()[0][:200]}


# --------------------------------------------------------------- batching
def batch_shapes(k=512, seed=4):
    """Dataset shapes and column densities of the batching workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ms = np.exp(rng.uniform(np.log(500), np.log(200_000), size=k)).round().astype(np.int64)
    ns = np.exp(rng.uniform(np.log(64), np.log(4096), size=k)).round().astype(np.int64)
    ps = [rng.beta(0.5, 5.0, size=int(n)) for n in ns]
    return ms, ns, ps


def measure_batch(dev, reps=3, k=512, seed=4):
    """512 datasets of uneven m and n: one autotuned grouped graph vs separate calls."""
    import torch

    from paper_2411_19702_gb300 import autotune, gbmi
    ms, ns, ps = batch_shapes(k, seed)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    Xs = []
    for m, n, p in zip(ms, ns, ps):
        pt = torch.as_tensor(p, dtype=torch.float32, device=dev)
        Xs.append((torch.rand((int(m), int(n)), generator=g, device=dev) < pt).to(torch.uint8))
    pairs = int(sum(int(n) * (int(n) - 1) // 2 for n in ns))
    t0 = time.perf_counter()
    table = autotune.tune(list(zip(ms.tolist(), ns.tolist())), reps=2)
    # the batch-level choice: rule / per-bucket table / all single / all pairs
    batch_choice = autotune.tune_batch(Xs, table=table, reps=2)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)

    def timed(fn, r):
        fn()
        gbmi.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(r):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        gbmi.sync()
        return e0.elapsed_time(e1) / r

    plan = gbmi.Batch(Xs)
    batch_ms = timed(plan.run, reps)
    l0 = gbmi.launch_count()
    plan.run()
    gbmi.sync()
    launches_per_run = gbmi.launch_count() - l0
    outs = plan.outs
    sep_out = [torch.empty_like(o) for o in outs]

    def separate(path):
        def f():
            for X, o in zip(Xs, sep_out):
                gbmi.mi_all_pairs(X, out=o, path=path)
        return f
    plain_ms = timed(separate("plain"), 1)
    fused_ms = timed(separate("fused"), 1)
    # bit identity of the grouped run with the separate fused calls
    same = all(torch.equal(a, b) for a, b in zip(outs, sep_out))
    res = {"datasets": k, "pairs": pairs,
           "m_range": [int(ms.min()), int(ms.max())], "n_range": [int(ns.min()), int(ns.max())],
           "input_bytes": int(sum(int(m) * int(n) for m, n in zip(ms, ns))),
           "grouped_graph_ms": batch_ms, "grouped_pairs_per_s": pairs / (batch_ms * 1e-3),
           "separate_plain_ms": plain_ms, "separate_fused_ms": fused_ms,
           "speedup_vs_separate_plain": plain_ms / batch_ms,
           "speedup_vs_separate_fused": fused_ms / batch_ms,
           "tiles": plan.tiles, "launches_per_run": launches_per_run,
           "autotuned_buckets": len(table), "autotune_s": tune_s,
           "autotune_choices": {k: {"tile_n": v["tile_n"], "pair": v["pair"],
                                    "split": v.get("split", 0),
                                    "ms": {c: round(t, 4) for c, t in v["ms"].items()},
                                    "ms_split": {c: round(t, 4)
                                                 for c, t in v.get("ms_split", {}).items()}}
                                for k, v in table.items()},
           "autotune_split_buckets": sum(1 for v in table.values() if v.get("split", 0) != 0),
           "autotune_knobs": "per (floor(log2 m), floor(2 log2 n)) bucket: single-CTA tile "
                             "width 64/128/256, single-CTA vs CTA-pair kernel, and (n <= 3000) "
                             "the sample split of single calls (model / none / 2-32 ranges); "
                             "per batch: the kernel assignment (rule / table / all single / "
                             "all pairs)",
           "batch_kernel_choice": batch_choice,
           "bit_identical_to_separate": bool(same)}
    plan.close()
    gbmi.tuner_clear()
    gbmi.set_option(gbmi.OPT_PAIR, 1)
    del Xs, outs, sep_out
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------- out-of-core output
def measure_out_of_core(dev, m=100_000, n=50_000, reps=2, seed=6):
    """All-pairs MI of n = 50,000 variables in row panels into page-locked host memory
    (10 GB of output), against the in-core fused call on the same input."""
    import torch

    from paper_2411_19702_gb300 import gbmi
    rng = np.random.Generator(np.random.PCG64(seed))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    X = _beta_matrix(m, n, g, rng, dev)
    pairs = n * (n - 1) // 2
    host = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    gbmi.mi_all_pairs_to_host(X, out=host)
    t0 = time.perf_counter()
    for _ in range(reps):
        gbmi.mi_all_pairs_to_host(X, out=host)
    ooc_s = (time.perf_counter() - t0) / reps
    dev_out = torch.empty((n, n), dtype=torch.float32, device=dev)
    gbmi.mi_all_pairs(X, out=dev_out, path="fused")
    gbmi.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        gbmi.mi_all_pairs(X, out=dev_out, path="fused")
    e1.record()
    torch.cuda.synchronize(dev)
    in_s = e0.elapsed_time(e1) / reps * 1e-3
    rows = torch.arange(0, n, 997, device=dev)
    same = bool(torch.equal(host[rows.cpu()], dev_out[rows].cpu()))
    res = {"m": m, "n": n, "output_bytes": n * n * 4, "host_memory": "page-locked",
           "to_host_s": ooc_s, "to_host_pairs_per_s": pairs / ooc_s,
           "d2h_gbs": n * n * 4 / ooc_s / 1e9,
           "in_core_device_s": in_s, "in_core_pairs_per_s": pairs / in_s,
           "to_host_over_in_core": ooc_s / in_s,
           "rows_checked_bit_identical": same}
    del X, dev_out, host
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------- the paper's shapes
# Table 1 (samples x variables) and the Fig. 2 shape, with the paper's times on its CPU
# (Opt-T = its PyTorch optimised method; best = its fastest method at that shape).
PAPER_TABLE = [((1000, 100), 0.021, 0.001), ((100_000, 100), 0.061, 0.013),
               ((100_000, 1000), 0.086, 0.086), ((100_000, 10_000), 5.6, 5.6)]
ROW_SWEEP = [(10_000, 1000), (100_000, 1000), (1_000_000, 1000)]       # Fig. 1: rows vary
COL_SWEEP = [(100_000, 1000), (100_000, 2500), (100_000, 5000), (100_000, 10_000),
             (100_000, 20_000)]                                          # Fig. 2: columns vary


def measure_paper_shapes(dev, reps=5, seed=9):
    """mi_all_pairs (automatic path) at the paper's benchmark shapes, inputs resident, each
    with p_j ~ Beta(0.5, 5) columns; the paper's CPU times alongside (context only)."""
    import torch

    import simdata
    from paper_2411_19702_gb300 import gbmi

    def time_shape(m, n):
        X, _ = simdata.make(m, n, seed, "beta", 0.0, 0.05, device=str(dev))
        out = torch.empty((n, n), dtype=torch.float32, device=dev)
        gbmi.mi_all_pairs(X, out=out)
        gbmi.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            gbmi.mi_all_pairs(X, out=out)
        e1.record()
        torch.cuda.synchronize(dev)
        gbmi.sync()
        ms = e0.elapsed_time(e1) / reps
        del X, out
        return ms

    table = []
    for (m, n), opt_t, best in PAPER_TABLE:
        ms = time_shape(m, n)
        table.append({"m": m, "n": n, "ms": ms, "pairs_per_s": n * (n - 1) / 2 / (ms * 1e-3),
                      "paper_opt_t_s": opt_t, "paper_fastest_s": best,
                      "vs_paper_opt_t": opt_t / (ms * 1e-3)})
    rows = [{"m": m, "n": n, "ms": time_shape(m, n)} for m, n in ROW_SWEEP]
    cols = [{"m": m, "n": n, "ms": time_shape(m, n)} for m, n in COL_SWEEP]
    torch.cuda.empty_cache()
    return {"table1_and_fig2": table, "rows_vary_fig1": rows, "columns_vary_fig2": cols,
            "note": "paper times: Apple M2 CPU (Sec. 4.1), context only"}


# --------------------------------------------------------------- cross MI
def measure_cross(dev, X, reps=5, seed=8, check_pairs=256, use_oracle=True):
    """mi_cross between the workload's X and a second seeded matrix Y of the same shape
    (n1 = n2 = n: every one of the n^2 pairs is computed, none mirrored), fused path; the
    parity sample includes the planted (X column, Y column) pairs."""
    import torch

    import simdata
    from paper_2411_19702_gb300 import gbmi
    m, n = X.shape
    Y, _ = simdata.make(m, n, seed, "beta", 0.0, 0.05, device=str(dev))
    # 1% of Y's columns are noisy copies (flip probability 0.05) of seeded columns of X
    rng = np.random.Generator(np.random.PCG64([seed, 3]))
    yc = rng.choice(n, size=max(1, n // 100), replace=False)
    xc = rng.choice(n, size=yc.size, replace=False)
    g = torch.Generator(device=dev)
    g.manual_seed(seed + 1000)
    for a, b in zip(yc.tolist(), xc.tolist()):
        flip = (torch.rand(m, generator=g, device=dev) < 0.05).to(torch.uint8)
        Y[:, a] = X[:, b] ^ flip
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    gbmi.mi_cross(X, Y, out=out, path="fused")
    gbmi.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        gbmi.mi_cross(X, Y, out=out, path="fused")
    e1.record()
    torch.cuda.synchronize(dev)
    gbmi.sync()
    ms = e0.elapsed_time(e1) / reps
    res = {"m": m, "n1": n, "n2": n, "pairs": n * n, "ms_per_step": ms,
           "pairs_per_s": n * n / (ms * 1e-3), "tflops_step": 2.0 * m * n * n / (ms * 1e-3) / 1e12}
    if use_oracle:
        import oracle
        pi, pj = simdata.sample_pairs(n, n, check_pairs, 41, symmetric=False)
        pi, pj = np.concatenate([pi, xc]), np.concatenate([pj, yc])   # with the planted pairs
        a_cols, ia = np.unique(pi, return_inverse=True)
        b_cols, ib = np.unique(pj, return_inverse=True)
        A = X[:, torch.from_numpy(a_cols).to(dev)].cpu().numpy()
        B = Y[:, torch.from_numpy(b_cols).to(dev)].cpu().numpy()
        _, want = oracle.mi_pairs(A, ia, ib, Y=B)
        got = out[torch.from_numpy(pi).to(dev), torch.from_numpy(pj).to(dev)].double().cpu()
        err = float(np.max(np.abs(got.numpy() - want)))
        res["parity"] = {"pairs": int(len(pi)), "max_abs_err_vs_oracle": err,
                         "tolerance": 1e-6, "ok": err <= 1e-6}
    del Y, out
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------- precision configuration
def measure_precision(dev, reps=3, check_cols=448, use_oracle=True):
    """All-pairs MI at 2^20 samples x 2^14 variables (one Gram launch: 2^20 < 2^24),
    p_j ~ U(0.02, 0.5), with FP4 operands (the default) and FP8 operands: throughput,
    tensor rate, whether the two forms agree bit for bit on the whole matrix, and the
    largest |dMI| against the FP64 oracle on every pair among `check_cols` seeded
    columns (448 columns: 100,576 pairs with the diagonal; only those columns are
    copied to the host)."""
    import torch

    import simdata
    from paper_2411_19702_gb300 import gbmi
    r = simdata.PRECISION
    X, _ = simdata.from_recipe(r, device=str(dev))
    m, n = r.m, r.n
    pairs = n * (n - 1) // 2
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None

    def run(fp4):
        gbmi.set_option(gbmi.OPT_FP4, 1 if fp4 else 0)
        try:
            out = torch.empty((n, n), dtype=torch.float32, device=dev)
            gbmi.mi_all_pairs(X, out=out, path="fused")
            gbmi.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(uuid) as clocks:
                e0.record()
                for _ in range(reps):
                    gbmi.mi_all_pairs(X, out=out, path="fused")
                e1.record()
                torch.cuda.synchronize(dev)
            gbmi.sync()
        finally:
            gbmi.set_option(gbmi.OPT_FP4, 1)
        ms = e0.elapsed_time(e1) / reps
        return out, {"ms_per_step": ms, "clocks": clocks.summary(),
                     "pairs_per_s": pairs / (ms * 1e-3),
                     "tflops_step": float(m) * n * n / (ms * 1e-3) / 1e12}

    out4, fp4 = run(True)
    out8, fp8 = run(False)
    same = bool(torch.equal(out4, out8))
    res = dict(m=m, n=n, dist="p_j ~ U(0.02, 0.5), iid Bernoulli", **fp4)
    res["fp8_operands"] = fp8
    res["fp4_fp8_whole_matrix_bit_identical"] = same
    if use_oracle:
        import oracle
        cols = np.sort(np.random.Generator(np.random.PCG64([r.seed, 17])).choice(
            n, check_cols, replace=False)).astype(np.int64)
        sub = X[:, torch.from_numpy(cols).to(dev)].cpu().numpy()
        iu, ju = np.triu_indices(len(cols))
        t0 = time.perf_counter()
        _, want = oracle.mi_pairs(sub, iu.astype(np.int64), ju.astype(np.int64))
        oracle_s = time.perf_counter() - t0
        ti, tj = torch.from_numpy(cols[iu]).to(dev), torch.from_numpy(cols[ju]).to(dev)
        got = out4[ti, tj].double().cpu().numpy()
        err = float(np.max(np.abs(got - want)))
        err8 = float(np.max(np.abs(out8[ti, tj].double().cpu().numpy() - want)))
        res["parity"] = {"pairs": int(len(iu)), "columns": int(len(cols)),
                         "max_abs_err_vs_oracle": err, "tolerance": 1e-6,
                         "fp8_max_abs_err_vs_oracle": err8,
                         "ok": err <= 1e-6 and err8 <= 1e-6,
                         "oracle_s": oracle_s, "oracle_threads": oracle.max_threads()}
    del X, out4, out8
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------- sparse input
def measure_sparse(dev, m=100_000, n=10_000, densities=(0.01, 0.005, 0.001), reps=3, seed=7):
    """Paper-shape inputs at 99%, 99.5% and 99.9% zeros (iid Bernoulli): the CSR call
    (inputs resident in CSR) with pair enumeration forced and with the cost model's choice,
    against the dense fused path on the same matrix."""
    import torch

    from paper_2411_19702_gb300 import gbmi
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    res = []
    for d in densities:
        X = (torch.rand((m, n), generator=g, device=dev) < d).to(torch.uint8)
        rp, ci = gbmi.csr_from_dense(X)
        torch.cuda.synchronize(dev)

        def timed(fn):
            fn()
            gbmi.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize(dev)
            gbmi.sync()
            return e0.elapsed_time(e1) / reps
        gbmi.set_option(gbmi.OPT_CSR_PATH, 1)       # pair enumeration, forced
        sparse_ms = timed(lambda: gbmi.mi_all_pairs_csr(rp, ci, n, out=out))
        sparse_out = out.clone()
        gbmi.set_option(gbmi.OPT_CSR_PATH, 0)       # the cost model's choice (default)
        gbmi.profile(enable=True, reset=True)
        gbmi.mi_all_pairs_csr(rp, ci, n, out=out)
        choice = "dense" if "csr_densify" in gbmi.profile(enable=False) else "enumerate"
        auto_ms = timed(lambda: gbmi.mi_all_pairs_csr(rp, ci, n, out=out))
        auto_same = bool(torch.equal(out, sparse_out))
        dense_ms = timed(lambda: gbmi.mi_all_pairs(X, out=out, path="fused"))
        rows = torch.arange(0, n, 211, device=dev)
        diff = float((sparse_out[rows] - out[rows]).abs().max())
        res.append({"zeros_pct": 100.0 * (1.0 - d), "nnz": int(ci.numel()),
                    "pair_increments": int(((rp[1:] - rp[:-1]) * (rp[1:] - rp[:-1] + 1) // 2)
                                           .sum()),
                    "csr_ms": sparse_ms, "dense_fused_ms": dense_ms,
                    "csr_over_dense_speedup": dense_ms / sparse_ms,
                    "csr_auto_ms": auto_ms, "csr_auto_form": choice,
                    "csr_auto_bit_identical": auto_same,
                    "max_abs_diff_sampled_rows": diff})
        del X, rp, ci, sparse_out
        torch.cuda.empty_cache()
    return {"m": m, "n": n, "densities": res}


# --------------------------------------------------------------- serving
def serve_pool(k_all=48, k_cross=24, seed=5):
    """Dataset shapes of the serving workload's pool: all-pairs (m, n) and cross (m, n1, n2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lu = lambda lo, hi, k: np.exp(rng.uniform(np.log(lo), np.log(hi), size=k)).round().astype(int)
    alls = list(zip(lu(1_000, 500_000, k_all), lu(100, 8_000, k_all)))
    cross = list(zip(lu(1_000, 500_000, k_cross), lu(100, 4_000, k_cross), lu(100, 4_000, k_cross)))
    return alls, cross


def _beta_matrix(m, n, g, rng, dev):
    import torch
    p = torch.as_tensor(rng.beta(0.5, 5.0, size=n), dtype=torch.float32, device=dev)
    X = torch.empty((m, n), dtype=torch.uint8, device=dev)
    rows = max(1, (1 << 28) // n)
    for r in range(0, m, rows):
        X[r:r + rows] = (torch.rand((min(rows, m - r), n), generator=g, device=dev) < p)
    return X


def measure_serving(dev, seconds=60.0, rate=200.0, budget=40 << 30, seed=5, burst=400, check=20,
                    sweep_rates=(1000.0, 3000.0, 6000.0), sweep_seconds=5.0, host_seconds=10.0):
    """Poisson arrivals of mixed all-pairs / cross requests through the native server.

    Each request registers its dataset(s) from a pool of resident inputs
    (so the server packs them for that request), submits, and removes them
    (dropped once the request is done); a collector waits for the tickets in
    order and releases the outputs.  Latency is submit -> completion, timed
    inside the server, and arrival -> result, timed by the client.  After the
    main window: shorter windows at higher offered rates (the sweep), and one
    at the main rate whose requests upload their inputs from pinned host
    memory before registering them.
    """
    import torch

    from paper_2411_19702_gb300 import gbmi
    alls, cross = serve_pool(seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    pool_all = [_beta_matrix(int(m), int(n), g, rng, dev) for m, n in alls]
    pool_cross = [(_beta_matrix(int(m), int(a), g, rng, dev), _beta_matrix(int(m), int(b), g, rng, dev))
                  for m, a, b in cross]
    torch.cuda.synchronize(dev)

    upload_stream = torch.cuda.Stream(dev)

    def run(srv, arrivals, picks, keep=0, host=None):
        # host: pinned host copies of the pool (index -> tensors); each request
        # then uploads its input(s) before registering them
        tickets, kept, errors, client_ms = [], [], [], []
        done = threading.Event()

        def collector():
            k = 0
            try:
                while k < len(arrivals):
                    while k >= len(tickets):
                        if done.is_set() and k >= len(tickets):
                            return
                        time.sleep(0.0002)
                    t, req, t_arr = tickets[k]
                    out, _ = srv.wait(t, timeout_ms=120_000)
                    client_ms.append((time.perf_counter() - t_arr) * 1e3)
                    if k < keep:
                        kept.append((req, out.clone()))
                    srv.release(t)
                    k += 1
            except Exception as e:  # reported by the caller
                errors.append(e)

        def upload(Xh):
            with torch.cuda.stream(upload_stream):
                Xd = Xh.to(dev, non_blocking=True)
            upload_stream.synchronize()
            return Xd

        th = threading.Thread(target=collector)
        th.start()
        t0 = time.perf_counter()
        try:
            for at, req in zip(arrivals, picks):
                d = t0 + at - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                t_arr = time.perf_counter()
                kind, j = req
                if kind == "all":
                    Xa = upload(host[0][j]) if host else pool_all[j]
                    a = srv.add_dataset(Xa)
                    t = srv.submit(a)
                    srv.remove_dataset(a)
                else:
                    Xa, Xb = (upload(host[1][j][0]), upload(host[1][j][1])) if host \
                        else pool_cross[j]
                    a = srv.add_dataset(Xa)
                    b = srv.add_dataset(Xb)
                    t = srv.submit(a, b)
                    srv.remove_dataset(a)
                    srv.remove_dataset(b)
                tickets.append((t, req, t_arr))
        finally:
            done.set()
            th.join()
        wall = time.perf_counter() - t0
        if errors:
            raise errors[0]
        return wall, kept, client_ms

    def pairs_of(req):
        kind, j = req
        if kind == "all":
            n = int(alls[j][1])
            return n * (n - 1) // 2
        return int(cross[j][1]) * int(cross[j][2])

    def picks_for(k, r):
        out = []
        for _ in range(k):
            if r.random() < 0.5:
                out.append(("all", int(r.integers(len(alls)))))
            else:
                out.append(("cross", int(r.integers(len(cross)))))
        return out

    # open loop: Poisson arrivals at `rate` for `seconds`
    r = np.random.Generator(np.random.PCG64(seed + 2))
    gaps = r.exponential(1.0 / rate, size=int(rate * seconds * 1.5) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < seconds]
    picks = picks_for(len(arrivals), r)
    with gbmi.Server(budget, max_batch=64, device=dev) as srv:
        wall, kept, cms = run(srv, arrivals, picks, keep=check)
        st = srv.stats()
    same = True
    for (kind, j), got in kept:
        want = (gbmi.mi_all_pairs(pool_all[j], path="fused") if kind == "all"
                else gbmi.mi_cross(pool_cross[j][0], pool_cross[j][1], path="fused"))
        gbmi.sync()
        same = same and bool(torch.equal(got, want))
    pairs = sum(pairs_of(q) for q in picks)
    poisson = {"requests": len(arrivals), "offered_req_per_s": rate, "seconds": seconds,
               "wall_s": wall, "pairs": pairs, "pairs_per_s_offered_window": pairs / wall,
               "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
               "max_ms": st["max_ms"], "completed": int(st["completed"]),
               "batches": int(st["batches"]), "requests_per_batch": st["requests_per_batch"],
               "bit_identical_to_single_calls": f"{len(kept)} of {len(kept)} checked" if same
               else "MISMATCH",
               "client_p50_ms": float(np.percentile(cms, 50)) if cms else None,
               "client_p99_ms": float(np.percentile(cms, 99)) if cms else None}

    # offered-rate sweep: shorter windows at rates up to saturation
    sweep = []
    for srate in sweep_rates:
        sr = np.random.Generator(np.random.PCG64(seed + 10 + int(srate)))
        sa = np.cumsum(sr.exponential(1.0 / srate, size=int(srate * sweep_seconds * 1.5) + 16))
        sa = sa[sa < sweep_seconds]
        sp = picks_for(len(sa), sr)
        with gbmi.Server(budget, max_batch=64, device=dev) as srv:
            sw, skept, scms = run(srv, sa, sp, keep=check)
            sst = srv.stats()
        ssame = True
        for (kind, j), got in skept:
            want = (gbmi.mi_all_pairs(pool_all[j], path="fused") if kind == "all"
                    else gbmi.mi_cross(pool_cross[j][0], pool_cross[j][1], path="fused"))
            gbmi.sync()
            ssame = ssame and bool(torch.equal(got, want))
        sweep.append({"offered_req_per_s": srate, "seconds": sweep_seconds,
                      "requests": len(sa), "completed_req_per_s": len(sa) / sw,
                      "pairs_per_s": sum(pairs_of(q) for q in sp) / sw,
                      "p50_ms": sst["p50_ms"], "p99_ms": sst["p99_ms"],
                      "client_p50_ms": float(np.percentile(scms, 50)) if scms else None,
                      "client_p99_ms": float(np.percentile(scms, 99)) if scms else None,
                      "batches": int(sst["batches"]),
                      "requests_per_batch": sst["requests_per_batch"],
                      "bit_identical_to_single_calls": ssame})

    # requests whose inputs come from pinned host memory: each is uploaded (its own
    # copy stream) and registered on arrival, so the latency includes the upload
    host_all = [X.cpu().pin_memory() for X in pool_all]
    host_cross = [(A.cpu().pin_memory(), B.cpu().pin_memory()) for A, B in pool_cross]
    hr = np.random.Generator(np.random.PCG64(seed + 3))
    ha = np.cumsum(hr.exponential(1.0 / rate, size=int(rate * host_seconds * 1.5) + 16))
    ha = ha[ha < host_seconds]
    hp = picks_for(len(ha), hr)
    with gbmi.Server(budget, max_batch=64, device=dev) as srv:
        hw, hkept, hcms = run(srv, ha, hp, keep=check, host=(host_all, host_cross))
        hst = srv.stats()
    hsame = True
    for (kind, j), got in hkept:
        want = (gbmi.mi_all_pairs(pool_all[j], path="fused") if kind == "all"
                else gbmi.mi_cross(pool_cross[j][0], pool_cross[j][1], path="fused"))
        gbmi.sync()
        hsame = hsame and bool(torch.equal(got, want))
    host_upload = {"offered_req_per_s": rate, "seconds": host_seconds, "requests": len(ha),
                   "upload": "pinned host -> device copy per request (its own stream), then "
                             "registration and submit",
                   "h2d_bytes": int(sum(pool_all[j].numel() if k == "all" else
                                        pool_cross[j][0].numel() + pool_cross[j][1].numel()
                                        for k, j in hp)),
                   "client_p50_ms": float(np.percentile(hcms, 50)) if hcms else None,
                   "client_p99_ms": float(np.percentile(hcms, 99)) if hcms else None,
                   "server_p50_ms": hst["p50_ms"], "server_p99_ms": hst["p99_ms"],
                   "bit_identical_to_single_calls": hsame}
    del host_all, host_cross
    # closed loop: `burst` requests submitted at once (capacity under continuous batching)
    bpicks = picks_for(burst, r)
    with gbmi.Server(budget, max_batch=64, device=dev) as srv:
        bwall, _, _ = run(srv, np.zeros(burst), bpicks)
        bst = srv.stats()
    bpairs = sum(pairs_of(q) for q in bpicks)
    res = {"budget_bytes": budget, "mix": "50% all-pairs m in [1e3,5e5] n in [100,8000], "
           "50% cross n1,n2 in [100,4000], log-uniform; pool of "
           f"{len(alls)} + {len(cross)} resident inputs, densities Beta(0.5,5)",
           "poisson": poisson, "sweep": sweep, "host_upload": host_upload,
           "latency_note": "p50/p99 are the server's submit -> completion times; client_* "
                           "are arrival -> result in hand, measured by the client",
           "burst": {"requests": burst, "wall_s": bwall, "req_per_s": burst / bwall,
                     "pairs_per_s": bpairs / bwall, "p50_ms": bst["p50_ms"],
                     "p99_ms": bst["p99_ms"], "batches": int(bst["batches"]),
                     "requests_per_batch": bst["requests_per_batch"]}}
    del pool_all, pool_cross
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    import simdata
    from paper_2411_19702_gb300 import gbmi

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    gbmi.load()
    m, n = args.m, args.n
    pairs = n * (n - 1) // 2

    def barrier():
        if dist is not None:
            dist.barrier()

    def reduce_max(x):
        return max_over_ranks(x, dist, dev)

    strong = args.scaling == "strong"
    seed = workload_seed(simdata.PAPER.seed, rank, strong)
    X, info = simdata.make(m, n, seed, "beta", 0.01, 0.05, device=str(dev))
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(path="fused"):
        if strong and world > 1 and path == "fused":
            gbmi.mi_all_pairs_shard(X, rank, world, out=out)
        else:
            gbmi.mi_all_pairs(X, out=out, path=path)

    def job_rate(ms):   # whole-job pairs/s from the slowest rank's time per step
        return strong_rate(pairs, ms * 1e-3) if strong else whole_job_rate(pairs, world, ms * 1e-3)

    def timed(path, steps, warmup, sample_clocks=False, profile=False):
        for _ in range(warmup):
            step(path)
        gbmi.sync()
        barrier()
        torch.cuda.synchronize(dev)
        if profile:
            gbmi.profile(enable=True, reset=True)
        launches0 = gbmi.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(dev).uuid)
            if uuid and not uuid.startswith("GPU-"):
                uuid = "GPU-" + uuid
        except Exception:
            uuid = None
        sampler = ClockSampler(uuid) if sample_clocks else None
        if sampler:
            sampler.__enter__()
            time.sleep(0.3)
        e0.record(stream)
        for _ in range(steps):
            step(path)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.__exit__(None, None, None)
        gbmi.sync()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        prof = gbmi.profile(enable=False) if profile else None
        return {"ms": ms, "launches": gbmi.launch_count() - launches0,
                "clocks": sampler.summary() if sampler else None, "profile": prof}

    # correctness gate on this input before timing: sampled pairs vs the oracle
    parity = None
    XT = None
    if rank == 0 and not args.skip_oracle:
        import oracle
        gbmi.mi_all_pairs(X, out=out, path="fused")   # the whole matrix, also when sharded
        gbmi.sync()
        XT = oracle.transpose(X.cpu().numpy())
        pi, pj = simdata.sample_pairs(n, n, 2000, 99)
        tg, sr = info["planted_targets"], info["planted_sources"]
        pi = np.concatenate([pi, np.minimum(tg, sr)])
        pj = np.concatenate([pj, np.maximum(tg, sr)])
        _, want = oracle.mi_pairs_t(XT, XT, pi, pj)
        got = out[torch.from_numpy(pi).to(dev), torch.from_numpy(pj).to(dev)].double().cpu()
        err = float(np.max(np.abs(got.numpy() - want)))
        parity = {"pairs": int(len(pi)), "max_abs_err_vs_oracle": err, "tolerance": 1e-6,
                  "ok": err <= 1e-6}

    fused = timed("fused", args.steps, args.warmup, sample_clocks=True, profile=False)
    fused_ms = reduce_max(fused["ms"])
    # the same loop again with the event profiler on: per-kernel device times
    prof = timed("fused", max(3, min(args.steps, 20)), 1, profile=True)["profile"]
    plain = timed("plain", max(3, min(args.steps, 20)), 2, profile=True)
    popc_steps = max(1, min(args.steps, 3))
    popc = timed("popcount", popc_steps, 1)
    # the fused path with the FP64 combine switched to its non-default setting
    fix_default = 0
    gbmi.set_option(gbmi.OPT_FIXUP, 1 - fix_default)
    try:
        alt = timed("fused", max(3, min(args.steps, 20)), 2, profile=True)
        alt_plain = timed("plain", max(3, min(args.steps, 20)), 2, profile=True)
    finally:
        gbmi.set_option(gbmi.OPT_FIXUP, fix_default)
    # the fused path with FP8 operands (the FP4 form is the default)
    gbmi.set_option(gbmi.OPT_FP4, 0)
    try:
        fp8 = timed("fused", max(3, min(args.steps, 20)), 2, profile=True)
    finally:
        gbmi.set_option(gbmi.OPT_FP4, 1)

    # roofline of the dominant kernel (tensor-bound): m*n^2/2 MACs = m*n^2 flops per launch
    peaks = _peaks()
    # the measured tensor-core rate of the Gram's own MMA forms (shared-memory operands,
    # no global traffic): FP4 256 x 240 x 64 and FP8 256 x 256 x 32 on CTA pairs
    probe4 = max(gbmi.mma_peak(1, 1, 240, 1 << 15)["flops_per_s"] for _ in range(3)) / 1e12
    probe8 = max(gbmi.mma_peak(0, 1, 256, 1 << 14)["flops_per_s"] for _ in range(3)) / 1e12
    gram = prof.get("gram_tc_fused_mi", {"ms": float("nan"), "launches": 1})
    gram_ms = gram["ms"] / max(gram["launches"], 1)
    flops = float(m) * n * n / (world if strong else 1)   # a shard's launch does its share
    achieved = flops / (gram_ms * 1e-3) / 1e12
    # FP4 contraction: 6 x measured BF16 (nominal dense ratio 13.5 / 2.25 PFLOP/s)
    peak = FP4_OVER_BF16 * peaks["bf16_tflops"]
    traffic, tsrc = _profiled_traffic()
    cublas_fp8 = _fp8_gemm_tflops(dev)
    # popcount path: ALU-bound on the population-count rate, one POPC per 32-bit word pair
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = (fused["clocks"] or {}).get("sm_mhz") or peaks["sm_max_mhz"]
    words = (m + 31) // 32
    popc_rate = pairs * words / (popc["ms"] * 1e-3)
    popc_peak = sm_count * POPC_PER_CLK_PER_SM * clk_mhz * 1e6
    g8 = (fp8["profile"] or {}).get("gram_tc_fused_mi")
    fp8_tf = flops / (g8["ms"] / max(g8["launches"], 1) * 1e-3) / 1e12 if g8 else None
    step_total = sum(v["ms"] for v in prof.values())
    kernels = {k: {"ms_per_launch": v["ms"] / max(v["launches"], 1),
                   "launches": v["launches"],
                   "share": v["ms"] / step_total if step_total > 0 else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    library = None
    if rank == 0 and not args.skip_library:
        step("fused")
        gbmi.sync()
        library = measure_library_plain(X, m, n, out)

    # end to end through the host-buffer C-ABI call (pinned buffers)
    e2e = None
    if strong and world > 1:
        e2e = {"unavailable": "strong scaling: the host-buffer call is not sharded"}
    elif not args.skip_e2e:
        Xh = X.cpu().pin_memory()
        outh = torch.empty((n, n), dtype=torch.float32).pin_memory()
        gbmi.mi_all_pairs_host(Xh, outh)
        e2e_steps = max(2, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            gbmi.mi_all_pairs_host(Xh, outh)
        dt = reduce_max((time.perf_counter() - t0) / e2e_steps)
        e2e = {"value": whole_job_rate(pairs, world, dt), "unit": UNIT, "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": int(m) * n, "d2h_bytes_per_step": int(n) * n * 4}

    # FP64 oracle on the host cores, bounded sample (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.skip_oracle:
        import oracle
        rate, k, dt = _oracle_rate(XT, n, args.oracle_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"{k} seeded pairs of this workload in {dt:.1f} s (each pair walks all "
                         f"{m} samples; FP64, OpenMP over pairs); transposition of X excluded"}

    batch = None
    if not args.skip_batch:
        batch = measure_batch(dev)
    paper_shapes = None
    if not args.skip_paper_shapes and rank == 0:
        paper_shapes = measure_paper_shapes(dev)
    cross = None
    if not args.skip_cross and rank == 0:
        cross = measure_cross(dev, X, use_oracle=not args.skip_oracle)
    precision = None
    if not args.skip_precision and rank == 0:
        precision = measure_precision(dev, use_oracle=not args.skip_oracle)
    sparse = None
    if not args.skip_sparse and rank == 0:
        sparse = measure_sparse(dev)
    out_of_core = None
    if not args.skip_ooc and rank == 0:
        out_of_core = measure_out_of_core(dev)
    serving = None
    if not args.skip_serve and rank == 0:
        serving = measure_serving(dev, seconds=args.serve_seconds)

    value = job_rate(fused_ms)
    plain_ms = reduce_max(plain["ms"])
    popc_ms = reduce_max(popc["ms"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": fused_ms,
        "higher_is_better": True, "scaling": args.scaling,
        "vs_baseline": value / (pairs / PAPER_OPT_T_S),
        "dtype": "e2m1", "data": "synthetic",
        "config": dict(_workload(m, n), path="fused",
                       arithmetic="FP4 E2M1 0/1 operands (block-scaled tcgen05 MMA, every "
                                  "scale factor 1.0), FP32 tensor-core accumulation (exact "
                                  "counts), FP32 epilogue"),
        "plain": {"value": job_rate(plain_ms), "ms_per_step": plain_ms,
                  "path": "tcgen05 Gram -> int32 N11 in HBM -> elementwise MI kernel",
                  "kernels": {k: v["ms"] / max(v["launches"], 1)
                              for k, v in (plain["profile"] or {}).items()}},
        "fixup_toggled": {"fp64_combine": bool(1 - fix_default),
                          "value": job_rate(reduce_max(alt["ms"])),
                          "ms_per_step": reduce_max(alt["ms"]),
                          "over_default": reduce_max(alt["ms"]) / fused_ms,
                          "kernels": {k: v["ms"] / max(v["launches"], 1)
                                      for k, v in (alt["profile"] or {}).items()},
                          "plain": {"value": job_rate(reduce_max(alt_plain["ms"])),
                                    "ms_per_step": reduce_max(alt_plain["ms"]),
                                    "kernels": {k: v["ms"] / max(v["launches"], 1)
                                                for k, v in (alt_plain["profile"] or {}).items()}},
                          "fused_over_plain": reduce_max(alt_plain["ms"]) /
                                              reduce_max(alt["ms"])},
        "fp8_operands": {"value": job_rate(reduce_max(fp8["ms"])),
                         "ms_per_step": reduce_max(fp8["ms"]),
                         "gram_tflops": fp8_tf, "peak_probe": probe8,
                         "frac_of_probe": fp8_tf / probe8 if fp8_tf else None,
                         "frac_of_bf16x2": fp8_tf / (2.0 * peaks["bf16_tflops"]) if fp8_tf
                         else None,
                         "arithmetic": "FP8 E4M3 0/1 operands, kind::f8f6f4 MMA, 256 x 256 "
                                       "pair tiles",
                         "kernels": {k: v["ms"] / max(v["launches"], 1)
                                     for k, v in (fp8["profile"] or {}).items()}},
        "popcount": {"value": job_rate(popc_ms), "ms_per_step": popc_ms,
                     "roofline": {"bound": "alu", "achieved": popc_rate / 1e12,
                                  "peak": popc_peak / 1e12, "unit": "Tpopc/s",
                                  "frac": popc_rate / popc_peak,
                                  "peak_source": f"{sm_count} SMs x {POPC_PER_CLK_PER_SM} POPC/clk "
                                                 f"x {clk_mhz:.0f} MHz (median SM clock)",
                                  "words_per_pair": words}},
        "fused_over_plain": plain_ms / fused_ms,
        "library_plain": library,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "gram_tc_fused_mi",
                     "peak_source": f"{peaks['source']} bf16 burst x {FP4_OVER_BF16:g} "
                                    "(FP4/BF16 nominal dense ratio)",
                     "flops_per_launch": flops, "ms_per_launch": gram_ms,
                     "peak_probe": probe4, "frac_of_probe": achieved / probe4,
                     "probe_source": "gbmi_mma_peak: tcgen05.mma kind::mxf4 256 x 240 x 64 on "
                                     "CTA pairs, operands resident in shared memory, every SM, "
                                     "best of 3 (this run)",
                     "context_cublas_fp8_tflops": cublas_fp8,
                     "achieved_over_cublas_fp8": achieved / cublas_fp8 if cublas_fp8 else None,
                     "traffic_source": tsrc},
        "kernels": kernels,
        "clocks": fused["clocks"],
        "gpu_launches": int(fused["launches"]),
        "parity": parity,
        "batch": batch,
        "serving": serving,
        "out_of_core": out_of_core,
        "sparse": sparse,
        "cross": cross,
        "paper_shapes": paper_shapes,
        "precision_config": precision,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m", type=int, default=100_000)
    ap.add_argument("--n", type=int, default=10_000)
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    ap.add_argument("--skip-oracle", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-ooc", action="store_true")
    ap.add_argument("--skip-sparse", action="store_true")
    ap.add_argument("--skip-library", action="store_true")
    ap.add_argument("--skip-precision", action="store_true")
    ap.add_argument("--skip-cross", action="store_true")
    ap.add_argument("--skip-paper-shapes", action="store_true")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
