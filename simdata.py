"""Seeded synthetic binary datasets (samples x variables, uint8 0/1).

The paper's experiments use simulated binary matrices of fixed sparsity
(about 90% zeros, Sec. 4.2.1 and Sec. 4.2.3) whose generator it does not
describe.  These generators stand in for them.  This module holds no part of
the mutual-information arithmetic; it only draws inputs, and it is the one
module both the CUDA path's tests and the oracle read.

Recipes (m = samples, n = variables; every column j is iid Bernoulli(p_j)):
  tiny        m=1,000     n=200     p_j ~ Uniform(0.02, 0.5)
  paper       m=100,000   n=10,000  p_j ~ Beta(0.5, 5) (mean density 1/11, ~91% zeros);
                                   1% of the columns are replaced by a copy of another
                                   column with every bit flipped with probability 0.05
  precision   m=1,048,576 n=16,384  p_j ~ Uniform(0.02, 0.5)
The per-column probabilities and the planted-column choice come from numpy's
PCG64 seeded with the config's seed; the bits come from numpy (device='cpu')
or from a seeded torch CUDA generator (device='cuda', for the large inputs).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Recipe:
    name: str
    m: int
    n: int
    dist: str              # "uniform" -> U(0.02, 0.5); "beta" -> Beta(0.5, 5)
    planted_frac: float    # fraction of columns replaced by noisy copies of others
    flip: float            # flip probability of a planted copy
    seed: int


TINY = Recipe("tiny", 1000, 200, "uniform", 0.0, 0.05, 1)
PAPER = Recipe("paper", 100_000, 10_000, "beta", 0.01, 0.05, 2)
PRECISION = Recipe("precision", 1 << 20, 1 << 14, "uniform", 0.0, 0.05, 3)
RECIPES = {r.name: r for r in (TINY, PAPER, PRECISION)}


def column_probabilities(n: int, dist: str, rng: np.random.Generator) -> np.ndarray:
    """Per-column Bernoulli probabilities p_j."""
    if dist == "uniform":
        return rng.uniform(0.02, 0.5, size=n)
    if dist == "beta":
        return rng.beta(0.5, 5.0, size=n)
    raise ValueError(f"unknown column distribution {dist!r}")


def planted_pairs(n: int, frac: float, rng: np.random.Generator):
    """(targets, sources): target column t becomes a noisy copy of source column s."""
    k = int(round(frac * n))
    if k == 0 or n < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    perm = rng.permutation(n)
    tgt = np.sort(perm[:k]).astype(np.int64)
    pool = perm[k:]
    src = rng.choice(pool, size=k, replace=True).astype(np.int64)
    return tgt, src


def make(m: int, n: int, seed: int, dist: str = "uniform", planted_frac: float = 0.0,
         flip: float = 0.05, device: str = "cpu", row_chunk: int = 8192):
    """Draw an m x n binary matrix.

    Returns (X, info) where X is a numpy uint8 array (device='cpu') or a torch
    uint8 CUDA tensor (device='cuda'), and info holds p, the planted pairs and
    the seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = column_probabilities(n, dist, rng)
    tgt, src = planted_pairs(n, planted_frac, rng)
    info = {"p": p, "planted_targets": tgt, "planted_sources": src, "seed": seed,
            "dist": dist, "flip": flip}
    if device == "cpu":
        bits_rng = np.random.Generator(np.random.PCG64([seed, 1]))
        X = np.empty((m, n), dtype=np.uint8)
        p32 = p.astype(np.float32)
        for r0 in range(0, m, row_chunk):
            r1 = min(m, r0 + row_chunk)
            X[r0:r1] = bits_rng.random((r1 - r0, n), dtype=np.float32) < p32
        if tgt.size:
            noise = bits_rng.random((m, tgt.size), dtype=np.float32) < np.float32(flip)
            X[:, tgt] = X[:, src] ^ noise.astype(np.uint8)
        return X, info
    import torch
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    X = torch.empty((m, n), dtype=torch.uint8, device=dev)
    pt = torch.as_tensor(p, dtype=torch.float32, device=dev)
    for r0 in range(0, m, row_chunk):
        r1 = min(m, r0 + row_chunk)
        u = torch.rand((r1 - r0, n), generator=g, device=dev, dtype=torch.float32)
        X[r0:r1] = (u < pt).to(torch.uint8)
        del u
    if tgt.size:
        tg = torch.as_tensor(tgt, device=dev)
        sr = torch.as_tensor(src, device=dev)
        noise = (torch.rand((m, tgt.size), generator=g, device=dev) < flip).to(torch.uint8)
        X[:, tg] = X[:, sr] ^ noise
    return X, info


def from_recipe(recipe: Recipe | str, device: str = "cpu", m: int | None = None,
                n: int | None = None):
    """Draw a dataset from a named recipe (optionally overriding its sizes)."""
    r = RECIPES[recipe] if isinstance(recipe, str) else recipe
    return make(m or r.m, n or r.n, r.seed, r.dist, r.planted_frac, r.flip, device)


def sample_pairs(n1: int, n2: int, k: int, seed: int, symmetric: bool = True):
    """k seeded (i, j) index pairs; with symmetric=True they satisfy i <= j."""
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    i = rng.integers(0, n1, size=k, dtype=np.int64)
    j = rng.integers(0, n2, size=k, dtype=np.int64)
    if symmetric:
        i, j = np.minimum(i, j), np.maximum(i, j)
    return i, j
