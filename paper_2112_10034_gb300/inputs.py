"""Seeded synthetic inputs for the warp-collective workloads.

This module serves both the CUDA path and the CPU oracle (tests, bench,
smoke).  It holds random draws only -- none of the arithmetic of the ops
themselves -- so that neither side has to import the other.

Workload shapes follow the paper's warp-function workloads: the reduction of
Code 1 (Section 2.3) over int32 values, the shuffle scan kernel of the SDK
(Table 1, ``shfl_scan_test``) over N(0,1) floats, the vote/filter kernels
(Table 1, ``VoteAny``/``filter_arr``) over uniform keys, and match-based
histograms over Zipf-distributed keys.  The paper ships none of its inputs,
so every generator here is a stand-in whose distribution is stated.
"""
from __future__ import annotations

import math

import numpy as np

# Base seed of every workload; workload k draws from BASE_SEED + k.
BASE_SEED = 2112100340


def rng(seed: int) -> np.random.Generator:
    """A PCG64 generator for ``seed`` (numpy's published default bit generator)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_int32(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``n`` int32 values uniform on the closed range [lo, hi]."""
    return rng(seed).integers(lo, hi, size=int(n), endpoint=True, dtype=np.int32)


def uniform_u31(n: int, seed: int) -> np.ndarray:
    """``n`` int32 keys uniform on [0, 2^31)."""
    return rng(seed).integers(0, 2**31, size=int(n), dtype=np.int32)


def normal_f32(n: int, seed: int) -> np.ndarray:
    """``n`` float32 values drawn from N(0, 1)."""
    return rng(seed).standard_normal(int(n), dtype=np.float32)


def bits_u32(n: int, seed: int) -> np.ndarray:
    """``n`` uint32 words with every bit pattern equally likely."""
    return rng(seed).integers(0, 2**32, size=int(n), dtype=np.uint32)


def zipf_keys(n: int, seed: int, bins: int = 256, s: float = 1.1) -> np.ndarray:
    """``n`` int32 keys in [0, bins) with P(key = k-1) proportional to k^-s.

    Finite-support Zipf over ranks 1..bins, sampled by inverse CDF; rank k maps
    to key k-1 (so key 0 is the hottest bin, p ~ 0.2065 for s = 1.1, bins = 256).
    """
    ranks = np.arange(1, bins + 1, dtype=np.float64)
    w = ranks ** (-s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    u = rng(seed).random(int(n))
    return np.searchsorted(cdf, u, side="right").astype(np.int32)


def loguniform_lengths(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` int64 lengths L = floor(exp(U[ln lo, ln hi])) clamped to [lo, hi]."""
    u = rng(seed).uniform(math.log(lo), math.log(hi), size=int(count))
    return np.clip(np.floor(np.exp(u)), lo, hi).astype(np.int64)


def density_threshold(d: float) -> int:
    """Threshold t with P(key < t) = d for keys uniform on [0, 2^31): floor(d * 2^31)."""
    return int(math.floor(d * 2**31))


def poisson_arrivals(count: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    gaps = rng(seed).exponential(1.0 / float(rate_hz), size=int(count))
    return np.cumsum(gaps)


def choice(count: int, options: int, seed: int) -> np.ndarray:
    """``count`` uniform draws from range(options), as int64."""
    return rng(seed).integers(0, options, size=int(count), dtype=np.int64)
