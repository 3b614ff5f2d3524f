"""Seeded synthetic inputs for the MTGP32 workloads.

This module only draws inputs (stream seeds, per-stream output counts, request
traces, toy parameter fields).  It holds none of the generator's arithmetic, so
both the CUDA path and its CPU checker can take their inputs from here.

Workloads (Mexp 11213 unless stated; parameter set = seed-generated from
``PARAM_SEED``):

* single   -- one stream from seed 1, 2^20 outputs.
* equal    -- 4096 streams (seeds 0..4095), 2^18 outputs each, one launch.
* long     -- Mexp 23209 and 44497, 1024 streams (seeds 0..1023), 2^20 each,
              as uint32, float32 [1,2) and float32 [0,1).
* uneven   -- 10 000 streams (seeds 0..9999), counts floor(2^U) with
              U ~ Uniform[10, 22] drawn from NumPy's PCG64 seeded with 7.
* serving  -- 65 536 resident streams; Poisson arrivals at 50 000 req/s
              (seed 11); stream uniform; k = floor(2^U), U ~ Uniform[8, 20];
              format uint32 or float32 [0,1) with probability 1/2 each.
"""
from __future__ import annotations

import numpy as np

PARAM_SEED = 0x5EED
MEXP_MAIN = 11213


def single():
    return {"mexp": MEXP_MAIN, "seeds": np.array([1], np.uint32),
            "counts": np.array([1 << 20], np.uint64)}


def equal(n_streams: int = 4096, count: int = 1 << 18):
    return {"mexp": MEXP_MAIN, "seeds": np.arange(n_streams, dtype=np.uint32),
            "counts": np.full(n_streams, count, np.uint64)}


def long_streams(mexp: int, n_streams: int = 1024, count: int = 1 << 20):
    return {"mexp": mexp, "seeds": np.arange(n_streams, dtype=np.uint32),
            "counts": np.full(n_streams, count, np.uint64)}


def uneven_counts(n_streams: int = 10000, lo: float = 10.0, hi: float = 22.0, seed: int = 7):
    rng = np.random.default_rng(seed)
    u = rng.uniform(lo, hi, size=n_streams)
    return np.floor(np.exp2(u)).astype(np.uint64)


def uneven(n_streams: int = 10000):
    return {"mexp": MEXP_MAIN, "seeds": np.arange(n_streams, dtype=np.uint32),
            "counts": uneven_counts(n_streams)}


def serving_trace(duration_s: float = 10.0, rate: float = 50000.0, n_streams: int = 65536,
                  klo: float = 8.0, khi: float = 20.0, seed: int = 11):
    """Arrival times (s), stream ids, counts and formats (0 = u32, 2 = f32 [0,1))."""
    rng = np.random.default_rng(seed)
    n_est = int(duration_s * rate * 1.2) + 1000
    gaps = rng.exponential(1.0 / rate, size=n_est)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    n = t.size
    ids = rng.integers(0, n_streams, size=n).astype(np.uint32)
    k = np.floor(np.exp2(rng.uniform(klo, khi, size=n))).astype(np.uint64)
    fmt = np.where(rng.random(n) < 0.5, 0, 2).astype(np.int32)
    return {"t": t, "ids": ids, "counts": k, "fmt": fmt, "n_streams": n_streams}


def param_seeds(n_streams: int, n_sets: int):
    """Per-stream parameter-set seeds for the one-set-per-stream setting:
    stream s uses the set generated from seed PARAM_SEED + 1 + (s mod n_sets)."""
    return (PARAM_SEED + 1 + np.arange(n_streams) % n_sets).astype(np.uint64)


def toy_fields(rng: np.random.Generator, n: int):
    """Random parameter fields for a toy status with N = n words (1 <= pos <= n-1)."""
    r = int(rng.integers(1, 32))
    mexp = 32 * n - r
    return {
        "mexp": mexp,
        "pos": int(rng.integers(1, n)),
        "sh1": int(rng.integers(1, 32)),
        "sh2": int(rng.integers(1, 32)),
        "rec_basis": [int(v) for v in rng.integers(0, 1 << 32, size=4, dtype=np.uint64)],
        "tmp_basis": [int(v) for v in rng.integers(0, 1 << 32, size=4, dtype=np.uint64)],
    }


def random_states(rng: np.random.Generator, n_streams: int, n: int):
    return rng.integers(0, 1 << 32, size=(n_streams, n), dtype=np.uint64).astype(np.uint32)
