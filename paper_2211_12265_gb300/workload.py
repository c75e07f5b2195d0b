"""Seeded synthetic inputs for batched Dilithium workloads.

This module holds no part of the signature scheme's arithmetic: it only draws
seeds, message lengths, message bytes and request arrival times from seeded
``numpy`` generators (PCG64).  It is shared by the tests, the benchmark and the
serving driver so that the CUDA path and the oracle see identical inputs.

Recipe (the paper's workloads are batches of 10,000 independent random tasks,
section 5.4; message lengths are not stated there):
  * config c draws key-generation seeds (32 bytes each) from PCG64(1000 + c),
    message lengths from PCG64(2000 + c) and message bytes from PCG64(3000 + c);
  * configs 1, 2 and 4 use 32-byte messages; config 3 uses lengths uniform in
    [32, 4096]; the serving workload uses lengths log-uniform in [32, 16384].
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def seeds(n: int, config: int = 1, offset: int = 0) -> np.ndarray:
    """n key-generation seeds (uint8 [n, 32]); ``offset`` skips that many seeds."""
    g = _rng(1000 + config)
    if offset:
        g.integers(0, 256, size=(offset, 32), dtype=np.uint8)
    return g.integers(0, 256, size=(n, 32), dtype=np.uint8)


def message_lengths(n: int, config: int = 1, kind: str = "fixed", lo: int = 32, hi: int = 32) -> np.ndarray:
    """Message lengths in bytes (int64 [n]).

    kind = "fixed" (all ``lo``), "uniform" (integers in [lo, hi]) or
    "loguniform" (exp of a uniform draw in [log lo, log hi], rounded down).
    """
    g = _rng(2000 + config)
    if kind == "fixed":
        return np.full(n, lo, dtype=np.int64)
    if kind == "uniform":
        return g.integers(lo, hi + 1, size=n, dtype=np.int64)
    if kind == "loguniform":
        u = g.uniform(np.log(lo), np.log(hi), size=n)
        return np.clip(np.floor(np.exp(u)).astype(np.int64), lo, hi)
    raise ValueError(kind)


def messages(lengths: np.ndarray, config: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Concatenated message bytes (uint8) and byte offsets (uint64 [n + 1])."""
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.zeros(lengths.size + 1, dtype=np.uint64)
    np.cumsum(lengths, out=off[1:])
    total = int(off[-1])
    g = _rng(3000 + config)
    msg = g.integers(0, 256, size=max(total, 1), dtype=np.uint8)
    return msg, off


CONFIG_MSG = {1: ("fixed", 32, 32), 2: ("fixed", 32, 32), 3: ("uniform", 32, 4096),
              4: ("fixed", 32, 32), 5: ("loguniform", 32, 16384)}


def workload(config: int, n: int) -> dict:
    """Seeds and messages of one of the five benchmark configurations."""
    kind, lo, hi = CONFIG_MSG[config]
    lens = message_lengths(n, config, kind, lo, hi)
    msg, off = messages(lens, config)
    return {"seeds": seeds(n, config), "msg": msg, "msg_off": off, "lengths": lens}


def arrivals(n: int, rate_per_s: float, seed: int = 5005) -> np.ndarray:
    """Poisson arrival times in seconds (float64 [n]) at the given mean rate."""
    g = _rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=n))


def request_mix(n: int, n_keys: int, seed: int = 5006, p_verify: float = 0.6,
                levels=(2, 3, 5)) -> dict:
    """Serving mix: op (0 = sign, 1 = verify), level and resident-key index."""
    g = _rng(seed)
    op = (g.uniform(size=n) < p_verify).astype(np.int32)
    level = np.asarray(levels, dtype=np.int32)[g.integers(0, len(levels), size=n)]
    key = g.integers(0, n_keys, size=n, dtype=np.int64)
    return {"op": op, "level": level, "key": key}
