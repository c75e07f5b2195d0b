"""Algorithmic work of Sign and Verify (Alg 2, Alg 3 of arXiv 2211.12265).

Counts what the algorithm itself requires, independent of how a kernel does
it: Keccak-f[1600] permutations, NTT/INTT butterflies (1024 per 256-point
transform), pointwise products mod q, and sampled or (un)packed coefficients.
Sign's count depends on the number of loop repetitions per task, which the
engine reports (``dil_sign_ex``); the masking term (Alg 2) is counted
once per task, for the accepted repetition, so the figure is a lower bound.

``int_ops`` converts the counts to 32-bit integer operations with fixed
weights (the roofline numerator):
  * Keccak-f round on 32-bit halves with 3-input logic ops: theta 90 (column
    parities 20, D 20, A ^= D 50), rho 48 funnel shifts, chi 50, iota 2
    -> 190 per round, 4560 per permutation;
  * Montgomery butterfly: 4 multiplies (lo, hi, q^-1, hi) + 3 add/sub = 7;
  * pointwise Montgomery product with accumulation: 6;
  * sampled or (un)packed coefficient: 5.
"""
from __future__ import annotations

import math

import numpy as np

N = 256
OPS_PER_PERMUTATION = 24 * 190
OPS_PER_BUTTERFLY = 7
OPS_PER_POINTWISE = 6
OPS_PER_COEFFICIENT = 5

LEVELS = {
    2: dict(k=4, l=4, tau=39, pk=1312, w1_bytes=192),
    3: dict(k=6, l=5, tau=49, pk=1952, w1_bytes=128),
    5: dict(k=8, l=7, tau=60, pk=2592, w1_bytes=128),
}


def _absorb_perms(nbytes, rate=136):
    """Permutations to absorb nbytes and pad (one per full block, plus one)."""
    return np.floor_divide(np.asarray(nbytes, dtype=np.int64), rate) + 1


def sign_work(level: int, iterations, msg_lengths) -> dict:
    """Total work of a batch of Sign tasks with the given repetition counts."""
    p = LEVELS[level]
    k, l, tau = p["k"], p["l"], p["tau"]
    it = np.asarray(iterations, dtype=np.int64)
    n = it.size
    reps = int(it.sum())
    hash_ct = int(_absorb_perms(64 + k * p["w1_bytes"]))
    perms = int(_absorb_perms(32 + np.asarray(msg_lengths)).sum())   # mu
    perms += n * (1 + 5 * k * l)                                      # rho', ExpandA
    perms += reps * (5 * l + hash_ct + 1)                            # ExpandMask, c~, SampleInBall
    bfly = 1024 * (n * (l + 2 * k) + reps * (2 * l + 2 * k + 1) + n * k)
    pw = N * (reps * (k * l + l + k) + n * k)
    coef = n * N * (l + 2 * k + k * l) + reps * (N * (l + k) + tau) + n * N * l
    return dict(permutations=perms, butterflies=bfly, pointwise=pw, coefficients=coef)


def verify_work(level: int, msg_lengths) -> dict:
    """Total work of a batch of Verify tasks on valid signatures."""
    p = LEVELS[level]
    k, l, tau = p["k"], p["l"], p["tau"]
    m = np.asarray(msg_lengths)
    n = m.size
    perms = n * (int(_absorb_perms(p["pk"])) + 1 + 5 * k * l + int(_absorb_perms(64 + k * p["w1_bytes"])))
    perms += int(_absorb_perms(32 + m).sum())
    bfly = 1024 * n * (l + 2 * k + 1)
    pw = N * n * (k * l + k)
    coef = n * (N * (k + l + k * l + k) + tau)
    return dict(permutations=perms, butterflies=bfly, pointwise=pw, coefficients=coef)


def int_ops(work: dict) -> int:
    return (work["permutations"] * OPS_PER_PERMUTATION + work["butterflies"] * OPS_PER_BUTTERFLY
            + work["pointwise"] * OPS_PER_POINTWISE + work["coefficients"] * OPS_PER_COEFFICIENT)


def add(a: dict, b: dict) -> dict:
    return {key: a[key] + b[key] for key in a}


def expected_iterations(level: int) -> float:
    """The paper's expected repetition counts (section 2.3 'Rejection Loop')."""
    return {2: 4.25, 3: 5.1, 5: 3.85}[level]


def ceil_div(a: int, b: int) -> int:
    return -(-a // b) if b else 0


__all__ = ["sign_work", "verify_work", "int_ops", "add", "expected_iterations", "ceil_div", "math"]
