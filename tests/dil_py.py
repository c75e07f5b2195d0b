"""Independent pieces used by the oracle pins: schoolbook ring products and
closed-form rounding, written without the oracle's NTT, Keccak or encoders."""
import hashlib

import numpy as np

Q = 8380417
N = 256


def negacyclic(a, b):
    """Schoolbook product in Z_q[X]/(X^256 + 1); inputs are small enough for int64."""
    full = np.convolve(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))
    c = full[:N].copy()
    c[: N - 1] -= full[N:]
    return c % Q


def split_bits(data: bytes, count: int, bits: int) -> np.ndarray:
    v = int.from_bytes(data, "little")
    return np.array([(v >> (bits * i)) & ((1 << bits) - 1) for i in range(count)], dtype=np.int64)


def join_bits(vals, bits: int) -> bytes:
    acc = 0
    for i, x in enumerate(vals):
        acc |= int(x) << (bits * i)
    return acc.to_bytes((len(vals) * bits + 7) // 8, "little")


def decompose(r, g2):
    r = np.asarray(r, dtype=np.int64) % Q
    alpha = 2 * g2
    r1 = (r + g2 - 1) // alpha
    r0 = r - r1 * alpha
    wrap = r1 == (Q - 1) // alpha
    return np.where(wrap, 0, r1), np.where(wrap, r0 - 1, r0)


def centred(a):
    a = np.asarray(a, dtype=np.int64) % Q
    return np.where(a > (Q - 1) // 2, a - Q, a)


def shake256(data: bytes, n: int) -> bytes:
    return hashlib.shake_256(data).digest(n)
