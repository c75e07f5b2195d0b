"""Pins the oracle's Keccak-f[1600] / SHAKE (section 2.3 "Sampling") to hashlib."""
import hashlib

import numpy as np


def test_shake_all_short_lengths(orc):
    data = bytes(np.random.default_rng(7).integers(0, 256, 700, dtype=np.uint8))
    for n in range(0, 601):
        m = data[:n]
        assert orc.shake128(m, 200) == hashlib.shake_128(m).digest(200), n
        assert orc.shake256(m, 200) == hashlib.shake_256(m).digest(200), n


def test_shake_block_boundaries_both_sides(orc):
    rng = np.random.default_rng(8)
    for n in (134, 135, 136, 137, 166, 167, 168, 169, 271, 272, 273, 335, 336, 337):
        m = bytes(rng.integers(0, 256, n, dtype=np.uint8))
        for out in (0, 1, 32, 64, 135, 136, 137, 167, 168, 169, 840, 1000):
            assert orc.shake128(m, out) == hashlib.shake_128(m).digest(out)
            assert orc.shake256(m, out) == hashlib.shake_256(m).digest(out)


def test_shake_long_random(orc):
    rng = np.random.default_rng(9)
    for _ in range(25):
        n = int(rng.integers(600, 20_000))
        m = bytes(rng.integers(0, 256, n, dtype=np.uint8))
        assert orc.shake128(m, 64) == hashlib.shake_128(m).digest(64)
        assert orc.shake256(m, 64) == hashlib.shake_256(m).digest(64)


def test_permutation_is_a_bijection_on_samples(orc):
    # distinct states stay distinct and the permutation moves every sample
    rng = np.random.default_rng(10)
    seen = set()
    for _ in range(64):
        st = rng.integers(0, 2**63, 25, dtype=np.uint64)
        out = orc.keccak_f1600(st)
        assert not np.array_equal(out, st)
        seen.add(out.tobytes())
    assert len(seen) == 64
