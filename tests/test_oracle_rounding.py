"""Pins Power2Round / Decompose / MakeHint / UseHint (section 2.3, "Bits
Extraction and Hints") exhaustively over every r in [0, q)."""
import numpy as np
import pytest

Q = 8380417
ALL = np.arange(Q, dtype=np.int32)


def test_power2round_exhaustive(orc):
    r1, r0 = orc.power2round(ALL)
    r1 = r1.astype(np.int64)
    r0 = r0.astype(np.int64)
    assert np.array_equal(r1 * 8192 + r0, ALL.astype(np.int64))      # exact split
    assert r0.min() == -4095 and r0.max() == 4096                     # (-2^12, 2^12]
    assert r1.min() == 0 and r1.max() == 1023                          # fits the 10-bit t1


@pytest.mark.parametrize("level", [2, 3])
def test_decompose_exhaustive(orc, level):
    g2 = 95232 if level == 2 else 261888
    alpha = 2 * g2
    m = (Q - 1) // alpha
    r1, r0 = orc.decompose(level, ALL)
    r = ALL.astype(np.int64)
    # independent closed form: r1' = ceil((r - g2) / alpha), wrap when r1' = m
    r1c = (r + g2 - 1) // alpha
    r0c = r - r1c * alpha
    wrap = r1c == m
    r1c = np.where(wrap, 0, r1c)
    r0c = np.where(wrap, r0c - 1, r0c)
    assert np.array_equal(r1, r1c) and np.array_equal(r0, r0c)
    # properties: range, reconstruction mod q, wrap region
    assert r1.min() == 0 and r1.max() == m - 1
    assert np.all((r1.astype(np.int64) * alpha + r0 - r) % Q == 0)
    assert np.array_equal(wrap, r >= Q - g2)
    assert np.all((r0[~wrap] > -g2) & (r0[~wrap] <= g2))
    assert np.all((r0[wrap] >= -g2) & (r0[wrap] < 0))


@pytest.mark.parametrize("level", [2, 5])
def test_use_hint_recovers_high_bits(orc, level):
    # Lemma: UseHint(MakeHint(z, r), r) = HighBits(r + z) whenever |z| <= gamma2
    g2 = 95232 if level == 2 else 261888
    rng = np.random.default_rng(level)
    for _ in range(2):
        z = rng.integers(-g2, g2 + 1, Q).astype(np.int64)
        zq = (z % Q).astype(np.int32)
        h = orc.make_hint(level, zq, ALL)
        got = orc.use_hint(level, h, ALL)
        want, _ = orc.decompose(level, ((ALL.astype(np.int64) + z) % Q).astype(np.int32))
        assert np.array_equal(got, want)
    assert 0 < h.mean() < 1


def test_use_hint_wraps_modulo_m(orc):
    level = 2
    m = 44
    r1, r0 = orc.decompose(level, ALL)
    ones = np.ones(Q, dtype=np.uint8)
    u = orc.use_hint(level, ones, ALL)
    up = r0 > 0
    assert np.array_equal(u[up], (r1[up] + 1) % m)
    assert np.array_equal(u[~up], (r1[~up] - 1) % m)
    assert u.min() == 0 and u.max() == m - 1


def test_high_bits_stable_under_small_shift(orc):
    # if |LowBits(r)| < gamma2 - beta and |s| <= beta then HighBits(r + s) = HighBits(r)
    level, g2, beta = 2, 95232, 78
    rng = np.random.default_rng(3)
    s = rng.integers(-beta, beta + 1, Q)
    r1, r0 = orc.decompose(level, ALL)
    sel = np.abs(r0) < g2 - beta
    r1s, _ = orc.decompose(level, ((ALL.astype(np.int64) + s) % Q).astype(np.int32))
    assert np.array_equal(r1s[sel], r1[sel])
