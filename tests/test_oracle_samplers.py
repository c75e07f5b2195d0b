"""Pins the oracle's samplers (section 2.3; Alg 1 and Alg 2).

Each sampler is re-derived here from a hashlib SHAKE stream (a second,
independent reading of the same definition) and its output ranges and
distribution are checked.
"""
import hashlib

import numpy as np
import pytest

Q = 8380417
P = {2: dict(k=4, l=4, eta=2, tau=39, g1=1 << 17),
     3: dict(k=6, l=5, eta=4, tau=49, g1=1 << 19),
     5: dict(k=8, l=7, eta=2, tau=60, g1=1 << 19)}


def py_expand_a(rho, k, l):
    out = np.zeros((k, l, 256), dtype=np.int64)
    for i in range(k):
        for j in range(l):
            stream = hashlib.shake_128(rho + bytes([j, i])).digest(168 * 8)
            vals, pos = [], 0
            while len(vals) < 256:
                t = int.from_bytes(stream[pos:pos + 3], "little") & 0x7FFFFF
                pos += 3
                if t < Q:
                    vals.append(t)
            out[i, j] = vals
    return out


def py_eta(rhop, nonce, eta):
    stream = hashlib.shake_256(rhop + nonce.to_bytes(2, "little")).digest(136 * 6)
    vals = []
    for byte in stream:
        for t in (byte & 15, byte >> 4):
            if len(vals) == 256:
                break
            if eta == 2 and t < 15:
                vals.append(2 - t % 5)
            elif eta == 4 and t < 9:
                vals.append(4 - t)
        if len(vals) == 256:
            break
    return np.array(vals)


def py_mask(rhop, nonce, g1):
    bits = 18 if g1 == 1 << 17 else 20
    stream = int.from_bytes(hashlib.shake_256(rhop + nonce.to_bytes(2, "little")).digest(32 * bits), "little")
    return np.array([g1 - ((stream >> (bits * i)) & ((1 << bits) - 1)) for i in range(256)])


def py_ball(ctilde, tau):
    stream = hashlib.shake_256(ctilde).digest(136 * 4)
    signs = int.from_bytes(stream[:8], "little")
    pos = 8
    c = [0] * 256
    for i in range(256 - tau, 256):
        while True:
            b = stream[pos]
            pos += 1
            if b <= i:
                break
        c[i] = c[b]
        c[b] = -1 if signs & 1 else 1
        signs >>= 1
    return np.array(c)


@pytest.mark.parametrize("level", [2, 3, 5])
def test_expand_a_second_reading(orc, level):
    p = P[level]
    rho = bytes(range(level, level + 32))
    got = orc.expand_a(level, rho)
    assert np.array_equal(got, py_expand_a(rho, p["k"], p["l"]))
    assert got.min() >= 0 and got.max() < Q


def test_expand_a_uniform(orc):
    vals = np.concatenate([orc.expand_a(5, bytes([s]) * 32).ravel() for s in range(4)])
    hist = np.bincount(vals // (Q // 16 + 1), minlength=16)
    exp = vals.size / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45          # 15 d.o.f.; p ~ 1e-4


@pytest.mark.parametrize("level", [2, 3, 5])
def test_expand_s_second_reading(orc, level):
    p = P[level]
    rhop = bytes(range(100, 164))
    s1, s2 = orc.expand_s(level, rhop)
    for i in range(p["l"]):
        assert np.array_equal(s1[i], py_eta(rhop, i, p["eta"]))
    for i in range(p["k"]):
        assert np.array_equal(s2[i], py_eta(rhop, p["l"] + i, p["eta"]))
    allv = np.concatenate([s1.ravel(), s2.ravel()])
    assert allv.min() >= -p["eta"] and allv.max() <= p["eta"]


@pytest.mark.parametrize("eta_level", [2, 3])
def test_expand_s_uniform(orc, eta_level):
    eta = P[eta_level]["eta"]
    vals = np.concatenate([np.concatenate(orc.expand_s(eta_level, bytes([s]) * 64)).ravel() for s in range(20)])
    hist = np.bincount(vals + eta, minlength=2 * eta + 1)
    exp = vals.size / (2 * eta + 1)
    assert ((hist - exp) ** 2 / exp).sum() < 30


@pytest.mark.parametrize("level", [2, 3, 5])
def test_expand_mask_second_reading(orc, level):
    p = P[level]
    rhop = bytes(range(7, 71))
    for kappa in (0, p["l"], 65536 - p["l"] - 3):
        y = orc.expand_mask(level, rhop, kappa)
        for i in range(p["l"]):
            assert np.array_equal(y[i], py_mask(rhop, (kappa + i) & 0xFFFF, p["g1"]))
        assert y.min() >= -p["g1"] + 1 and y.max() <= p["g1"]


@pytest.mark.parametrize("level", [2, 3, 5])
def test_sample_in_ball_second_reading(orc, level):
    tau = P[level]["tau"]
    rng = np.random.default_rng(level)
    for _ in range(40):
        ct = bytes(rng.integers(0, 256, 32, dtype=np.uint8))
        c = orc.sample_in_ball(level, ct)
        assert np.array_equal(c, py_ball(ct, tau))
        assert np.count_nonzero(c) == tau and set(np.unique(c)) <= {-1, 0, 1}
