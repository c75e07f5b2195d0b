"""Pins the oracle's Alg 1 (Gen), Alg 2 (Sign) and Alg 3 (Verify).

* Verify(Sign(m)) accepts; every single-bit flip of the signature, public key
  or message is rejected (Alg 3).
* Gen's public and secret key satisfy t = A s1 + s2 with A s1 computed by the
  schoolbook product, and (t1, t0) = Power2Round(t) (Alg 1).
* A second Verify, written here with schoolbook products and the closed-form
  rounding, accepts the oracle's signatures (Alg 3).
* The mean number of Sign loop repetitions matches the values the paper prints
  (section 2.3 "Rejection Loop": 4.25 / 5.1 / 3.85) within 3 standard errors.
"""
import json
import os

import numpy as np
import pytest

from dil_py import Q, centred, decompose, join_bits, negacyclic, shake256, split_bits
from paper_2211_12265_gb300 import workload as W
from test_oracle_samplers import py_ball, py_eta, py_expand_a

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))["levels"]


@pytest.mark.parametrize("level", [2, 3, 5])
def test_params_match_table1(orc, level):
    g = GOLD[str(level)]
    p = orc.params(level)
    for key in ("k", "l", "eta", "tau", "beta", "omega", "gamma1", "gamma2", "d", "q"):
        assert p[key] == g[key], key
    assert g["beta"] == g["tau"] * g["eta"]


@pytest.mark.parametrize("level", [2, 3, 5])
def test_sign_verify_roundtrip(orc, level):
    seeds = W.seeds(24, config=50 + level)
    pk, sk = orc.keygen_batch(level, seeds)
    lens = W.message_lengths(24, 50 + level, "uniform", 0, 700)
    msg, off = W.messages(lens, 50 + level)
    sig, st, it = orc.sign_batch(level, sk, msg, off)
    assert (st == 0).all() and (it >= 1).all()
    assert orc.verify_batch(level, pk, msg, off, sig).all()
    # signing is deterministic
    sig2, _, _ = orc.sign_batch(level, sk, msg, off, nthreads=1)
    assert np.array_equal(sig, sig2)
    # a signature does not verify under another key or message
    assert not orc.verify_batch(level, np.roll(pk, 1, axis=0), msg, off, sig).any()


def _flip(buf: np.ndarray, bit: int) -> np.ndarray:
    out = buf.copy()
    out[bit // 8] ^= 1 << (bit % 8)
    return out


def test_every_signature_bit_flip_rejected_level2(orc):
    level = 2
    pk, sk = orc.keygen(level, bytes(range(32)))
    m = b"single-bit flips of the signature"
    st, sig, _ = orc.sign(level, sk, m)
    assert st == 0
    s = np.frombuffer(sig, dtype=np.uint8)
    nbits = s.size * 8
    sigs = np.stack([_flip(s, b) for b in range(nbits)])
    off = np.arange(nbits + 1, dtype=np.uint64) * len(m)
    msgs = np.frombuffer(m * nbits, dtype=np.uint8)
    pks = np.repeat(np.frombuffer(pk, dtype=np.uint8)[None], nbits, axis=0)
    assert not orc.verify_batch(level, pks, msgs, off, sigs).any()


@pytest.mark.parametrize("level", [2, 3, 5])
def test_sampled_bit_flips_rejected(orc, level):
    rng = np.random.default_rng(level)
    pk, sk = orc.keygen(level, bytes([level]) * 32)
    m = bytes(rng.integers(0, 256, 32, dtype=np.uint8))
    st, sig, _ = orc.sign(level, sk, m)
    p = np.frombuffer(pk, dtype=np.uint8)
    s = np.frombuffer(sig, dtype=np.uint8)
    mm = np.frombuffer(m, dtype=np.uint8)
    cases_pk, cases_sig, cases_m = [], [], []
    for b in rng.choice(p.size * 8, 600, replace=False):
        cases_pk.append(_flip(p, b)); cases_sig.append(s); cases_m.append(mm)
    for b in rng.choice(s.size * 8, 900, replace=False):
        cases_pk.append(p); cases_sig.append(_flip(s, b)); cases_m.append(mm)
    for b in range(mm.size * 8):
        cases_pk.append(p); cases_sig.append(s); cases_m.append(_flip(mm, b))
    n = len(cases_pk)
    off = np.arange(n + 1, dtype=np.uint64) * mm.size
    ok = orc.verify_batch(level, np.stack(cases_pk), np.concatenate(cases_m), off, np.stack(cases_sig))
    assert not ok.any()
    assert orc.verify(level, pk, m, sig)


@pytest.mark.parametrize("level", [2, 3, 5])
def test_noncanonical_hint_encodings_rejected(orc, level):
    """Strict hint decoding: re-encodings of a valid signature's own hint set
    (a nonzero byte in an unused index slot; two indices of one polynomial
    swapped) leave c~ matching, so only the decoding rules reject them.  The
    oracle rejects every one and accepts the originals."""
    p = orc.params(level)
    omega, k = p["omega"], p["k"]
    seeds = W.seeds(24, 6)
    msg, off = W.messages(W.message_lengths(24, 6, "fixed", 32, 32), 6)
    pk, sk = orc.keygen_batch(level, seeds)
    sig, _, _ = orc.sign_batch(level, sk, msg, off)
    hoff = sig.shape[1] - omega - k
    kinds = {"unused": 0, "order": 0}
    for i in range(sig.shape[0]):
        counts = [int(c) for c in sig[i, hoff + omega:]]
        variants = []
        if counts[-1] < omega:
            t = sig[i].copy()
            t[hoff + counts[-1]] = 0x5A
            variants.append(("unused", t))
        prev = 0
        for c in counts:
            if c - prev >= 2:
                t = sig[i].copy()
                t[hoff + prev], t[hoff + prev + 1] = t[hoff + prev + 1], t[hoff + prev]
                variants.append(("order", t))
                break
            prev = c
        m = msg[off[i]:off[i + 1]]
        o = np.array([0, m.size], dtype=np.uint64)
        assert orc.verify_batch(level, pk[i:i + 1], m, o, sig[i:i + 1])[0] == 1
        for kind, t in variants:
            assert orc.verify_batch(level, pk[i:i + 1], m, o, t[None])[0] == 0, (i, kind)
            kinds[kind] += 1
    assert kinds["unused"] > 0 and kinds["order"] > 0


def test_empty_message(orc):
    for level in (2, 3, 5):
        pk, sk = orc.keygen(level, bytes(32))
        st, sig, _ = orc.sign(level, sk, b"")
        assert st == 0 and orc.verify(level, pk, b"", sig)
        assert not orc.verify(level, pk, b"\x00", sig)


def test_iteration_cap(orc):
    level = 2
    seeds = W.seeds(64, config=60)
    pk, sk = orc.keygen_batch(level, seeds)
    msg, off = W.messages(np.full(64, 32), 60)
    sig, st, it = orc.sign_batch(level, sk, msg, off)
    capped, cst, cit = orc.sign_batch(level, sk, msg, off, max_iter=1)
    one = it == 1
    assert one.any() and (~one).any()
    assert (cst[one] == 0).all() and np.array_equal(capped[one], sig[one])
    assert (cst[~one] == -5).all() and (capped[~one] == 0).all() and (cit[~one] == 1).all()


def _params(orc, level):
    p = orc.params(level)
    p["zb"] = 18 if p["gamma1"] == 1 << 17 else 20
    p["w1b"] = 6 if p["gamma2"] == (Q - 1) // 88 else 4
    p["etab"] = 3 if p["eta"] == 2 else 4
    return p


@pytest.mark.parametrize("level", [2, 3, 5])
def test_keygen_against_schoolbook(orc, level):
    p = _params(orc, level)
    k, l = p["k"], p["l"]
    seed = bytes(range(40, 72))
    pk, sk = orc.keygen(level, seed)
    hb = shake256(seed, 128)
    rho, rhop, key = hb[:32], hb[32:96], hb[96:]
    A = np.array([[orc.intt(row) for row in rows] for rows in py_expand_a(rho, k, l).astype(np.int32)])
    s1 = [py_eta(rhop, j, p["eta"]) for j in range(l)]
    s2 = [py_eta(rhop, l + i, p["eta"]) for i in range(k)]
    assert pk[:32] == rho and sk[:32] == rho and sk[32:64] == key
    assert sk[64:96] == shake256(pk, 32)
    t1_pk = split_bits(pk[32:], k * 256, 10).reshape(k, 256)
    eb = 256 * p["etab"] // 8
    t0_off = 96 + (k + l) * eb
    t0_sk = 4096 - split_bits(sk[t0_off:], k * 256, 13).reshape(k, 256)
    for i in range(k):
        t = (sum(negacyclic(A[i, j], s1[j]) for j in range(l)) + s2[i]) % Q
        t0 = t % 8192
        t0 = np.where(t0 > 4096, t0 - 8192, t0)
        assert np.array_equal(t1_pk[i], (t - t0) // 8192)
        assert np.array_equal(t0_sk[i], t0)
    s_sk = p["eta"] - split_bits(sk[96:t0_off], (k + l) * 256, p["etab"]).reshape(k + l, 256)
    assert np.array_equal(s_sk, np.array(s1 + s2))


def py_verify(orc, level, pk, m, sig):
    p = _params(orc, level)
    k, l, g1, g2 = p["k"], p["l"], p["gamma1"], p["gamma2"]
    rho = pk[:32]
    t1 = split_bits(pk[32:], k * 256, 10).reshape(k, 256)
    ct = sig[:32]
    zb = 256 * p["zb"] // 8
    z = g1 - split_bits(sig[32:32 + l * zb], l * 256, p["zb"]).reshape(l, 256)
    hb = sig[32 + l * zb:]
    h = np.zeros((k, 256), dtype=np.int64)
    prev = 0
    for i in range(k):
        end = hb[p["omega"] + i]
        if end < prev or end > p["omega"]:
            return False
        for j in range(prev, end):
            if j > prev and hb[j] <= hb[j - 1]:
                return False
            h[i, hb[j]] = 1
        prev = end
    if any(hb[prev:p["omega"]]):
        return False
    if np.abs(z).max() >= g1 - p["beta"]:
        return False
    A = np.array([[orc.intt(row) for row in rows] for rows in py_expand_a(rho, k, l).astype(np.int32)])
    c = py_ball(ct, p["tau"])
    mu = shake256(shake256(pk, 32) + m, 64)
    w1 = []
    m_hi = (Q - 1) // (2 * g2)
    for i in range(k):
        v = (sum(negacyclic(A[i, j], z[j]) for j in range(l)) - negacyclic(c, t1[i] * 8192)) % Q
        r1, r0 = decompose(v, g2)
        adj = np.where(r0 > 0, (r1 + 1) % m_hi, (r1 - 1) % m_hi)
        w1.extend(np.where(h[i] == 1, adj, r1))
    return shake256(mu + join_bits(w1, p["w1b"]), 32) == ct and h.sum() <= p["omega"]


@pytest.mark.parametrize("level", [2, 3, 5])
def test_signatures_pass_schoolbook_verify(orc, level):
    rng = np.random.default_rng(200 + level)
    for t in range(2):
        pk, sk = orc.keygen(level, bytes(rng.integers(0, 256, 32, dtype=np.uint8)))
        m = bytes(rng.integers(0, 256, 40 + t, dtype=np.uint8))
        st, sig, _ = orc.sign(level, sk, m)
        assert st == 0
        assert py_verify(orc, level, pk, m, sig)
        bad = bytearray(sig)
        bad[40] ^= 4
        assert not py_verify(orc, level, pk, m, bytes(bad))
        # the signature's z and hint satisfy the Alg 2 bounds
        p = _params(orc, level)
        zb = 256 * p["zb"] // 8
        z = p["gamma1"] - split_bits(sig[32:32 + p["l"] * zb], p["l"] * 256, p["zb"])
        assert np.abs(z).max() < p["gamma1"] - p["beta"]
        assert sig[32 + p["l"] * zb + p["omega"] + p["k"] - 1] <= p["omega"]


@pytest.mark.parametrize("level", [2, 3, 5])
def test_mean_repetitions_match_paper(orc, level):
    expected = GOLD[str(level)]["expected_repetitions"]
    n_keys, per_key = 100, 100
    pk, sk = orc.keygen_batch(level, W.seeds(n_keys, config=90 + level))
    sks = np.repeat(sk, per_key, axis=0)
    msg, off = W.messages(np.full(n_keys * per_key, 32), 80 + level)
    orc.counters_reset()
    _, st, it = orc.sign_batch(level, sks, msg, off)
    c = orc.counters()
    assert (st == 0).all()
    pacc = 1.0 / expected
    se = np.sqrt((1 - pacc) / pacc ** 2 / it.size)      # geometric number of repetitions
    assert abs(it.mean() - expected) < 3 * se + 0.005, (it.mean(), expected, se)
    # the two readings of the r0 check (LowBits(w - cs2) versus LowBits(w) - cs2) agree
    assert c["sign_iterations"] == it.sum()
    assert c["r0_form_disagreements"] == 0
