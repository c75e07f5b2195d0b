"""Parity of each hot-path primitive (SHAKE, NTT/INTT, samplers, rounding) on
the GPU against the oracle, bit-exact, through the test-only C entry points."""
import hashlib

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

Q = 8380417


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_12265_gb300 import dil
    c = dil.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("form", [1, 2, 6, 16])
def test_keccak_f_forms(ctx, orc, form):
    """Every permutation form against the oracle's Keccak-f[1600] on random
    states, including a partly filled last warp (37 states) and the zero
    state (whose image is a FIPS 202 constant the oracle is pinned to)."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    rng = np.random.default_rng(100 + form)
    n = 37
    st = rng.integers(0, 2 ** 64, (n, 25), dtype=np.uint64)
    st[5] = 0
    out = torch.empty((n, 25), dtype=torch.int64, device="cuda")
    dil.dil_test_keccak_f(ctx.handle, form, n, dev(st.view(np.int64)), out)
    got = host(out).view(np.uint64)
    for i in range(n):
        assert np.array_equal(got[i], orc.keccak_f1600(st[i])), (form, i)


def test_shake_lengths(ctx, orc):
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    rng = np.random.default_rng(1)
    lens = np.concatenate([np.arange(0, 350), [407, 408, 409, 1000, 4096, 16384, 0]])
    msg = rng.integers(0, 256, int(lens.sum()) + 1, dtype=np.uint8)
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    for kind, outlen in ((128, 840), (256, 700), (256, 32)):
        out = torch.empty((lens.size, outlen), dtype=torch.uint8, device="cuda")
        dil.dil_test_shake(ctx.handle, kind, lens.size, dev(msg), dev(off), out, outlen)
        got = host(out)
        for i in range(lens.size):
            m = msg[off[i]:off[i + 1]].tobytes()
            want = hashlib.shake_128(m).digest(outlen) if kind == 128 else hashlib.shake_256(m).digest(outlen)
            assert got[i].tobytes() == want, (kind, i, lens[i])
        assert got[5].tobytes() == (orc.shake128 if kind == 128 else orc.shake256)(msg[off[5]:off[6]].tobytes(), outlen)


def test_k16_rider_hash(ctx, orc):
    """The hash that rides in the spare sixteen-state instance (Verify's
    tr = H(pk) for Dilithium3/5) against the oracle's SHAKE256 for every
    way the ride can end: finished on the 25-lane form from the zero state
    (0 permutations), part way, one block short, exactly at the final padded
    block, and past it (later permutations must not touch the taken output);
    lengths around the 136-byte rate, a whole number of blocks (pure padding
    block), the three public-key sizes; each on an 8-byte-aligned and an
    unaligned start (the two load paths).  One launch per case, so that each
    string's start is chosen freely."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    rng = np.random.default_rng(7)
    cases = []
    for ln in (0, 1, 7, 8, 9, 135, 136, 137, 271, 272, 273, 1000, 1312, 1952, 2592):
        total = ln // 136 + 1
        for p in sorted({0, 1, max(total - 1, 0), total, total + 1, total + 3}):
            cases += [(ln, p, 0), (ln, p, 3)]          # start mod 8
    buf = rng.integers(0, 256, 4096, dtype=np.uint8)
    d_buf = dev(buf)
    out = torch.empty((len(cases), 32), dtype=torch.uint8, device="cuda")
    for i, (ln, p, mis) in enumerate(cases):
        start = 64 + mis
        dil.dil_test_k16_rider(ctx.handle, 1, d_buf, dev(np.array([start, start + ln], dtype=np.uint64)),
                               dev(np.array([p], dtype=np.int32)), out[i:i + 1])
    got = host(out)
    for i, (ln, p, mis) in enumerate(cases):
        want = orc.shake256(buf[64 + mis:64 + mis + ln].tobytes(), 32)
        assert got[i].tobytes() == want, (ln, p, mis)


def test_k16_chain_rider_hash(ctx, orc):
    """The hash KeyGen carries while pk is being written (tr = H(pk) for
    Dilithium3/5) against the oracle's SHAKE256: input made available in
    steps of 0 (nothing until the end), less than, exactly and more than one
    136-byte block, a t1 row (320 bytes) and all at once; no permutation,
    fewer than the blocks, and more; the riding instance overwritten between
    permutations; strings at assorted alignments (one launch)."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    rng = np.random.default_rng(8)
    lens, perms, steps = [], [], []
    for ln in (0, 1, 135, 136, 137, 1000, 1312, 1952, 2592):
        total = ln // 136 + 1
        for st in (0, 50, 136, 137, 320, 5000):
            for p in sorted({0, 3, total, total + 5, 4 * total}):
                lens.append(ln)
                steps.append(st)
                perms.append(p)
    off = np.zeros(len(lens) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    buf = rng.integers(0, 256, int(off[-1]) + 8, dtype=np.uint8)
    out = torch.empty((len(lens), 32), dtype=torch.uint8, device="cuda")
    dil.dil_test_k16_chain_rider(ctx.handle, len(lens), dev(buf), dev(off), dev(np.array(perms, dtype=np.int32)),
                                 dev(np.array(steps, dtype=np.int32)), out)
    got = host(out)
    for i in range(len(lens)):
        want = orc.shake256(buf[off[i]:off[i + 1]].tobytes(), 32)
        assert got[i].tobytes() == want, (lens[i], steps[i], perms[i])


def test_ntt_forward_and_inverse(ctx, orc):
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    rng = np.random.default_rng(2)
    n = 300
    a = rng.integers(0, Q, (n, 256)).astype(np.int32)
    a[0] = 0
    a[1] = Q - 1
    a[2] = rng.integers(-(Q - 1), Q, 256)          # signed representatives
    out = torch.empty((n, 256), dtype=torch.int32, device="cuda")
    dil.dil_test_ntt(ctx.handle, n, dev(a), out, 0)
    f = host(out)
    for i in range(n):
        assert np.array_equal(f[i], orc.ntt(a[i] % Q)), i
    dil.dil_test_ntt(ctx.handle, n, dev(f), out, 1)
    g = host(out)
    assert np.array_equal(g, a % Q)
    for i in range(0, n, 37):
        assert np.array_equal(g[i], orc.intt(f[i]))


@pytest.mark.parametrize("level", [2, 3, 5])
def test_samplers(ctx, orc, level):
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    p = orc.params(level)
    k, l = p["k"], p["l"]
    rng = np.random.default_rng(level)
    n = 40
    rho = rng.integers(0, 256, (n, 32), dtype=np.uint8)
    rhop = rng.integers(0, 256, (n, 64), dtype=np.uint8)
    kappa = rng.integers(0, 65536 - l, n).astype(np.int32)
    kappa[:3] = [0, l, 65536 - l]
    ct = rng.integers(0, 256, (n, 32), dtype=np.uint8)
    A = torch.empty((n, k, l, 256), dtype=torch.int32, device="cuda")
    S = torch.empty((n, l + k, 256), dtype=torch.int32, device="cuda")
    Y = torch.empty((n, l, 256), dtype=torch.int32, device="cuda")
    C = torch.empty((n, 256), dtype=torch.int32, device="cuda")
    dil.dil_test_expand_a(ctx.handle, level, n, dev(rho), A)
    dil.dil_test_expand_s(ctx.handle, level, n, dev(rhop), S)
    dil.dil_test_expand_mask(ctx.handle, level, n, dev(rhop), dev(kappa), Y)
    dil.dil_test_sample_in_ball(ctx.handle, level, n, dev(ct), C)
    A, S, Y, C = host(A), host(S), host(Y), host(C)
    for i in range(n):
        assert np.array_equal(A[i], orc.expand_a(level, rho[i].tobytes())), i
        s1, s2 = orc.expand_s(level, rhop[i].tobytes())
        assert np.array_equal(S[i], np.concatenate([s1, s2])), i
        assert np.array_equal(Y[i], orc.expand_mask(level, rhop[i].tobytes(), int(kappa[i]))), i
        assert np.array_equal(C[i], orc.sample_in_ball(level, ct[i].tobytes())), i


@pytest.mark.parametrize("level", [2, 3, 5])
def test_rounding_exhaustive(ctx, orc, level):
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    r = np.arange(Q, dtype=np.int32)
    rng = np.random.default_rng(level)
    g2 = orc.params(level)["gamma2"]
    z = (rng.integers(-g2, g2 + 1, Q) % Q).astype(np.int32)
    h = rng.integers(0, 2, Q, dtype=np.uint8)
    out = torch.empty((Q, 6), dtype=torch.int32, device="cuda")
    dil.dil_test_rounding(ctx.handle, level, Q, dev(r), dev(z), dev(h), out)
    o = host(out)
    p1, p0 = orc.power2round(r)
    d1, d0 = orc.decompose(level, r)
    assert np.array_equal(o[:, 0], p1) and np.array_equal(o[:, 1], p0)
    assert np.array_equal(o[:, 2], d1) and np.array_equal(o[:, 3], d0)
    assert np.array_equal(o[:, 4], orc.make_hint(level, z, r))
    assert np.array_equal(o[:, 5], orc.use_hint(level, h, r))


def test_probes_report_plausible_rates(ctx):
    """The roofline probes: issue rates within the SM's 128 lanes per clock,
    and the six-state Keccak form cheaper per state-round than the one-state
    form it replaces in the samplers."""
    from paper_2211_12265_gb300 import dil
    for op in dil.ISSUE_OPS.values():
        r = dil.dil_test_issue_rate(ctx.handle, op)
        assert 1.0 < r <= 128.0, (op, r)
    one = dil.dil_test_keccak_rate(ctx.handle, 1)
    six = dil.dil_test_keccak_rate(ctx.handle, 6)
    sixteen = dil.dil_test_keccak_rate(ctx.handle, 16)
    assert 0.5 < six < one, (six, one)
    assert 0.25 < sixteen < six, (sixteen, six)
    with pytest.raises(dil.DilError):
        dil.dil_test_keccak_rate(ctx.handle, 3)


@pytest.mark.parametrize("level", [2, 3, 5])
def test_t0_ntt_breakdown_variants(ctx, orc, level):
    """The four forms of the t^0 = NTT(t0) breakdown (two kernels through
    global memory, fused, registers with a conflicting exchange, registers
    with the conflict-free one) give the same t^0, equal to the oracle's NTT
    of t0 unpacked from sk."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    from paper_2211_12265_gb300 import workload as W
    n = 300
    k = {2: 4, 3: 6, 5: 8}[level]
    _, sk = ctx.keygen(level, dev(W.seeds(n, 60 + level)))
    outs = []
    for variant in range(4):
        out = torch.full((n, k, 256), -1, dtype=torch.int32, device="cuda")
        dil.dil_test_t0_ntt(ctx.handle, level, variant, n, sk, out)
        outs.append(host(out))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    skh = host(sk)
    eta_bits = 3 if level in (2, 5) else 4
    l = {2: 4, 3: 5, 5: 7}[level]
    t0_at = 96 + (k + l) * 32 * eta_bits
    for i in range(0, n, 7):
        for j in range(k):
            field = orc.unpack_bits(skh[i, t0_at + 416 * j: t0_at + 416 * (j + 1)].tobytes(), 256, 13)
            t0 = (4096 - field.astype(np.int64)) % Q
            assert np.array_equal(outs[3][i, j], orc.ntt(t0)), (i, j)
    with pytest.raises(dil.DilError):
        dil.dil_test_t0_ntt(ctx.handle, level, 4, n, sk, out)


def _sib_reference(blocks, tau):
    """SampleInBall's drawing and swapping (section 2.3) over a given byte
    stream, one step at a time; past the last block the last one repeats."""
    signs = int.from_bytes(bytes(blocks[0][:8]), "little")
    c = [0] * 256
    state = {"blk": 0, "pos": 8}

    def next_byte():
        if state["pos"] == 136:
            state["blk"] += 1
            state["pos"] = 0
        b = int(blocks[min(state["blk"], len(blocks) - 1)][state["pos"]])
        state["pos"] += 1
        return b

    for k, i in enumerate(range(256 - tau, 256)):
        while True:
            b = next_byte()
            if b <= i:
                break
        c[i] = c[b]
        c[b] = -1 if (signs >> k) & 1 else 1
    return np.array(c, dtype=np.int32)


@pytest.mark.parametrize("level", [2, 3, 5])
def test_sample_in_ball_adversarial_streams(ctx, level):
    """The warp-parallel SampleInBall against the sequential definition on
    streams built to stress it: heavy rejection, a first block rejected
    entirely (the draw continues in the next block), repeated positions
    (values moved several times), b = i, draws of every i, and random bytes."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    tau = {2: 39, 3: 49, 5: 60}[level]
    lo = 256 - tau
    rng = np.random.default_rng(500 + level)
    nb = 4
    cases = []
    for kind in range(8):
        for _ in range(12):
            s = rng.integers(0, 256, (nb, 136), dtype=np.uint8)
            if kind == 1:                                  # heavy rejection
                s = rng.integers(lo - 20, 256, (nb, 136)).astype(np.uint8)
            elif kind == 2:                                # block 0 all rejected
                s[0, 8:] = 255
            elif kind == 3:                                # few distinct positions
                s[:, :] = rng.choice([0, 1, 2, lo, lo + 1, lo + 2], (nb, 136)).astype(np.uint8)
                s[0, :8] = rng.integers(0, 256, 8, dtype=np.uint8)
            elif kind == 4:                                # b = i at every step
                s[0, 8:8 + tau] = np.arange(lo, 256, dtype=np.uint8)
            elif kind == 5:                                # draws of earlier i's
                s[:, :] = rng.integers(lo, 256, (nb, 136)).astype(np.uint8)
                s[0, :8] = rng.integers(0, 256, 8, dtype=np.uint8)
            elif kind == 6:                                # rejections across the first chunk boundaries
                s[0, 8:136] = np.where(rng.random(128) < 0.6, 255, s[0, 8:136]).astype(np.uint8)
            elif kind == 7:                                # two blocks fully rejected
                s[0, 8:] = 255
                s[1, :] = 255
            cases.append(s)
    data = np.stack(cases)
    n = data.shape[0]
    out = torch.empty((n, 256), dtype=torch.int32, device="cuda")
    dil.dil_test_sample_in_ball_stream(ctx.handle, level, n, dev(data), nb, out)
    got = host(out)
    for i in range(n):
        want = _sib_reference(list(data[i]), tau)
        assert np.array_equal(got[i], want), (i, i // 12)
        assert int(np.abs(got[i]).sum()) == tau
