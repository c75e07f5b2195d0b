"""Parity of the fused Gen / Sign / Verify kernels against the oracle: keys,
signatures and accept bits bit-exact on the same seeded inputs."""
import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_12265_gb300 import dil
    c = dil.Context(0)
    yield c
    c.close()


def _batch(orc, level, n, config, kind="fixed", lo=32, hi=32):
    seeds = W.seeds(n, config)
    lens = W.message_lengths(n, config, kind, lo, hi)
    msg, off = W.messages(lens, config)
    return seeds, msg, off


def test_config1_dilithium2_1024_bit_exact(ctx, orc):
    """Dilithium2, 1024 tasks, 32-byte seeds and 32-byte messages: pk, sk,
    signatures and accept bits equal the oracle's byte for byte."""
    from gpu_util import gpu_keygen, gpu_sign, gpu_verify
    level, n = 2, 1024
    seeds, msg, off = _batch(orc, level, n, 1)
    pk, sk = gpu_keygen(ctx, level, seeds)
    opk, osk = orc.keygen_batch(level, seeds)
    assert np.array_equal(pk, opk) and np.array_equal(sk, osk)
    sig, st, it = gpu_sign(ctx, level, sk, msg, off)
    osig, ost, oit = orc.sign_batch(level, osk, msg, off)
    assert np.array_equal(st, ost) and np.array_equal(it, oit)
    assert np.array_equal(sig, osig)
    ok = gpu_verify(ctx, level, pk, msg, off, sig)
    assert ok.all()


@pytest.mark.parametrize("level", [3, 5])
def test_levels_3_5_ragged_messages(ctx, orc, level):
    from gpu_util import gpu_keygen, gpu_sign, gpu_verify
    n = 200
    seeds, msg, off = _batch(orc, level, n, 3, "uniform", 0, 4096)
    pk, sk = gpu_keygen(ctx, level, seeds)
    opk, osk = orc.keygen_batch(level, seeds)
    assert np.array_equal(pk, opk) and np.array_equal(sk, osk)
    sig, st, it = gpu_sign(ctx, level, sk, msg, off)
    osig, ost, oit = orc.sign_batch(level, osk, msg, off)
    assert np.array_equal(it, oit) and np.array_equal(sig, osig)
    assert gpu_verify(ctx, level, pk, msg, off, sig).all()


@pytest.mark.parametrize("level", [2, 3, 5])
def test_verify_rejections_match_oracle(ctx, orc, level):
    """Tampered signatures, keys and messages (and malformed hints) are
    rejected exactly as the oracle rejects them."""
    from gpu_util import gpu_verify
    rng = np.random.default_rng(10 + level)
    seeds, msg, off = _batch(orc, level, 16, 4)
    pk, sk = orc.keygen_batch(level, seeds)
    sig, _, _ = orc.sign_batch(level, sk, msg, off)
    reps = 24
    P = np.repeat(pk, reps, axis=0)
    S = np.repeat(sig, reps, axis=0)
    M = np.concatenate([msg[off[i]:off[i + 1]] for i in range(16) for _ in range(reps)])
    O = np.arange(16 * reps + 1, dtype=np.uint64) * 32
    for t in range(16 * reps):
        kind = t % reps
        if kind == 0:
            continue                                   # untouched
        if kind < 10:                                  # signature bit
            b = rng.integers(0, S.shape[1] * 8)
            S[t, b // 8] ^= 1 << (b % 8)
        elif kind < 14:                                # hint region byte
            p = orc.params(level)
            start = S.shape[1] - p["omega"] - p["k"]
            S[t, start + rng.integers(0, p["omega"] + p["k"])] ^= 1 << rng.integers(0, 8)
        elif kind < 19:                                # public-key bit
            b = rng.integers(0, P.shape[1] * 8)
            P[t, b // 8] ^= 1 << (b % 8)
        else:                                          # message bit
            M[32 * t + rng.integers(0, 32)] ^= 1 << rng.integers(0, 8)
    ok = gpu_verify(ctx, level, P, M, O, S)
    want = orc.verify_batch(level, P, M, O, S)
    assert np.array_equal(ok, want)
    assert ok[::reps].all() and ok.sum() == 16


@pytest.mark.parametrize("level", [2, 3, 5])
def test_verify_rejects_noncanonical_hints(ctx, orc, level):
    """Two encodings of a valid signature's own hint set that a lenient
    decoder would accept (c~ still matches): a nonzero byte in an unused
    index slot, and two indices of one polynomial swapped.  The strict
    decoding of the round-3 hint encoding rejects both, on the GPU exactly as
    in the oracle; the unmodified signatures verify."""
    from gpu_util import gpu_verify
    p = orc.params(level)
    omega, k = p["omega"], p["k"]
    seeds, msg, off = _batch(orc, level, 48, 5)
    pk, sk = orc.keygen_batch(level, seeds)
    sig, _, _ = orc.sign_batch(level, sk, msg, off)
    hoff = sig.shape[1] - omega - k
    rows, kinds = [], []
    for i in range(sig.shape[0]):
        h = sig[i, hoff:]
        counts = [int(c) for c in h[omega:]]
        if counts[-1] < omega:                                  # an unused index slot exists
            t = sig[i].copy()
            t[hoff + counts[-1]] = 1 + (i % 200)
            rows.append((i, t))
            kinds.append("unused")
        prev = 0
        for c in counts:                                        # a polynomial with two or more hints
            if c - prev >= 2:
                t = sig[i].copy()
                t[hoff + prev], t[hoff + prev + 1] = t[hoff + prev + 1], t[hoff + prev]
                rows.append((i, t))
                kinds.append("order")
                break
            prev = c
    assert "unused" in kinds and "order" in kinds
    idx = np.array([r[0] for r in rows])
    S = np.stack([r[1] for r in rows])
    P = pk[idx]
    M = np.concatenate([msg[off[i]:off[i + 1]] for i in idx])
    O = np.zeros(idx.size + 1, dtype=np.uint64)
    O[1:] = np.cumsum([int(off[i + 1] - off[i]) for i in idx])
    want = orc.verify_batch(level, P, M, O, S)
    assert not want.any()                                       # the oracle decodes strictly
    assert not gpu_verify(ctx, level, P, M, O, S).any()
    assert gpu_verify(ctx, level, pk, msg, off, sig).all()


def test_empty_and_single(ctx, orc):
    import torch
    from gpu_util import dev, gpu_keygen, gpu_sign, gpu_verify
    from paper_2211_12265_gb300 import dil
    level = 2
    # n = 0 is a no-op
    dil.dil_keygen(ctx.handle, level, 0, None, None, None)
    seeds = W.seeds(1, 7)
    pk, sk = gpu_keygen(ctx, level, seeds)
    msg = np.zeros(1, dtype=np.uint8)
    off = np.zeros(2, dtype=np.uint64)                 # one empty message
    sig, st, _ = gpu_sign(ctx, level, sk, msg, off)
    osig, ost, _ = orc.sign_batch(level, sk, msg, off)
    assert np.array_equal(sig, osig) and st[0] == 0
    assert gpu_verify(ctx, level, pk, msg, off, sig)[0] == 1


@pytest.mark.parametrize("level", [2, 3, 5])
def test_long_and_empty_messages(ctx, orc, level):
    """Messages of 0 bytes, exactly one and two SHAKE256 blocks around the mu
    hash's boundaries, and 64 KB / 1 MB, mixed in one batch: signatures equal
    the oracle's in the plain, persistent and caller-owned A^ forms and all
    verify (also with the caller's A^); a flipped byte at the end of the
    longest message is rejected."""
    import torch
    from gpu_util import dev, gpu_keygen, gpu_sign, gpu_verify, host
    from paper_2211_12265_gb300 import dil
    lens = np.array([0, 1, 72, 103, 104, 135, 136, 239, 240, 65536, 1 << 20, 0, 5], dtype=np.int64)
    n = lens.size
    rng = np.random.default_rng(31)
    msg = rng.integers(0, 256, int(lens.sum()) + 1, dtype=np.uint8)
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    seeds = W.seeds(n, 70 + level)
    pk, sk = gpu_keygen(ctx, level, seeds)
    sig, st, _ = gpu_sign(ctx, level, sk, msg, off)
    osig, ost, _ = orc.sign_batch(level, sk, msg, off)
    assert np.array_equal(sig, osig) and (st == 0).all()
    assert gpu_verify(ctx, level, pk, msg, off, sig).all()
    bad = msg.copy()
    bad[int(off[11]) - 1] ^= 0x80                       # last byte of the 1 MB message
    ok = gpu_verify(ctx, level, pk, bad, off, sig)
    assert not ok[10] and ok[:10].all() and ok[11:].all()
    # the persistent form and the caller-owned A^ forms on the same batch
    d_sk, d_pk, d_msg, d_off = dev(sk), dev(pk), dev(msg), dev(off)
    psig = torch.full((n, sig.shape[1]), 0x5A, dtype=torch.uint8, device="cuda")
    pst = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    dil.dil_sign_persistent(ctx.handle, [dil.sign_job(level, n, d_sk, d_msg, d_off, psig, pst)])
    k, l = {2: (4, 4), 3: (6, 5), 5: (8, 7)}[level]
    ahat = torch.empty((n, k * l * 256), dtype=torch.int32, device="cuda")
    dil.dil_expand_a(ctx.handle, level, n, d_pk, pk.shape[1], ahat)
    asig = torch.zeros_like(psig)
    ast = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    dil.dil_sign_a(ctx.handle, level, n, d_sk, d_msg, d_off, ahat, asig, ast)
    aok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    dil.dil_verify_a(ctx.handle, level, n, d_pk, dev(bad), d_off, dev(sig), ahat, aok)
    torch.cuda.synchronize()
    assert dil.dil_persistent_status(ctx.handle) == dil.OK
    assert np.array_equal(host(psig), osig) and (host(pst) == 0).all()
    assert np.array_equal(host(asig), osig) and (host(ast) == 0).all()
    assert np.array_equal(host(aok), ok)


def test_iteration_cap(ctx, orc):
    from gpu_util import gpu_sign
    level = 2
    seeds, msg, off = _batch(orc, level, 128, 6)
    _, sk = orc.keygen_batch(level, seeds)
    ctx.set_max_iter(1)
    try:
        sig, st, it = gpu_sign(ctx, level, sk, msg, off)
    finally:
        ctx.set_max_iter(0)
    osig, ost, oit = orc.sign_batch(level, sk, msg, off, max_iter=1)
    assert np.array_equal(st, ost) and np.array_equal(sig, osig) and np.array_equal(it, oit)
    assert (st == -5).any() and (st == 0).any()


def test_chunked_launches_match(orc):
    """A workspace budget smaller than the batch forces several launches; the
    output is unchanged."""
    from gpu_util import gpu_sign
    from paper_2211_12265_gb300 import dil
    level = 5
    seeds, msg, off = _batch(orc, level, 100, 8)
    _, sk = orc.keygen_batch(level, seeds)
    small = dil.Context(0, workspace_budget=13 * 108 * 1024)   # 13 tasks per launch
    try:
        sig, st, _ = gpu_sign(small, level, sk, msg, off)
    finally:
        small.close()
    osig, ost, _ = orc.sign_batch(level, sk, msg, off)
    assert np.array_equal(sig, osig) and np.array_equal(st, ost)


def test_host_forms_match_device_forms(ctx, orc):
    from paper_2211_12265_gb300 import dil
    level = 3
    seeds, msg, off = _batch(orc, level, 64, 9, "uniform", 0, 300)
    pkb, skb, sigb = dil.SIZES[level]
    pk = np.zeros((64, pkb), np.uint8)
    sk = np.zeros((64, skb), np.uint8)
    dil.dil_keygen_host(ctx.handle, level, 64, seeds, pk, sk)
    opk, osk = orc.keygen_batch(level, seeds)
    assert np.array_equal(pk, opk) and np.array_equal(sk, osk)
    sig = np.zeros((64, sigb), np.uint8)
    st = np.zeros(64, np.int32)
    dil.dil_sign_host(ctx.handle, level, 64, sk, msg, off, sig, st)
    osig, _, _ = orc.sign_batch(level, osk, msg, off)
    assert np.array_equal(sig, osig)
    ok = np.zeros(64, np.uint8)
    dil.dil_verify_host(ctx.handle, level, 64, pk, msg, off, sig, ok)
    assert ok.all()


def test_host_pipeline_chunks_match_device_forms(orc):
    """A batch large enough for the chunked two-stream host pipeline (with a
    budget that forces extra, smaller chunks) gives the device forms' bytes;
    sampled tasks against the oracle."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    level, n = 2, 3001                              # 4 ragged chunks
    seeds, msg, off = _batch(orc, level, n, 17, "uniform", 0, 200)
    pkb, skb, sigb = dil.SIZES[level]
    for budget in (0, 300 * dil._sign_scratch_polys(level) * 1024):
        c = dil.Context(0, budget)
        try:
            pk = np.zeros((n, pkb), np.uint8)
            sk = np.zeros((n, skb), np.uint8)
            dil.dil_keygen_host(c.handle, level, n, seeds, pk, sk)
            dpk, dsk = c.keygen(level, dev(seeds))
            assert np.array_equal(pk, host(dpk)) and np.array_equal(sk, host(dsk))
            sig = np.zeros((n, sigb), np.uint8)
            st = np.zeros(n, np.int32)
            dil.dil_sign_host(c.handle, level, n, sk, msg, off, sig, st)
            dsig, dst = c.sign(level, dsk, dev(msg), dev(off))
            assert np.array_equal(sig, host(dsig)) and (st == 0).all()
            bad = sig.copy()
            bad[::5, 7] ^= 4
            ok = np.zeros(n, np.uint8)
            dil.dil_verify_host(c.handle, level, n, pk, msg, off, bad, ok)
            assert np.array_equal(ok.astype(bool), np.arange(n) % 5 != 0)
        finally:
            c.close()
    for i in (0, 751, 1502, 3000):
        _, s, _ = orc.sign(level, sk[i].tobytes(), msg[off[i]:off[i + 1]].tobytes())
        assert s == sig[i].tobytes()


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (4, 2), (4, 4), (8, 4), (8, 1)])
@pytest.mark.parametrize("level", [2, 3, 5])
def test_launch_shapes_bit_exact(orc, level, shape):
    """Every launch shape (warps per CTA, warps per task) gives the oracle's
    bytes: keys, signatures, repetition counts and accept bits."""
    from gpu_util import gpu_keygen, gpu_sign, gpu_verify
    from paper_2211_12265_gb300 import dil
    n = 37                                          # ragged against every group size
    seeds, msg, off = _batch(orc, level, n, 11 + level, "uniform", 0, 900)
    opk, osk = orc.keygen_batch(level, seeds)
    osig, ost, oit = orc.sign_batch(level, osk, msg, off)
    c = dil.Context(0)
    try:
        for op in range(3):
            c.set_tuning(op, shape[0], shape[1])
        pk, sk = gpu_keygen(c, level, seeds)
        sig, st, it = gpu_sign(c, level, osk, msg, off)
        bad = osig.copy()
        bad[::3, 40] ^= 1
        ok = gpu_verify(c, level, opk, msg, off, bad)
    finally:
        c.close()
    assert np.array_equal(pk, opk) and np.array_equal(sk, osk)
    assert np.array_equal(sig, osig) and np.array_equal(it, oit) and np.array_equal(st, ost)
    assert np.array_equal(ok, orc.verify_batch(level, opk, msg, off, bad))


@pytest.mark.parametrize("level", [2, 3, 5])
def test_split_sign_equals_fused(orc, level):
    """The fusion ablation (precompute kernel + two kernels per repetition
    round) gives the fused kernel's signatures, statuses and repetition
    counts, also under a repetition cap; sampled against the oracle."""
    import torch
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    n = 613
    seeds, msg, off = _batch(orc, level, n, 60 + level, "uniform", 0, 700)
    c = dil.Context(0)
    try:
        c.apply_tuning()
        _, sk = c.keygen(level, dev(seeds))
        split = {}
        for cap in (0, 3):
            c.set_max_iter(cap)
            fsig, fst, fit = c.sign(level, sk, dev(msg), dev(off), iterations=True)
            ssig = torch.full_like(fsig, 0x33)
            sst = torch.full_like(fst, 7)
            sit = torch.zeros_like(fit)
            rounds = dil.dil_test_sign_split(c.handle, level, n, sk, dev(msg), dev(off), ssig, sst, sit)
            assert np.array_equal(host(ssig), host(fsig))
            assert np.array_equal(host(sst), host(fst)) and np.array_equal(host(sit), host(fit))
            assert rounds == int(host(fit).max())
            if cap:
                assert (host(fst) == dil.EITER).any() and (host(fst) == 0).any()
            split[cap] = host(ssig)
        c.set_max_iter(0)
        skn = host(sk)
    finally:
        c.close()
    for i in (0, n // 2, n - 1):
        _, s, _ = orc.sign(level, skn[i].tobytes(), msg[off[i]:off[i + 1]].tobytes())
        assert s == split[0][i].tobytes()


def test_decreasing_offsets_rejected(ctx, orc):
    """A task whose message offsets decrease is rejected by the kernels (Sign:
    DIL_EINVAL and a zeroed signature; Verify: 0) without touching the others,
    in the plain, persistent and split forms; the host forms refuse the call."""
    import torch
    from gpu_util import dev, gpu_keygen, gpu_sign, gpu_verify, host
    from paper_2211_12265_gb300 import dil
    level = 2
    seeds = W.seeds(3, 77)
    pk, sk = gpu_keygen(ctx, level, seeds)
    msg = np.arange(64, dtype=np.uint8)
    off = np.array([0, 32, 10, 64], dtype=np.uint64)   # task 1: [32, 10)
    sig, st, _ = gpu_sign(ctx, level, sk, msg, off)
    assert st[1] == dil.EINVAL and not sig[1].any()
    assert st[0] == 0 and st[2] == 0
    for i, (a, b) in ((0, (0, 32)), (2, (10, 64))):
        _, s, _ = orc.sign(level, sk[i].tobytes(), msg[a:b].tobytes())
        assert s == sig[i].tobytes()
    ok = gpu_verify(ctx, level, pk, msg, off, sig)
    assert ok[0] == 1 and ok[1] == 0 and ok[2] == 1
    # persistent and split forms
    dsk, dmsg, doff = dev(sk), dev(msg), dev(off)
    psig = torch.full((3, sig.shape[1]), 7, dtype=torch.uint8, device="cuda")
    pst = torch.full((3,), 9, dtype=torch.int32, device="cuda")
    dil.dil_sign_persistent(ctx.handle, [dil.sign_job(level, 3, dsk, dmsg, doff, psig, pst)])
    assert dil.dil_persistent_status(ctx.handle) == dil.OK
    assert np.array_equal(host(psig), sig) and np.array_equal(host(pst), st)
    ssig = torch.full_like(psig, 5)
    sst = torch.full_like(pst, 9)
    dil.dil_test_sign_split(ctx.handle, level, 3, dsk, dmsg, doff, ssig, sst)
    assert np.array_equal(host(ssig), sig) and np.array_equal(host(sst), st)
    # host forms validate on the host
    with pytest.raises(dil.DilError):
        dil.dil_sign_host(ctx.handle, level, 3, sk, msg, off, np.zeros_like(sig), np.zeros(3, np.int32))
