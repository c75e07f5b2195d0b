"""Resident-key operations and the continuous-batching server, against the
oracle.

Every trace here is built without the GPU: key pairs come from the oracle's
Gen, and the signatures carried by Verify requests from the oracle's Sign.
Every third Verify request is tampered with (a flipped bit of z, a changed
hint byte or a changed message byte), so the served accept bits must contain
rejections.  Each served Sign result (status and signature bytes) and each
served accept bit is compared with what the oracle computes for the same
request, under continuous batching, static batching and a small memory
budget; each result is also the same alone and in the mix.
"""
import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu

SIG_STRIDE = 4595
LEVELS = (2, 3, 5)
N_KEYS = 64


def _sig_layout(level):
    """(signature bytes, offset of the hint, omega + k): the round-3 layout
    c~ (32) || z (l polys of 576 / 640 bytes) || h (omega + k bytes)."""
    return {2: (2420, 32 + 4 * 576, 80 + 4), 3: (3293, 32 + 5 * 640, 55 + 6), 5: (4595, 32 + 7 * 640, 75 + 8)}[level]


@pytest.fixture(scope="module")
def keys(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return {lv: orc.keygen_batch(lv, W.seeds(N_KEYS, 60 + lv)) for lv in LEVELS}


def _gather(msg, off, idx):
    """Messages of requests idx as one concatenated array with offsets."""
    parts = [msg[int(off[i]):int(off[i + 1])] for i in idx]
    o = np.zeros(len(idx) + 1, dtype=np.uint64)
    o[1:] = np.cumsum([p.size for p in parts])
    return np.concatenate(parts + [np.zeros(1, np.uint8)]), o


def oracle_trace(orc, keys, n, rate, seed, lo=32, hi=16384):
    """A serving trace (the request layout of dil_server_replay) and the
    oracle's expected result of every request.  Verify requests carry oracle
    signatures; every third one is tampered with, cycling through three kinds."""
    mix = W.request_mix(n, N_KEYS, seed=seed, levels=LEVELS)
    op, level, key = mix["op"].astype(np.int32), mix["level"].astype(np.int32), mix["key"].astype(np.int32)
    lens = W.message_lengths(n, seed, "loguniform", lo, hi)
    msg, off = W.messages(lens, seed)
    msg = msg.copy()
    arrival = W.arrivals(n, rate, seed=seed + 1)
    arrival -= arrival[0]
    sig_in = np.zeros((n, SIG_STRIDE), dtype=np.uint8)
    tamper = np.zeros(n, dtype=np.int32)           # 0 none, 1 z bit, 2 hint byte, 3 message byte
    rng = np.random.default_rng(seed + 2)
    for lv in LEVELS:
        sigb, hoff, hlen = _sig_layout(lv)
        vi = np.nonzero((level == lv) & (op == 1))[0]
        if vi.size:
            m, o = _gather(msg, off, vi)
            sig, st, _ = orc.sign_batch(lv, keys[lv][1][key[vi]], m, o)
            assert (st == 0).all()
            sig_in[vi, :sigb] = sig
    vi_all = np.nonzero(op == 1)[0]
    for j, i in enumerate(vi_all[::3]):
        sigb, hoff, hlen = _sig_layout(int(level[i]))
        kind = 1 + j % 3
        tamper[i] = kind
        if kind == 1:
            sig_in[i, 32 + rng.integers(0, hoff - 32)] ^= np.uint8(1 << rng.integers(0, 8))
        elif kind == 2:
            sig_in[i, hoff + rng.integers(0, hlen)] ^= np.uint8(rng.integers(1, 256))
        else:
            msg[int(off[i]) + rng.integers(0, int(lens[i]))] ^= np.uint8(rng.integers(1, 256))
    exp_sig = np.zeros((n, SIG_STRIDE), dtype=np.uint8)
    exp_status = np.zeros(n, dtype=np.int32)
    exp_ok = np.zeros(n, dtype=np.uint8)
    for lv in LEVELS:
        sigb = _sig_layout(lv)[0]
        si = np.nonzero((level == lv) & (op == 0))[0]
        if si.size:
            m, o = _gather(msg, off, si)
            sig, st, _ = orc.sign_batch(lv, keys[lv][1][key[si]], m, o)
            exp_sig[si, :sigb] = sig
            exp_status[si] = st
        vi = np.nonzero((level == lv) & (op == 1))[0]
        if vi.size:
            m, o = _gather(msg, off, vi)
            exp_ok[vi] = orc.verify_batch(lv, keys[lv][0][key[vi]], m, o, np.ascontiguousarray(sig_in[vi, :sigb]))
    # the tampering is real: the oracle rejects every tampered request and accepts every other one
    verify = op == 1
    assert (exp_ok[verify & (tamper > 0)] == 0).all() and (exp_ok[verify & (tamper == 0)] == 1).all()
    req = {"arrival": np.ascontiguousarray(arrival), "op": op, "level": level, "key": key, "msg": msg,
           "msg_off": off, "sig_in": sig_in, "lengths": lens}
    return req, {"sig": exp_sig, "status": exp_status, "ok": exp_ok, "tamper": tamper}


def assert_matches_oracle(req, out, exp):
    sign, verify = req["op"] == 0, req["op"] == 1
    assert sign.any() and verify.any() and (exp["tamper"][verify] > 0).any()
    assert np.array_equal(out["status"][sign], exp["status"][sign])
    for i in np.nonzero(sign)[0]:
        sigb = _sig_layout(int(req["level"][i]))[0]
        assert np.array_equal(out["sig"][i, :sigb], exp["sig"][i, :sigb]), f"request {i}: signature differs"
    assert np.array_equal(out["ok"][verify], exp["ok"][verify])
    for lv in LEVELS:       # every level served both operations, with rejections among its verifies
        assert ((req["level"] == lv) & sign).any()
        assert ((req["level"] == lv) & verify & (exp["ok"] == 0)).any()


@pytest.mark.parametrize("sign_shape", [(2, 1), (8, 4), (4, 2)])
def test_keyed_ops_match_plain_and_oracle(keys, orc, sign_shape):
    """Keyed Sign / Verify equal the plain entry points and the oracle; task
    groups of more than one warp take mu and rho' from the one-warp prepass."""
    import torch
    from paper_2211_12265_gb300 import dil
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for level in LEVELS:
        pk, sk = keys[level]
        n = 90
        rng = np.random.default_rng(level)
        kidx = rng.integers(0, pk.shape[0], n).astype(np.int32)
        lens = W.message_lengths(n, 40 + level, "uniform", 0, 2000)
        msg, off = W.messages(lens, 40 + level)
        osig, ost, _ = orc.sign_batch(level, sk[kidx], msg, off)
        bad = osig.copy()
        bad[::4, 50] ^= 8
        ook = orc.verify_batch(level, pk[kidx], msg, off, bad)
        with dil.Context(0) as ctx:
            ctx.set_tuning(1, sign_shape[0], sign_shape[1], level)
            ks = dil.dil_keystore_create(ctx.handle, level, pk.shape[0], d(pk), d(sk))
            try:
                sig_k = torch.empty((n, dil.SIZES[level][2]), dtype=torch.uint8, device="cuda")
                st_k = torch.empty(n, dtype=torch.int32, device="cuda")
                dil.dil_sign_keyed(ctx.handle, ks, n, d(kidx), d(msg), d(off), sig_k, st_k)
                sig_p, st_p = ctx.sign(level, d(sk[kidx]), d(msg), d(off))
                assert torch.equal(sig_k, sig_p) and torch.equal(st_k, st_p)
                ok_k = torch.empty(n, dtype=torch.uint8, device="cuda")
                dil.dil_verify_keyed(ctx.handle, ks, n, d(kidx), d(msg), d(off), d(bad), ok_k)
                ok_p = ctx.verify(level, d(pk[kidx]), d(msg), d(off), d(bad))
                assert torch.equal(ok_k, ok_p)
                # an unknown key index is rejected, not read
                kb = d(np.array([pk.shape[0], -1], dtype=np.int32))
                st2 = torch.zeros(2, dtype=torch.int32, device="cuda")
                sig2 = torch.full((2, dil.SIZES[level][2]), 7, dtype=torch.uint8, device="cuda")
                dil.dil_sign_keyed(ctx.handle, ks, 2, kb, d(msg), d(off[:3]), sig2, st2)
                assert st2.cpu().tolist() == [-1, -1] and int(sig2.sum()) == 0
                torch.cuda.synchronize()
            finally:
                dil.dil_keystore_destroy(ks)
        assert np.array_equal(sig_k.cpu().numpy(), osig) and np.array_equal(st_k.cpu().numpy(), ost)
        assert np.array_equal(ok_k.cpu().numpy(), ook) and int(ook.sum()) == n - len(range(0, n, 4))


@pytest.mark.parametrize("setting", ["continuous", "static", "small-budget"])
def test_server_matches_oracle(keys, orc, setting):
    """Every served result equals the oracle's: Sign status and signature
    bytes, Verify accept bits including the tampered requests; all three
    levels, messages of 32 B..16 KB."""
    from paper_2211_12265_gb300 import serving
    budget, streams, max_batch, rate = {"continuous": (512 << 20, 3, 64, 2e6),
                                        "static": (512 << 20, 2, 128, 5e5),
                                        "small-budget": (48 << 20, 2, 4096, 1e6)}[setting]
    req, exp = oracle_trace(orc, keys, 450, rate, seed={"continuous": 301, "static": 302, "small-budget": 303}[setting])
    with serving.Server(0, memory_budget=budget, streams=streams, max_batch=max_batch) as srv:
        if setting == "small-budget":
            assert srv.max_batch < max_batch                 # admission shrank to fit the budget
        if setting == "static":
            srv.set_batching(64, 0.002)
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        out = srv.replay(req)
        batches, carried, _ = srv.stats()
    assert carried == req["op"].size and batches >= 2
    assert_matches_oracle(req, out, exp)
    assert (out["latency"] > 0).all()


def test_server_alone_and_in_the_mix(keys, orc):
    """Every request's result is identical when served alone (one request in
    flight) and when replayed in a burst with the others (continuous batching
    across slots), and both equal the oracle's."""
    from paper_2211_12265_gb300 import serving
    n = 240
    req, exp = oracle_trace(orc, keys, n, 5e4, seed=304, hi=6000)   # arrivals over about 5 ms
    with serving.Server(0, memory_budget=512 << 20, streams=3, max_batch=64) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        mix = srv.replay(req)
        batches, carried, launches = srv.stats()
        assert carried == n and batches >= 3       # admitted in several publications
        # requests joined while others were in flight: some request arrived
        # before an earlier one's result was visible
        done = req["arrival"] + mix["latency"]
        assert (req["arrival"][1:] < np.maximum.accumulate(done)[:-1]).sum() >= n // 4
        alone = {"sig": np.zeros_like(mix["sig"]), "ok": np.zeros_like(mix["ok"]),
                 "status": np.zeros_like(mix["status"])}
        for i in range(n):
            m = req["msg"][req["msg_off"][i]:req["msg_off"][i + 1]].tobytes()
            lv = int(req["level"][i])
            sb = _sig_layout(lv)[0]
            sig = req["sig_in"][i, :sb].tobytes() if req["op"][i] == 1 else None
            srv.submit(int(req["op"][i]), lv, int(req["key"][i]), m, sig)
            res = []
            while not res:
                res = srv.poll(4, 100000)
            r = res[0]
            alone["ok"][i] = r.ok
            alone["status"][i] = r.status
            if req["op"][i] == 0:
                alone["sig"][i, :sb] = np.frombuffer(bytes(r.sig), dtype=np.uint8)[:sb]
    sign = req["op"] == 0
    assert np.array_equal(mix["sig"][sign], alone["sig"][sign])
    assert np.array_equal(mix["status"][sign], alone["status"][sign])
    assert np.array_equal(mix["ok"][~sign], alone["ok"][~sign])
    assert_matches_oracle(req, mix, exp)
    assert (mix["latency"] > 0).all()


def test_server_policies_and_shapes_agree(keys, orc):
    """Continuous batching (the serving kernel), static batching (the keyed
    kernels) and static batching with other launch shapes of the keyed kernels
    give byte-identical results on the same arrival trace, each equal to the
    oracle's."""
    from paper_2211_12265_gb300 import dil, serving
    req, exp = oracle_trace(orc, keys, 200, 5e5, seed=305, hi=4000)
    with serving.Server(0, memory_budget=512 << 20, streams=2, max_batch=128) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        base = srv.replay(req)
        srv.set_batching(64, 0.002)
        static = srv.replay(req)
        for lv in keys:                            # the shapes apply to the static path's keyed kernels
            srv.set_tuning(0, lv, 2, 1)
            srv.set_tuning(1, lv, 8, 2)
        shaped = srv.replay(req)
        srv.set_batching(1, 0.0)
        again = srv.replay(req)
        with pytest.raises(dil.DilError):
            srv.set_tuning(0, 2, 6, 4)             # 4 does not divide 6
        with pytest.raises(dil.DilError):
            srv.set_batching(0, 0.0)
    for out in (base, static, shaped, again):
        assert_matches_oracle(req, out, exp)


def test_server_cancel_pending_requests(keys, orc):
    """Requests held back by a static batching policy can be withdrawn: they
    complete at once with DIL_ECANCELED; the others complete normally with the
    oracle's signatures; unknown and completed ids are refused."""
    from paper_2211_12265_gb300 import dil, serving
    pk, sk = keys[2]
    n = 20
    msgs = [bytes([i]) * (10 + i) for i in range(n)]
    with serving.Server(0, memory_budget=256 << 20, streams=2, max_batch=64) as srv:
        srv.add_keys(2, pk, sk)
        srv.set_batching(10_000, 30.0)            # hold everything back
        ids = [srv.submit(0, 2, i % pk.shape[0], msgs[i]) for i in range(n)]
        canceled = set(ids[::2])
        for rid in sorted(canceled):
            assert srv.cancel(rid)
        assert not srv.cancel(max(ids) + 1000)    # unknown id
        srv.set_batching(1, 0.0)                  # release the rest
        got = {}
        while len(got) < n:
            for r in srv.poll(64, 200000):
                got[r.id] = (r.status, bytes(r.sig)[:2420])
        assert not srv.cancel(ids[1])             # already completed
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(m) for m in msgs])
    msg = np.frombuffer(b"".join(msgs), dtype=np.uint8).copy()
    kidx = np.arange(n) % pk.shape[0]
    ref, st, _ = orc.sign_batch(2, sk[kidx], msg, off)
    for i, rid in enumerate(ids):
        status, sig = got[rid]
        if rid in canceled:
            assert status == dil.ECANCELED
        else:
            assert status == dil.OK and sig == ref[i].tobytes()


@pytest.mark.parametrize("policy", ["continuous", "static"])
def test_server_edge_lengths_and_unknown_keys(keys, orc, policy):
    """Messages of 0 and 1 bytes, around the block edges of mu = H(tr || M)
    (tr is 32 bytes and SHAKE256's rate 136, so M of 103..105 and 239..241
    bytes) and of the server's maximum length, at all levels and for both
    operations, equal the oracle's results; requests naming a key outside the
    store are answered with DIL_EINVAL and a zero signature (Sign) or a reject
    (Verify)."""
    from paper_2211_12265_gb300 import serving
    with serving.Server(0, memory_budget=512 << 20, streams=2, max_batch=256) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        cap = min(int(srv.msg_capacity), 16384)
        edge = [0, 1, 103, 104, 105, 239, 240, 241, cap]
        ops, lvls, lens = [], [], []
        for lv in LEVELS:
            for op in (0, 1):
                for m in edge:
                    ops.append(op)
                    lvls.append(lv)
                    lens.append(m)
        n = len(ops)
        op = np.array(ops, dtype=np.int32)
        level = np.array(lvls, dtype=np.int32)
        lens = np.array(lens, dtype=np.int64)
        key = np.random.default_rng(7).integers(0, N_KEYS, n).astype(np.int32)
        bad = np.zeros(n, dtype=bool)
        bad[5::7] = True                                     # some of each operation and level
        key[bad] = np.where(np.arange(n)[bad] % 2 == 0, N_KEYS, -1)
        msg, off = W.messages(lens, 91)
        sig_in = np.zeros((n, SIG_STRIDE), dtype=np.uint8)
        exp_sig = np.zeros((n, SIG_STRIDE), dtype=np.uint8)
        exp_status = np.zeros(n, dtype=np.int32)
        exp_ok = np.zeros(n, dtype=np.uint8)
        for lv in LEVELS:
            sigb = _sig_layout(lv)[0]
            for o in (0, 1):
                idx = np.nonzero((level == lv) & (op == o) & ~bad)[0]
                m, mo = _gather(msg, off, idx)
                s, st, _ = orc.sign_batch(lv, keys[lv][1][key[idx]], m, mo)
                if o == 0:
                    exp_sig[idx, :sigb] = s
                    exp_status[idx] = st
                else:
                    sig_in[idx, :sigb] = s
                    exp_ok[idx] = orc.verify_batch(lv, keys[lv][0][key[idx]], m, mo, s)
        exp_status[bad & (op == 0)] = -1                     # DIL_EINVAL
        assert exp_ok[(op == 1) & ~bad].all()
        req = {"arrival": np.zeros(n), "op": op, "level": level, "key": key, "msg": msg, "msg_off": off,
               "sig_in": sig_in}
        if policy == "static":
            srv.set_batching(16, 0.002)
        out = srv.replay(req)
    sign = op == 0
    assert np.array_equal(out["status"][sign], exp_status[sign])
    for i in np.nonzero(sign)[0]:
        sigb = _sig_layout(int(level[i]))[0]
        assert np.array_equal(out["sig"][i, :sigb], exp_sig[i, :sigb]), f"request {i} (len {lens[i]})"
    assert np.array_equal(out["ok"][~sign], exp_ok[~sign])
    assert bad[sign].any() and bad[~sign].any()


def test_server_burst_with_precomputed_mu(keys, orc):
    """A burst of 40,000 requests (enough that requests queue for several
    milliseconds and the hasher warps precompute mu = H(tr || M)): every
    result equals the oracle's, with rejections, at all levels, and some
    requests were served with a precomputed mu."""
    from paper_2211_12265_gb300 import dil, serving
    req, exp = oracle_trace(orc, keys, 40000, 1e9, seed=306, hi=1024)
    with serving.Server(0, memory_budget=2 << 30, streams=2, max_batch=4096) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        out = srv.replay(req)
        hashed = dil.dil_test_server_mu_hashed(srv.handle)
    assert_matches_oracle(req, out, exp)
    assert hashed > 0, "no request was served with a precomputed mu"
