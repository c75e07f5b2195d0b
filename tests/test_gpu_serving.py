"""Resident-key operations and the continuous-batching server: outputs equal
the plain entry points, and every request's result is the same alone and in
the mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def keys():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_12265_gb300 import serving
    return serving.make_keys((2, 3, 5), n_keys=64)


@pytest.mark.parametrize("sign_shape", [(2, 1), (8, 4), (4, 2)])
def test_keyed_ops_match_plain(keys, orc, sign_shape):
    """Keyed Sign / Verify equal the plain entry points; task groups of more
    than one warp take mu and rho' from the one-warp prepass."""
    import torch
    from paper_2211_12265_gb300 import dil, workload as W
    for level in (2, 3, 5):
        pk, sk = keys[level]
        n = 90
        rng = np.random.default_rng(level)
        kidx = rng.integers(0, pk.shape[0], n).astype(np.int32)
        lens = W.message_lengths(n, 40 + level, "uniform", 0, 2000)
        msg, off = W.messages(lens, 40 + level)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        with dil.Context(0) as ctx:
            ctx.set_tuning(1, sign_shape[0], sign_shape[1], level)
            ks = dil.dil_keystore_create(ctx.handle, level, pk.shape[0], d(pk), d(sk))
            try:
                sig_k = torch.empty((n, dil.SIZES[level][2]), dtype=torch.uint8, device="cuda")
                st_k = torch.empty(n, dtype=torch.int32, device="cuda")
                dil.dil_sign_keyed(ctx.handle, ks, n, d(kidx), d(msg), d(off), sig_k, st_k)
                sig_p, st_p = ctx.sign(level, d(sk[kidx]), d(msg), d(off))
                assert torch.equal(sig_k, sig_p) and torch.equal(st_k, st_p)
                bad = sig_p.clone()
                bad[::4, 50] ^= 8
                ok_k = torch.empty(n, dtype=torch.uint8, device="cuda")
                dil.dil_verify_keyed(ctx.handle, ks, n, d(kidx), d(msg), d(off), bad, ok_k)
                ok_p = ctx.verify(level, d(pk[kidx]), d(msg), d(off), bad)
                assert torch.equal(ok_k, ok_p)
                assert int(ok_k.sum()) == n - len(range(0, n, 4))
                # an unknown key index is rejected, not read
                kb = d(np.array([pk.shape[0], -1], dtype=np.int32))
                st2 = torch.zeros(2, dtype=torch.int32, device="cuda")
                sig2 = torch.full((2, dil.SIZES[level][2]), 7, dtype=torch.uint8, device="cuda")
                dil.dil_sign_keyed(ctx.handle, ks, 2, kb, d(msg), d(off[:3]), sig2, st2)
                assert st2.cpu().tolist() == [-1, -1] and int(sig2.sum()) == 0
                torch.cuda.synchronize()
            finally:
                dil.dil_keystore_destroy(ks)
        # spot-check against the oracle
        for i in range(0, n, 23):
            st, s, _ = orc.sign(level, sk[kidx[i]].tobytes(), msg[off[i]:off[i + 1]].tobytes())
            assert s == sig_k[i].cpu().numpy().tobytes()


def test_server_alone_and_in_the_mix(keys):
    """Every request's result is identical when served alone (one request in
    flight) and when replayed in a burst with the others (continuous batching
    across slots), and equals the plain entry points."""
    from paper_2211_12265_gb300 import serving
    n = 240
    req = serving.serving_workload(keys, n, rate=2e6, seed=3, hi=6000)
    with serving.Server(0, memory_budget=512 << 20, streams=3, max_batch=64) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        mix = srv.replay(req)
        batches, carried, launches = srv.stats()
        assert carried == n and batches >= 3       # several batches, some in flight together
        alone_sig = np.zeros_like(mix["sig"])
        alone_ok = np.zeros_like(mix["ok"])
        alone_st = np.zeros_like(mix["status"])
        for i in range(n):
            m = req["msg"][req["msg_off"][i]:req["msg_off"][i + 1]].tobytes()
            lv = int(req["level"][i])
            sb = {2: 2420, 3: 3293, 5: 4595}[lv]
            sig = req["sig_in"][i, :sb].tobytes() if req["op"][i] == 1 else None
            srv.submit(int(req["op"][i]), lv, int(req["key"][i]), m, sig)
            res = []
            while not res:
                res = srv.poll(4, 100000)
            r = res[0]
            alone_ok[i] = r.ok
            alone_st[i] = r.status
            if req["op"][i] == 0:
                alone_sig[i, :sb] = np.frombuffer(bytes(r.sig), dtype=np.uint8)[:sb]
    sign = req["op"] == 0
    assert np.array_equal(mix["sig"][sign], alone_sig[sign])
    assert np.array_equal(mix["status"][sign], alone_st[sign]) and (mix["status"][sign] == 0).all()
    assert np.array_equal(mix["ok"][~sign], alone_ok[~sign]) and mix["ok"][~sign].all()
    # the signatures made by the server verify and equal dil_sign's (inside serving_workload)
    assert (mix["latency"] > 0).all()


def test_server_admission_small_budget(keys):
    from paper_2211_12265_gb300 import serving
    with serving.Server(0, memory_budget=48 << 20, streams=2, max_batch=4096) as srv:
        assert srv.max_batch < 4096                # shrunk to fit the budget
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        req = serving.serving_workload(keys, 150, rate=1e6, seed=5, hi=3000)
        out = srv.replay(req)
    assert out["ok"][req["op"] == 1].all() and (out["status"][req["op"] == 0] == 0).all()


def test_server_policies_and_shapes_agree(keys):
    """Static batching, continuous batching and other launch shapes of the
    keyed kernels give byte-identical results on the same arrival trace."""
    from paper_2211_12265_gb300 import dil, serving
    req = serving.serving_workload(keys, 200, rate=5e5, seed=9, hi=4000)
    with serving.Server(0, memory_budget=512 << 20, streams=2, max_batch=128) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        base = srv.replay(req)
        srv.set_batching(64, 0.002)
        static = srv.replay(req)
        srv.set_batching(1, 0.0)
        for lv in keys:
            srv.set_tuning(0, lv, 2, 1)
            srv.set_tuning(1, lv, 8, 2)
        shaped = srv.replay(req)
        with pytest.raises(dil.DilError):
            srv.set_tuning(0, 2, 6, 4)             # 4 does not divide 6
        with pytest.raises(dil.DilError):
            srv.set_batching(0, 0.0)
    sign = req["op"] == 0
    for other in (static, shaped):
        assert np.array_equal(base["sig"][sign], other["sig"][sign])
        assert np.array_equal(base["status"], other["status"]) and (base["status"][sign] == 0).all()
        assert np.array_equal(base["ok"][~sign], other["ok"][~sign]) and base["ok"][~sign].all()


def test_server_cancel_pending_requests(keys):
    """Requests held back by a static batching policy can be withdrawn: they
    complete at once with DIL_ECANCELED; the others complete normally with the
    signatures dil_sign gives; unknown and completed ids are refused."""
    import torch
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
    msg = np.frombuffer(b"".join(msgs), dtype=np.uint8)
    kidx = np.arange(n) % pk.shape[0]
    with dil.Context(0) as ctx:
        ref, st = ctx.sign(2, torch.from_numpy(sk[kidx]).cuda(), torch.from_numpy(msg.copy()).cuda(),
                           torch.from_numpy(off).cuda())
        ref = ref.cpu().numpy()
    for i, rid in enumerate(ids):
        status, sig = got[rid]
        if rid in canceled:
            assert status == dil.ECANCELED
        else:
            assert status == dil.OK and sig == ref[i].tobytes()
