"""Parity at the benchmark's full sizes and in its launch configuration (the
committed tuning table), against the oracle run on all host cores.

  config 2: Dilithium2, 10,000 tasks, 32-byte messages
  config 3: Dilithium3 and Dilithium5, 10,000 tasks each, messages 32 B-4 KB
      every task's pk, sk, signature, status, repetition count and accept bit
      equals the oracle's, for the plain form and the persistent form; the
      oracle's own signatures, tampered in every 7th (a bit of z) and every
      11th (a hint byte) task, get the oracle's accept bits
  config 4: 100,000 Dilithium2 + 100,000 Dilithium5 signatures in one
      persistent launch: every task equals the plain form byte for byte and
      every signature is accepted (Verify(Sign(m)) = 1 is fixed by the scheme);
      a 1-in-16 sample of tasks (keys, signature bytes, repetition counts)
      equals the oracle's
"""
import time

import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_12265_gb300 import dil
    c = dil.Context(0)
    c.apply_tuning()
    yield torch, c
    c.close()


def _tamper(sig, level):
    """Every 7th signature with one flipped bit of z, every 11th with a changed
    hint byte (the round-3 layout: c~ (32) || z || h (omega + k bytes))."""
    hoff, hlen = {2: (32 + 4 * 576, 84), 3: (32 + 5 * 640, 61), 5: (32 + 7 * 640, 83)}[level]
    bad = sig.copy()
    n = sig.shape[0]
    idx7 = np.arange(0, n, 7)
    bad[idx7, 32 + (idx7 * 131) % (hoff - 32)] ^= np.uint8(1 << 3)
    idx11 = np.arange(5, n, 11)
    bad[idx11, hoff + (idx11 * 17) % hlen] ^= np.uint8(0x5A)
    tampered = np.zeros(n, dtype=bool)
    tampered[idx7] = tampered[idx11] = True
    return bad, tampered


@pytest.mark.parametrize("level,config", [(2, 2), (3, 3), (5, 3)])
def test_full_size_every_byte(tctx, orc, level, config):
    torch, c = tctx
    from paper_2211_12265_gb300 import autotune, dil
    n = 10000
    w = W.workload(config, n)
    lens = w["lengths"]
    assert lens.min() >= 32 and (config == 2 or lens.max() > 3000)
    t0 = time.perf_counter()
    opk, osk = orc.keygen_batch(level, w["seeds"])
    osig, ost, oit = orc.sign_batch(level, osk, w["msg"], w["msg_off"])
    bad, tampered = _tamper(osig, level)
    ook_bad = orc.verify_batch(level, opk, w["msg"], w["msg_off"], bad)
    oracle_s = time.perf_counter() - t0
    assert (ost == 0).all() and np.array_equal(ook_bad.astype(bool), ~tampered)   # the tampering is real

    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    seeds, msg, off = d(w["seeds"]), d(w["msg"]), d(w["msg_off"])
    pk, sk = c.keygen(level, seeds)
    sig, st, it = c.sign(level, sk, msg, off, iterations=True)
    ok = c.verify(level, pk, msg, off, sig)
    ok_bad = c.verify(level, pk, msg, off, d(bad))
    # the persistent form of the same batch, in the shape the benchmark times
    autotune.apply(c, persistent_level=level)
    psig = torch.full_like(sig, 0x5A)
    pst = torch.full_like(st, 9)
    pit = torch.zeros_like(it)
    dil.dil_sign_persistent(c.handle, [dil.sign_job(level, n, sk, msg, off, psig, pst, pit)])
    assert dil.dil_persistent_status(c.handle) == dil.OK
    torch.cuda.synchronize()
    h = lambda t: t.cpu().numpy()
    assert np.array_equal(h(pk), opk) and np.array_equal(h(sk), osk)
    assert np.array_equal(h(sig), osig) and np.array_equal(h(st), ost) and np.array_equal(h(it), oit)
    assert h(ok).all()
    assert np.array_equal(h(ok_bad), ook_bad)
    assert np.array_equal(h(psig), osig) and np.array_equal(h(pst), ost) and np.array_equal(h(pit), oit)
    print(f"\noracle (keygen, sign, verify of {n} Dilithium{level} tasks): {oracle_s:.1f} s")


def test_persistent_config4_equals_plain(tctx, orc):
    torch, c = tctx
    from paper_2211_12265_gb300 import autotune, dil
    n = 100000
    autotune.apply(c, persistent_level="mixed")
    jobs, outs, plain, inputs = [], [], [], []
    for level in (2, 5):
        w = W.workload(4, n)
        seeds_np = W.seeds(n, 4 + level)
        seeds = torch.from_numpy(seeds_np).cuda()
        msg = torch.from_numpy(w["msg"]).cuda()
        off = torch.from_numpy(w["msg_off"]).cuda()
        pk, sk = c.keygen(level, seeds)
        sigb = dil.SIZES[level][2]
        o = (torch.full((n, sigb), 0x5A, dtype=torch.uint8, device="cuda"),
             torch.full((n,), 9, dtype=torch.int32, device="cuda"),
             torch.zeros(n, dtype=torch.int32, device="cuda"))
        outs.append(o)
        jobs.append(dil.sign_job(level, n, sk, msg, off, *o))   # raw device pointers: keep the tensors alive
        plain.append(c.sign(level, sk, msg, off, iterations=True))
        inputs.append((level, pk, seeds_np, w, msg, off))
    dil.dil_sign_persistent(c.handle, jobs)
    assert dil.dil_persistent_status(c.handle) == dil.OK
    oks = [c.verify(level, pk, msg, off, o[0]) for (level, pk, _s, _w, msg, off), o in zip(inputs, outs)]
    torch.cuda.synchronize()
    for (level, pk, seeds_np, w, _msg, _off), o, p, okv in zip(inputs, outs, plain, oks):
        psig, pst, pit = (t.cpu().numpy() for t in p)
        sig, st, it = (t.cpu().numpy() for t in o)
        assert (st == 0).all() and (pst == 0).all()
        assert np.array_equal(sig, psig) and np.array_equal(it, pit)
        assert okv.cpu().numpy().all()                       # every task's accept bit
        sample = np.arange(level, n, 16)                     # 1 in 16
        opk, osk = orc.keygen_batch(level, seeds_np[sample])
        m, so = [], [0]
        for i in sample:
            m.append(w["msg"][w["msg_off"][i]:w["msg_off"][i + 1]])
            so.append(so[-1] + m[-1].size)
        osig, ost, oit = orc.sign_batch(level, osk, np.concatenate(m), np.array(so, dtype=np.uint64))
        assert np.array_equal(pk.cpu().numpy()[sample], opk)
        assert np.array_equal(sig[sample], osig) and np.array_equal(it[sample], oit) and (ost == 0).all()
