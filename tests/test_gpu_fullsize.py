"""Parity at the benchmark's full sizes and in its launch configuration (the
committed tuning table): every output is checked by a property that holds at
any size, and a sample of tasks against the oracle one by one.

  config 2: Dilithium2, 10,000 tasks, 32-byte messages (plain form)
  config 3: Dilithium3 and Dilithium5, 10,000 tasks each, messages 32 B-4 KB
  config 4: 100,000 Dilithium2 + 100,000 Dilithium5 signatures in one
            persistent launch, equal to the plain form task by task
"""
import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu

SAMPLE = 24


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


def _sample(n, seed):
    return np.unique(np.concatenate([[0, n - 1], np.random.default_rng(seed).integers(0, n, SAMPLE)]))


@pytest.mark.parametrize("level,config", [(2, 2), (3, 3), (5, 3)])
def test_plain_full_size(tctx, orc, level, config):
    torch, c = tctx
    n = 10000
    w = W.workload(config, n)
    seeds = torch.from_numpy(w["seeds"]).cuda()
    msg = torch.from_numpy(w["msg"]).cuda()
    off = torch.from_numpy(w["msg_off"]).cuda()
    pk, sk = c.keygen(level, seeds)
    sig, st, it = c.sign(level, sk, msg, off, iterations=True)
    ok = c.verify(level, pk, msg, off, sig)
    bad = sig.clone()
    bad[::7, 100] ^= 1                                   # one flipped bit in z of every 7th signature
    ok_bad = c.verify(level, pk, msg, off, bad)
    torch.cuda.synchronize()
    pk, sk, sig = pk.cpu().numpy(), sk.cpu().numpy(), sig.cpu().numpy()
    st, it = st.cpu().numpy(), it.cpu().numpy()
    assert (st == 0).all() and ok.cpu().numpy().all()
    assert np.array_equal(ok_bad.cpu().numpy().astype(bool), np.arange(n) % 7 != 0)
    lens = w["lengths"]
    assert lens.min() >= 32 and (config == 2 or lens.max() > 3000)
    for i in _sample(n, level):
        m = w["msg"][w["msg_off"][i]:w["msg_off"][i + 1]].tobytes()
        opk, osk = orc.keygen(level, w["seeds"][i].tobytes())
        assert pk[i].tobytes() == opk and sk[i].tobytes() == osk, i
        ost, osig, oit = orc.sign(level, osk, m)
        assert ost == 0 and sig[i].tobytes() == osig and it[i] == oit, i


def test_persistent_config4_equals_plain(tctx, orc):
    torch, c = tctx
    from paper_2211_12265_gb300 import dil
    n = 100000
    jobs, outs, plain, inputs = [], [], [], []
    for level in (2, 5):
        w = W.workload(4, n)
        seeds = torch.from_numpy(W.seeds(n, 4 + level)).cuda()
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
        inputs.append((level, sk, w, msg, off))
    dil.dil_sign_persistent(c.handle, jobs)
    assert dil.dil_persistent_status(c.handle) == dil.OK
    torch.cuda.synchronize()
    for (level, sk, w, _msg, _off), o, p in zip(inputs, outs, plain):
        psig, pst, pit = (t.cpu().numpy() for t in p)
        sig, st, it = (t.cpu().numpy() for t in o)
        assert (st == 0).all() and (pst == 0).all()
        assert np.array_equal(sig, psig) and np.array_equal(it, pit)
        skn = sk.cpu().numpy()
        for i in _sample(n, 40 + level)[:8]:
            m = w["msg"][w["msg_off"][i]:w["msg_off"][i + 1]].tobytes()
            ost, osig, oit = orc.sign(level, skn[i].tobytes(), m)
            assert sig[i].tobytes() == osig and it[i] == oit, (level, i)
