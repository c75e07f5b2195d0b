"""Caller-owned A^ (dil_expand_a, dil_sign_a, dil_verify_a) against the oracle.

A^ = ExpandA(rho) equals the oracle's matrix for every key, read from a bare
rho array and from a public-key array.  Sign and Verify with that A^ give the
oracle's signatures, statuses, repetition counts and accept bits, with
tampered signatures among the Verify tasks, ragged and empty messages, and a
workspace small enough to split the batch into several launches.  A NULL A^
is the plain form; an A^ of other keys gives signatures that do not verify
and Verify rejects with it.
"""
import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu

LEVELS = (2, 3, 5)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _kl(level):
    return {2: (4, 4), 3: (6, 5), 5: (8, 7)}[level]


@pytest.mark.parametrize("level", LEVELS)
def test_expand_a_matches_oracle(torch_cuda, orc, level):
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    k, l = _kl(level)
    n = 37                                   # several CTAs and a ragged tail
    pk, _sk = orc.keygen_batch(level, W.seeds(n, 70 + level))
    rho = np.ascontiguousarray(pk[:, :32])
    with dil.Context(0) as ctx:
        a1 = torch_cuda.zeros((n, k, l, 256), dtype=torch_cuda.int32, device="cuda")
        a2 = torch_cuda.full((n, k, l, 256), -1, dtype=torch_cuda.int32, device="cuda")
        dil.dil_expand_a(ctx.handle, level, n, dev(rho), 32, a1)
        dil.dil_expand_a(ctx.handle, level, n, dev(pk), pk.shape[1], a2)   # rho at the start of pk
        dil.dil_expand_a(ctx.handle, level, 0, None, 32, None)             # empty batch
        torch_cuda.cuda.synchronize()
        a1, a2 = host(a1), host(a2)
    assert np.array_equal(a1, a2)
    for i in range(n):
        assert np.array_equal(a1[i], orc.expand_a(level, rho[i].tobytes())), i


@pytest.mark.parametrize("level", LEVELS)
def test_sign_and_verify_with_caller_ahat(torch_cuda, orc, level):
    from gpu_util import dev, host
    from paper_2211_12265_gb300 import dil
    k, l = _kl(level)
    n = 150
    pk, sk = orc.keygen_batch(level, W.seeds(n, 80 + level))
    lens = W.message_lengths(n, 80 + level, "uniform", 0, 4096)
    lens[:3] = [0, 1, 4096]
    msg, off = W.messages(lens, 80 + level)
    off = off.astype(np.uint64)
    osig, ost, oit = orc.sign_batch(level, sk, msg, off)
    bad = osig.copy()
    bad[::5, 40] ^= np.uint8(0x10)           # a bit of z in every 5th signature
    ook = orc.verify_batch(level, pk, msg, off, bad)
    assert not ook[::5].any() and ook.sum() == n - len(range(0, n, 5))
    sigb = osig.shape[1]
    # a workspace for a few tasks per launch: the batch runs in several launches
    with dil.Context(0, workspace_budget=4 << 20) as ctx:
        ctx.apply_tuning()
        ahat = torch_cuda.empty((n, k, l, 256), dtype=torch_cuda.int32, device="cuda")
        dil.dil_expand_a(ctx.handle, level, n, dev(pk), pk.shape[1], ahat)
        d_sk, d_pk, d_msg, d_off = dev(sk), dev(pk), dev(msg), dev(off)
        sig = torch_cuda.full((n, sigb), 0x5A, dtype=torch_cuda.uint8, device="cuda")
        st = torch_cuda.full((n,), 9, dtype=torch_cuda.int32, device="cuda")
        it = torch_cuda.zeros(n, dtype=torch_cuda.int32, device="cuda")
        dil.dil_sign_a(ctx.handle, level, n, d_sk, d_msg, d_off, ahat, sig, st, it)
        ok = torch_cuda.full((n,), 7, dtype=torch_cuda.uint8, device="cuda")
        dil.dil_verify_a(ctx.handle, level, n, d_pk, d_msg, d_off, dev(bad), ahat, ok)
        # NULL A^: the plain forms
        sig0 = torch_cuda.zeros_like(sig)
        st0 = torch_cuda.zeros_like(st)
        dil.dil_sign_a(ctx.handle, level, n, d_sk, d_msg, d_off, None, sig0, st0, None)
        ok0 = torch_cuda.zeros_like(ok)
        dil.dil_verify_a(ctx.handle, level, n, d_pk, d_msg, d_off, dev(osig), None, ok0)
        # the A^ of other keys (rolled by one task)
        other = torch_cuda.roll(ahat, 1, 0).contiguous()
        ok_other = torch_cuda.full((n,), 7, dtype=torch_cuda.uint8, device="cuda")
        dil.dil_verify_a(ctx.handle, level, n, d_pk, d_msg, d_off, dev(osig), other, ok_other)
        m = 8
        sig_w = torch_cuda.zeros((m, sigb), dtype=torch_cuda.uint8, device="cuda")
        st_w = torch_cuda.zeros(m, dtype=torch_cuda.int32, device="cuda")
        dil.dil_sign_a(ctx.handle, level, m, d_sk, d_msg, d_off, other, sig_w, st_w, None)
        ok_w = ctx.verify(level, d_pk[:m].contiguous(), d_msg, d_off, sig_w)
        torch_cuda.cuda.synchronize()
        sig, st, it, ok = host(sig), host(st), host(it), host(ok)
        sig0, st0, ok0, ok_other = host(sig0), host(st0), host(ok0), host(ok_other)
        st_w, ok_w = host(st_w), host(ok_w)
    assert np.array_equal(sig, osig) and np.array_equal(st, ost) and np.array_equal(it, oit)
    assert np.array_equal(ok, ook.astype(np.uint8))
    assert np.array_equal(sig0, osig) and np.array_equal(st0, ost) and ok0.all()
    assert not ok_other.any()
    assert (st_w == 0).all() and not ok_w.any()


def test_caller_ahat_argument_errors(torch_cuda):
    from paper_2211_12265_gb300 import dil
    with dil.Context(0) as ctx:
        a = torch_cuda.zeros(4 * 4 * 256 + 4, dtype=torch_cuda.int32, device="cuda")
        rho = torch_cuda.zeros((1, 32), dtype=torch_cuda.uint8, device="cuda")
        with pytest.raises(dil.DilError):
            dil.dil_expand_a(ctx.handle, 2, 1, rho, 16, a)                 # stride below 32
        with pytest.raises(dil.DilError):
            dil.dil_expand_a(ctx.handle, 4, 1, rho, 32, a)                 # no such level
        with pytest.raises(dil.DilError):
            dil.dil_expand_a(ctx.handle, 2, 1, rho, 32, a.data_ptr() + 4)  # not 16-byte aligned
        sk = torch_cuda.zeros((1, 2528), dtype=torch_cuda.uint8, device="cuda")
        off = torch_cuda.zeros(2, dtype=torch_cuda.int64, device="cuda")
        sig = torch_cuda.zeros((1, 2420), dtype=torch_cuda.uint8, device="cuda")
        with pytest.raises(dil.DilError):
            dil.dil_sign_a(ctx.handle, 2, 1, sk, None, off, a.data_ptr() + 4, sig)
