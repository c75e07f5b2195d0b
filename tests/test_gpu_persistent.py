"""Persistent Sign (device work queue, speculative nonces, CUDA-graph launch):
outputs equal the plain one-launch form and the oracle byte for byte."""
import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _job_inputs(torch, level, n, config, lo=32, hi=32):
    from paper_2211_12265_gb300 import dil
    seeds = torch.from_numpy(W.seeds(n, config)).cuda()
    lens = W.message_lengths(n, config, "uniform" if hi > lo else "fixed", lo, hi)
    msg, off = W.messages(lens, config)
    with dil.Context(0) as c:
        pk, sk = c.keygen(level, seeds)
        torch.cuda.synchronize()
    return dict(level=level, n=n, sk=sk, msg=torch.from_numpy(msg).cuda(), off=torch.from_numpy(off).cuda(),
                lens=lens, msg_np=msg, off_np=off)


def _plain(torch, j):
    from paper_2211_12265_gb300 import dil
    with dil.Context(0) as c:
        sig, st, it = c.sign(j["level"], j["sk"], j["msg"], j["off"], iterations=True)
        torch.cuda.synchronize()
    return sig.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy()


def _persistent(torch, ctx, jobs, reps=1):
    from paper_2211_12265_gb300 import dil
    outs = []
    for j in jobs:
        sigb = dil.SIZES[j["level"]][2]
        outs.append((torch.full((j["n"], sigb), 0x5A, dtype=torch.uint8, device="cuda"),
                     torch.full((j["n"],), 9, dtype=torch.int32, device="cuda"),
                     torch.zeros(j["n"], dtype=torch.int32, device="cuda")))
    descs = [dil.sign_job(j["level"], j["n"], j["sk"], j["msg"], j["off"], o[0], o[1], o[2])
             for j, o in zip(jobs, outs)]
    for _ in range(reps):
        dil.dil_sign_persistent(ctx.handle, descs)
    assert dil.dil_persistent_status(ctx.handle) == dil.OK
    return [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy()) for o in outs]


@pytest.mark.parametrize("tuning", [(8, 1, 0, 1, 8), (8, 2, 0, 1, 4)])
def test_timed_out_waits_leave_defined_task_outputs(torch_cuda, tuning):
    """A test-only limit of one poll per bounded wait makes the real waits
    (the commit lock, an owner waiting for its helpers) run out under ordinary
    contention.  The launch then reports DIL_ETIMEOUT; every task a wait ran
    out on ends with status DIL_ETIMEOUT, 0 repetitions and a zeroed
    signature; every other task equals the plain form byte for byte; and the
    next launch on the same context, back at the default limit, is normal.
    The waits only return early: nothing here can hang the GPU."""
    from paper_2211_12265_gb300 import dil
    j = _job_inputs(torch_cuda, 2, 12000, 35)        # about 2.5 waves: early tasks have no helpers
    ref_sig, ref_st, ref_it = _plain(torch_cuda, j)
    assert (ref_st == 0).all()
    with dil.Context(0) as ctx:
        dil.dil_set_persistent_tuning(ctx.handle, *tuning)
        dil.dil_test_set_spin_limit(ctx.handle, 1)
        sig = torch_cuda.full((j["n"], dil.SIZES[2][2]), 0x5A, dtype=torch_cuda.uint8, device="cuda")
        st = torch_cuda.full((j["n"],), 9, dtype=torch_cuda.int32, device="cuda")
        it = torch_cuda.full((j["n"],), 77, dtype=torch_cuda.int32, device="cuda")
        desc = [dil.sign_job(2, j["n"], j["sk"], j["msg"], j["off"], sig, st, it)]
        dil.dil_sign_persistent(ctx.handle, desc)
        launch_status = dil.dil_persistent_status(ctx.handle)
        sig_n, st_n, it_n = sig.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy()
        timed = st_n == dil.ETIMEOUT
        assert set(np.unique(st_n).tolist()) <= {dil.OK, dil.ETIMEOUT}
        assert launch_status == (dil.ETIMEOUT if timed.any() else dil.OK)
        assert timed.any(), "no wait ran out: the test did not reach the timeout path"
        assert (sig_n[timed] == 0).all() and (it_n[timed] == 0).all()
        done = ~timed
        assert done.sum() > j["n"] // 4
        assert np.array_equal(sig_n[done], ref_sig[done]) and np.array_equal(it_n[done], ref_it[done])
        dil.dil_test_set_spin_limit(ctx.handle, 0)
        (got,) = _persistent(torch_cuda, ctx, [j])
    for a, b in zip(got, (ref_sig, ref_st, ref_it)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tuning", [(8, 2, 0, 1, 4), (4, 1, 0, 1, 0), (4, 1, 0, 3, 2), (8, 4, 2, 2, 8),
                                    (2, 2, 1, 1, 1), (8, 1, 0, 1, 8), (1, 1, 0, 1, 16)])
def test_single_job_matches_plain(torch_cuda, tuning):
    from paper_2211_12265_gb300 import dil
    j = _job_inputs(torch_cuda, 2, 700, 31)
    ref = _plain(torch_cuda, j)
    with dil.Context(0) as ctx:
        dil.dil_set_persistent_tuning(ctx.handle, *tuning)
        (got,) = _persistent(torch_cuda, ctx, [j])
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_mixed_levels_match_plain_and_oracle(torch_cuda, orc):
    from paper_2211_12265_gb300 import dil
    jobs = [_job_inputs(torch_cuda, 2, 300, 32, 0, 1500), _job_inputs(torch_cuda, 5, 211, 33, 0, 4096),
            _job_inputs(torch_cuda, 3, 97, 34, 32, 64)]
    with dil.Context(0) as ctx:
        got = _persistent(torch_cuda, ctx, jobs, reps=2)   # second call replays the captured graph
    for j, g in zip(jobs, got):
        ref = _plain(torch_cuda, j)
        for a, b in zip(g, ref):
            assert np.array_equal(a, b)
        sk = j["sk"].cpu().numpy()
        idx = np.arange(0, j["n"], 17)
        for i in idx:
            m = j["msg_np"][j["off_np"][i]:j["off_np"][i + 1]].tobytes()
            st, sig, it = orc.sign(j["level"], sk[i].tobytes(), m)
            assert st == g[1][i] and it == g[2][i] and sig == g[0][i].tobytes()


def test_graph_recaptured_when_arguments_change(torch_cuda):
    from paper_2211_12265_gb300 import dil
    a = _job_inputs(torch_cuda, 2, 150, 35)
    b = _job_inputs(torch_cuda, 2, 90, 36)
    with dil.Context(0) as ctx:
        ga = _persistent(torch_cuda, ctx, [a])
        gb = _persistent(torch_cuda, ctx, [b])
        ga2 = _persistent(torch_cuda, ctx, [a])
    for x, y in zip(ga[0], _plain(torch_cuda, a)):
        assert np.array_equal(x, y)
    for x, y in zip(gb[0], _plain(torch_cuda, b)):
        assert np.array_equal(x, y)
    for x, y in zip(ga[0], ga2[0]):
        assert np.array_equal(x, y)


def test_repetition_cap_with_speculation(torch_cuda, orc):
    from paper_2211_12265_gb300 import dil
    j = _job_inputs(torch_cuda, 2, 256, 37)
    sk = j["sk"].cpu().numpy()
    osig, ost, oit = orc.sign_batch(2, sk, j["msg_np"], j["off_np"], max_iter=2)
    with dil.Context(0) as ctx:
        ctx.set_max_iter(2)
        dil.dil_set_persistent_tuning(ctx.handle, 8, 2, 0, 1, 8)
        (got,) = _persistent(torch_cuda, ctx, [j])
    assert np.array_equal(got[1], ost) and np.array_equal(got[0], osig) and np.array_equal(got[2], oit)
    assert (ost == -5).any() and (ost == 0).any()


def test_cancel_running_launch(torch_cuda):
    """A host cancel during a long launch: every task ends either signed
    exactly as the plain form signs it, or DIL_ECANCELED with a zero
    signature; the next launch on the same context runs to completion."""
    import time
    from paper_2211_12265_gb300 import dil
    torch = torch_cuda
    n = 400_000
    j = _job_inputs(torch, 2, n, 38)
    with dil.Context(0) as ctx:
        assert dil.dil_persistent_cancel(ctx.handle) == dil.OK   # nothing launched yet: no effect
        sig = torch.full((n, dil.SIZES[2][2]), 0x5A, dtype=torch.uint8, device="cuda")
        st = torch.full((n,), 9, dtype=torch.int32, device="cuda")
        it = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        desc = dil.sign_job(2, n, j["sk"], j["msg"], j["off"], sig, st, it)
        dil.dil_sign_persistent(ctx.handle, [desc])
        time.sleep(0.02)
        assert dil.dil_persistent_cancel(ctx.handle) == dil.OK
        assert dil.dil_persistent_status(ctx.handle) == dil.ECANCELED
        s, g, i = st.cpu().numpy(), sig.cpu().numpy(), it.cpu().numpy()
        ok, canceled = s == dil.OK, s == dil.ECANCELED
        assert (ok | canceled).all()
        assert ok.sum() > 0 and canceled.sum() > 0
        assert not g[canceled].any() and not i[canceled].any()
        rsig, rst, rit = _plain(torch, j)
        assert np.array_equal(g[ok], rsig[ok]) and np.array_equal(i[ok], rit[ok])
        # the context is reusable and the next launch starts with the word cleared
        small = _job_inputs(torch, 2, 500, 39)
        (got,) = _persistent(torch, ctx, [small])
    for a, b in zip(got, _plain(torch, small)):
        assert np.array_equal(a, b)


def test_empty_job_among_others(torch_cuda):
    """A job with no tasks between two others: the launch signs the others
    exactly as the plain form does (task indices skip the empty job)."""
    from paper_2211_12265_gb300 import dil
    a = _job_inputs(torch_cuda, 2, 120, 40)
    c = _job_inputs(torch_cuda, 3, 70, 41, 0, 900)
    empty = dict(level=5, n=0, sk=a["sk"][:0], msg=a["msg"][:0], off=a["off"][:1])
    with dil.Context(0) as ctx:
        got = _persistent(torch_cuda, ctx, [a, empty, c])
    for j, g in ((a, got[0]), (c, got[2])):
        for x, y in zip(g, _plain(torch_cuda, j)):
            assert np.array_equal(x, y)
    assert got[1][0].size == 0
