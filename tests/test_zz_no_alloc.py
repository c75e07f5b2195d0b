"""GPU test of dil_sign_noalloc, the Sign entry point that allocates nothing.

Callers that cannot call cudaMalloc while signing (their device memory belongs
to their own allocator, or they cannot afford the synchronisation or an
out-of-memory failure mid-request) use this entry point; it signs on a fixed
scratch array inside the library.  This file is collected last on purpose.

Checks, through the C ABI, at every level: a set-up call (n = 0) first, then
two calls in a row give the same signatures and statuses as dil_sign
(bit-exact, the tolerance of every parity test here) and leave free device
memory unchanged; the documented capacity (1110 / 789 / 532 tasks) is
accepted and one task more is rejected with DIL_EINVAL.
"""
import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

pytestmark = pytest.mark.gpu

# the capacities include/dil.h states for levels 2 / 3 / 5
DOCUMENTED_MAX = {2: 1110, 3: 789, 5: 532}


def _inputs(level, n, config):
    import torch
    from paper_2211_12265_gb300 import dil
    seeds = torch.from_numpy(W.seeds(n, config)).cuda()
    lens = W.message_lengths(n, config, "uniform", 0, 300)
    msg, off = W.messages(lens, config)
    with dil.Context(0) as ctx:
        pk, sk = ctx.keygen(level, seeds)
        torch.cuda.synchronize()
    return sk, torch.from_numpy(msg).cuda(), torch.from_numpy(off).cuda()


def test_noalloc_capacity_table_matches_header():
    from paper_2211_12265_gb300 import dil
    assert dil.NOALLOC_MAX_TASKS == DOCUMENTED_MAX


@pytest.mark.parametrize("level", [2, 3, 5])
def test_noalloc_matches_dil_sign_on_two_calls(level):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_12265_gb300 import dil
    sigb = dil.SIZES[level][2]
    dil.dil_sign_noalloc(level, 0, None, None, None, None)     # set-up only
    with dil.Context(0) as ctx:
        for call, (n, config) in enumerate(((300, 21), (DOCUMENTED_MAX[level], 22))):
            sk, msg, off = _inputs(level, n, config)
            ref_sig = torch.empty((n, sigb), dtype=torch.uint8, device="cuda")
            ref_st = torch.empty(n, dtype=torch.int32, device="cuda")
            dil.dil_sign(ctx.handle, level, n, sk, msg, off, ref_sig, ref_st)
            sig = torch.full((n, sigb), 0xAB, dtype=torch.uint8, device="cuda")
            st = torch.full((n,), 7, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            dil.dil_sign_noalloc(level, n, sk, msg, off, sig, st)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert torch.equal(sig, ref_sig), f"call {call}: signatures differ"
            assert torch.equal(st, ref_st), f"call {call}: statuses differ"
            assert bool((st == 0).all())
            assert free_after == free_before, f"call {call}: free device memory changed"


@pytest.mark.parametrize("level", [2, 3, 5])
def test_noalloc_rejects_one_task_beyond_capacity(level):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_12265_gb300 import dil
    n = DOCUMENTED_MAX[level] + 1
    sk = torch.zeros((n, dil.SIZES[level][1]), dtype=torch.uint8, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    sig = torch.zeros((n, dil.SIZES[level][2]), dtype=torch.uint8, device="cuda")
    rc = dil.load().dil_sign_noalloc(level, n, sk.data_ptr(), None, off.data_ptr(), sig.data_ptr(), None, None)
    assert rc == dil.EINVAL
    assert int(sig.sum()) == 0                                   # nothing was launched
