"""Failure detection without faulting the GPU: a bounded device wait on a flag
nothing clears returns DIL_ETIMEOUT and the context keeps working; the Sign
repetition cap returns DIL_EITER per task; bad arguments are refused on the
host before any launch."""
import numpy as np
import pytest

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


def test_bounded_wait_times_out_and_context_survives(ctx, orc):
    from gpu_util import gpu_keygen, gpu_sign
    from paper_2211_12265_gb300 import dil, workload as W
    assert dil.dil_test_bounded_wait(ctx.handle, 0, 1000) == dil.OK
    assert dil.dil_test_bounded_wait(ctx.handle, 1, 20000) == dil.ETIMEOUT      # ~2.5 ms, nothing clears it
    seeds = W.seeds(8, 77)
    pk, sk = gpu_keygen(ctx, 2, seeds)
    msg, off = W.messages(np.full(8, 32), 77)
    sig, st, _ = gpu_sign(ctx, 2, sk, msg, off)
    osig, _, _ = orc.sign_batch(2, sk, msg, off)
    assert np.array_equal(sig, osig)


def test_host_side_refusals(ctx):
    import torch
    from paper_2211_12265_gb300 import dil
    L = dil.load()
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    assert L.dil_sign(ctx.handle, 4, 1, buf.data_ptr(), None, buf.data_ptr(), buf.data_ptr(), None, None) == dil.EINVAL
    assert L.dil_verify(ctx.handle, 2, 1, None, None, None, None, None, None) == dil.EINVAL
    assert L.dil_set_tuning(ctx.handle, 1, 0, 3, 2) == dil.EINVAL          # 3 warps not a multiple of 2
    assert L.dil_set_persistent_tuning(ctx.handle, 8, 3, 0, 1, 4) == dil.EINVAL
    small = dil.Context(0, workspace_budget=1024)                          # cannot hold one task
    try:
        with pytest.raises(dil.DilError) as e:
            dil.dil_sign(small.handle, 2, 1, buf, buf, torch.zeros(2, dtype=torch.int64, device="cuda"), buf)
        assert e.value.status == dil.ENOMEM
    finally:
        small.close()
