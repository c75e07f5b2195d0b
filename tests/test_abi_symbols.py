"""CPU checks of the C ABI: the library builds and loads, exports every entry
point declared in include/dil.h, answers host-only queries, and refuses to run
without a GPU (there is no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dil_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2211_12265_gb300 import dil
    return dil.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2211_12265_gb300 import dil
    syms = declared_symbols()
    assert len(syms) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", dil.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dil_[a-z0-9_]+)\b", out))
    missing = [s for s in syms if s not in exported]
    assert not missing, missing
    for s in syms:
        assert hasattr(lib, s)


def test_sizes_host_only(lib):
    from paper_2211_12265_gb300 import dil
    assert dil.dil_sizes(2) == (1312, 2528, 2420)
    assert dil.dil_sizes(3) == (1952, 4000, 3293)
    assert dil.dil_sizes(5) == (2592, 4864, 4595)
    with pytest.raises(dil.DilError):
        dil.dil_sizes(4)
    assert dil.status_string(-5) == "sign repetition cap reached"


def test_null_context_rejected(lib):
    from paper_2211_12265_gb300 import dil
    assert lib.dil_keygen(None, 2, 1, None, None, None, None) == dil.EINVAL
    assert lib.dil_sign(None, 2, 1, None, None, None, None, None, None) == dil.EINVAL
    assert lib.dil_verify(None, 2, 1, None, None, None, None, None, None) == dil.EINVAL
    assert lib.dil_ctx_destroy(None) == dil.OK


def test_no_gpu_means_error_not_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    from paper_2211_12265_gb300 import dil
    rc = lib.dil_ctx_create(0, 0, ctypes.byref(h))
    assert rc in (dil.ECUDA, dil.EINVAL) and not h.value
