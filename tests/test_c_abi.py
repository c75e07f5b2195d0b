"""The C ABI used from a plain C11 program (tests/c_abi_roundtrip.c): it
compiles against include/dil.h and links libdil.so alone; without a GPU it
gets a clean error from dil_ctx_create; on a GPU its keys, signatures,
statuses and accept bits equal the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2211_12265_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile(tmp_path):
    from paper_2211_12265_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    exe = str(tmp_path / "c_abi_roundtrip")
    subprocess.run([cc, "-std=c11", "-O2", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c_abi_roundtrip.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", os.path.dirname(lib), "-ldil",
                    f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", exe], check=True)
    return exe


def _inputs(tmp_path, n, config):
    seeds = W.seeds(n, config)
    msg, _ = W.messages(W.message_lengths(n, config, "fixed", 32, 32), config)
    path = tmp_path / "in.bin"
    path.write_bytes(seeds.tobytes() + msg.tobytes())
    return seeds, msg, str(path)


def test_c_program_builds_and_fails_cleanly_without_gpu(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: covered by the GPU test")
    exe = _compile(tmp_path)
    _, _, inp = _inputs(tmp_path, 4, 1)
    r = subprocess.run([exe, "2", "4", inp, str(tmp_path / "out.bin")], capture_output=True, text=True)
    assert r.returncode == 3, (r.returncode, r.stderr)     # dil_ctx_create refused: no device
    assert "dil_ctx_create" in r.stderr
    assert subprocess.run([exe, "4", "4", inp, str(tmp_path / "o")]).returncode == 2   # no such level


@pytest.mark.gpu
@pytest.mark.parametrize("level", [2, 3, 5])
def test_c_program_matches_oracle(tmp_path, orc, level):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = _compile(tmp_path)
    n = 300
    seeds, msg, inp = _inputs(tmp_path, n, 90 + level)
    out = tmp_path / "out.bin"
    r = subprocess.run([exe, str(level), str(n), inp, str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    opk, osk = orc.keygen_batch(level, seeds)
    off = np.arange(n + 1, dtype=np.uint64) * 32
    osig, ost, _ = orc.sign_batch(level, osk, msg, off)
    pkb, skb, sigb = opk.shape[1], osk.shape[1], osig.shape[1]
    b = np.frombuffer(out.read_bytes(), dtype=np.uint8)
    sizes = [pkb * n, skb * n, sigb * n, 4 * n, n, n]
    assert b.size == sum(sizes)
    parts = np.split(b, np.cumsum(sizes)[:-1])
    assert np.array_equal(parts[0].reshape(n, pkb), opk)
    assert np.array_equal(parts[1].reshape(n, skb), osk)
    assert np.array_equal(parts[2].reshape(n, sigb), osig)
    assert np.array_equal(parts[3].view(np.int32), ost)
    assert parts[4].all() and not parts[5].any()
