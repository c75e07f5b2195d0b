"""ctypes binding of the plain C Dilithium oracle (``dil_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product path never
imports this module; it shares no code with the CUDA path.

The oracle computes Alg 1 (Gen), Alg 2 (Sign) and Alg 3 (Verify) of
arXiv 2211.12265 with exact integer arithmetic; see the header of
``dil_oracle.c`` for the readings it takes where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dil_oracle.c")
HDR = os.path.join(HERE, "dil_oracle.h")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

OK = 0
EINVAL = -1
EITER = -5

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, scalar, no intrinsics)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(LIB_PATH)
             or os.path.getmtime(LIB_PATH) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-Wall", "-Wno-unused-function", SRC, "-o", tmp])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.c_void_p
            S = ctypes.c_size_t
            I = ctypes.c_int
            sigs = {
                "orc_sizes": (I, [I, P, P, P]),
                "orc_params": (I, [I, P]),
                "orc_keccak_f1600": (None, [P]),
                "orc_shake128": (None, [P, S, P, S]),
                "orc_shake256": (None, [P, S, P, S]),
                "orc_ntt_def": (None, [P, P]),
                "orc_intt_def": (None, [P, P]),
                "orc_ntt_fast": (None, [P, P]),
                "orc_intt_fast": (None, [P, P]),
                "orc_poly_mul": (None, [P, P, P]),
                "orc_use_def_ntt": (None, [I]),
                "orc_expand_a": (I, [I, P, P]),
                "orc_expand_s": (I, [I, P, P, P]),
                "orc_expand_mask": (I, [I, P, ctypes.c_uint32, P]),
                "orc_sample_in_ball": (I, [I, P, P]),
                "orc_power2round": (None, [S, P, P, P]),
                "orc_decompose": (I, [I, S, P, P, P]),
                "orc_make_hint": (I, [I, S, P, P, P]),
                "orc_use_hint": (I, [I, S, P, P, P]),
                "orc_pack_bits": (None, [S, P, I, P]),
                "orc_unpack_bits": (None, [S, P, I, P]),
                "orc_keygen": (I, [I, P, P, P]),
                "orc_sign": (I, [I, P, P, S, P, I, P]),
                "orc_verify": (I, [I, P, P, S, P]),
                "orc_keygen_batch": (I, [I, S, P, P, P, I]),
                "orc_sign_batch": (I, [I, S, P, P, P, P, P, P, I, I]),
                "orc_verify_batch": (I, [I, S, P, P, P, P, P, I]),
                "orc_counters_reset": (None, []),
                "orc_counters_get": (None, [P]),
            }
            for name, (res, args) in sigs.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(b) -> np.ndarray:
    if isinstance(b, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(b), dtype=np.uint8).copy()
    return np.ascontiguousarray(b, dtype=np.uint8)


# ---------------------------------------------------------------- parameters
def sizes(level: int) -> tuple[int, int, int]:
    pk, sk, sig = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    if lib().orc_sizes(level, ctypes.byref(pk), ctypes.byref(sk), ctypes.byref(sig)) != OK:
        raise ValueError(f"bad level {level}")
    return pk.value, sk.value, sig.value


def params(level: int) -> dict:
    out = np.zeros(10, dtype=np.int64)
    if lib().orc_params(level, _p(out)) != OK:
        raise ValueError(f"bad level {level}")
    keys = ["k", "l", "eta", "tau", "beta", "omega", "gamma1", "gamma2", "d", "q"]
    return {k: int(v) for k, v in zip(keys, out)}


# ---------------------------------------------------------------- hashing
def keccak_f1600(state: np.ndarray) -> np.ndarray:
    st = np.ascontiguousarray(state, dtype=np.uint64).copy()
    lib().orc_keccak_f1600(_p(st))
    return st


def shake128(data: bytes, outlen: int) -> bytes:
    a = _u8(data)
    out = np.zeros(outlen, dtype=np.uint8)
    lib().orc_shake128(_p(a) if a.size else None, a.size, _p(out) if outlen else None, outlen)
    return out.tobytes()


def shake256(data: bytes, outlen: int) -> bytes:
    a = _u8(data)
    out = np.zeros(outlen, dtype=np.uint8)
    lib().orc_shake256(_p(a) if a.size else None, a.size, _p(out) if outlen else None, outlen)
    return out.tobytes()


# ---------------------------------------------------------------- NTT
def _poly_op(fn, a):
    x = np.ascontiguousarray(a, dtype=np.int32)
    assert x.shape == (256,)
    out = np.zeros(256, dtype=np.int32)
    fn(_p(x), _p(out))
    return out


def ntt_def(a):
    return _poly_op(lib().orc_ntt_def, a)


def intt_def(a):
    return _poly_op(lib().orc_intt_def, a)


def ntt(a):
    return _poly_op(lib().orc_ntt_fast, a)


def intt(a):
    return _poly_op(lib().orc_intt_fast, a)


def poly_mul(a, b):
    x = np.ascontiguousarray(a, dtype=np.int32)
    y = np.ascontiguousarray(b, dtype=np.int32)
    out = np.zeros(256, dtype=np.int32)
    lib().orc_poly_mul(_p(x), _p(y), _p(out))
    return out


def use_def_ntt(on: bool) -> None:
    lib().orc_use_def_ntt(1 if on else 0)


# ---------------------------------------------------------------- samplers
def expand_a(level: int, rho: bytes) -> np.ndarray:
    p = params(level)
    out = np.zeros((p["k"], p["l"], 256), dtype=np.int32)
    r = _u8(rho)
    assert r.size == 32
    lib().orc_expand_a(level, _p(r), _p(out))
    return out


def expand_s(level: int, rhop: bytes):
    p = params(level)
    s1 = np.zeros((p["l"], 256), dtype=np.int32)
    s2 = np.zeros((p["k"], 256), dtype=np.int32)
    r = _u8(rhop)
    assert r.size == 64
    lib().orc_expand_s(level, _p(r), _p(s1), _p(s2))
    return s1, s2


def expand_mask(level: int, rhop: bytes, kappa: int) -> np.ndarray:
    p = params(level)
    y = np.zeros((p["l"], 256), dtype=np.int32)
    r = _u8(rhop)
    assert r.size == 64
    lib().orc_expand_mask(level, _p(r), kappa, _p(y))
    return y


def sample_in_ball(level: int, ctilde: bytes) -> np.ndarray:
    c = np.zeros(256, dtype=np.int32)
    r = _u8(ctilde)
    assert r.size == 32
    lib().orc_sample_in_ball(level, _p(r), _p(c))
    return c


# ---------------------------------------------------------------- rounding
def power2round(r):
    x = np.ascontiguousarray(r, dtype=np.int32)
    r1 = np.zeros_like(x)
    r0 = np.zeros_like(x)
    lib().orc_power2round(x.size, _p(x), _p(r1), _p(r0))
    return r1, r0


def decompose(level: int, r):
    x = np.ascontiguousarray(r, dtype=np.int32)
    r1 = np.zeros_like(x)
    r0 = np.zeros_like(x)
    lib().orc_decompose(level, x.size, _p(x), _p(r1), _p(r0))
    return r1, r0


def make_hint(level: int, z, r):
    zz = np.ascontiguousarray(z, dtype=np.int32)
    rr = np.ascontiguousarray(r, dtype=np.int32)
    h = np.zeros(zz.size, dtype=np.uint8)
    lib().orc_make_hint(level, zz.size, _p(zz), _p(rr), _p(h))
    return h


def use_hint(level: int, h, r):
    hh = np.ascontiguousarray(h, dtype=np.uint8)
    rr = np.ascontiguousarray(r, dtype=np.int32)
    out = np.zeros(rr.size, dtype=np.int32)
    lib().orc_use_hint(level, rr.size, _p(hh), _p(rr), _p(out))
    return out


def pack_bits(vals, bits: int) -> bytes:
    v = np.ascontiguousarray(vals, dtype=np.uint32)
    out = np.zeros((v.size * bits + 7) // 8, dtype=np.uint8)
    lib().orc_pack_bits(v.size, _p(v), bits, _p(out))
    return out.tobytes()


def unpack_bits(data: bytes, count: int, bits: int) -> np.ndarray:
    a = _u8(data)
    out = np.zeros(count, dtype=np.uint32)
    lib().orc_unpack_bits(count, _p(a), bits, _p(out))
    return out


# ---------------------------------------------------------------- procedures
def keygen(level: int, seed: bytes) -> tuple[bytes, bytes]:
    pkb, skb, _ = sizes(level)
    s = _u8(seed)
    assert s.size == 32
    pk = np.zeros(pkb, dtype=np.uint8)
    sk = np.zeros(skb, dtype=np.uint8)
    lib().orc_keygen(level, _p(s), _p(pk), _p(sk))
    return pk.tobytes(), sk.tobytes()


def sign(level: int, sk: bytes, msg: bytes, max_iter: int = 0) -> tuple[int, bytes, int]:
    """Returns (status, signature, loop repetitions)."""
    _, skb, sigb = sizes(level)
    s = _u8(sk)
    assert s.size == skb
    m = _u8(msg) if len(msg) else np.zeros(1, dtype=np.uint8)
    sig = np.zeros(sigb, dtype=np.uint8)
    it = ctypes.c_int(0)
    st = lib().orc_sign(level, _p(s), _p(m), len(msg), _p(sig), max_iter, ctypes.byref(it))
    return st, sig.tobytes(), it.value


def verify(level: int, pk: bytes, msg: bytes, sig: bytes) -> bool:
    p = _u8(pk)
    m = _u8(msg) if len(msg) else np.zeros(1, dtype=np.uint8)
    s = _u8(sig)
    return bool(lib().orc_verify(level, _p(p), _p(m), len(msg), _p(s)))


def _threads(nthreads):
    return nthreads if nthreads and nthreads > 0 else (os.cpu_count() or 1)


def keygen_batch(level: int, seeds: np.ndarray, nthreads: int = 0):
    """seeds: uint8 [n, 32] -> (pk [n, PK], sk [n, SK])."""
    seeds = np.ascontiguousarray(seeds, dtype=np.uint8)
    n = seeds.shape[0]
    pkb, skb, _ = sizes(level)
    pk = np.zeros((n, pkb), dtype=np.uint8)
    sk = np.zeros((n, skb), dtype=np.uint8)
    if n:
        lib().orc_keygen_batch(level, n, _p(seeds), _p(pk), _p(sk), _threads(nthreads))
    return pk, sk


def sign_batch(level: int, sk: np.ndarray, msg: np.ndarray, msg_off: np.ndarray,
               max_iter: int = 0, nthreads: int = 0):
    """-> (sig [n, SIG], status [n] int32, iterations [n] int32)."""
    sk = np.ascontiguousarray(sk, dtype=np.uint8)
    n = sk.shape[0]
    _, _, sigb = sizes(level)
    msg = np.ascontiguousarray(msg, dtype=np.uint8)
    if msg.size == 0:
        msg = np.zeros(1, dtype=np.uint8)
    off = np.ascontiguousarray(msg_off, dtype=np.uint64)
    sig = np.zeros((n, sigb), dtype=np.uint8)
    status = np.zeros(n, dtype=np.int32)
    iters = np.zeros(n, dtype=np.int32)
    if n:
        lib().orc_sign_batch(level, n, _p(sk), _p(msg), _p(off), _p(sig), _p(status), _p(iters),
                             max_iter, _threads(nthreads))
    return sig, status, iters


def verify_batch(level: int, pk: np.ndarray, msg: np.ndarray, msg_off: np.ndarray,
                 sig: np.ndarray, nthreads: int = 0) -> np.ndarray:
    pk = np.ascontiguousarray(pk, dtype=np.uint8)
    n = pk.shape[0]
    msg = np.ascontiguousarray(msg, dtype=np.uint8)
    if msg.size == 0:
        msg = np.zeros(1, dtype=np.uint8)
    off = np.ascontiguousarray(msg_off, dtype=np.uint64)
    sig = np.ascontiguousarray(sig, dtype=np.uint8)
    ok = np.zeros(n, dtype=np.uint8)
    if n:
        lib().orc_verify_batch(level, n, _p(pk), _p(msg), _p(off), _p(sig), _p(ok), _threads(nthreads))
    return ok


def counters_reset() -> None:
    lib().orc_counters_reset()


def counters() -> dict:
    out = np.zeros(6, dtype=np.uint64)
    lib().orc_counters_get(_p(out))
    keys = ["permutations", "butterflies", "pointwise", "coefficients", "sign_iterations",
            "r0_form_disagreements"]
    return {k: int(v) for k, v in zip(keys, out)}
