"""ctypes binding of the C ABI in ``include/dil.h`` (argument marshalling only).

Module-level functions carry the C entry points' names and signatures; device
buffers may be passed as ``torch.Tensor`` (CUDA, contiguous), as raw integer
device pointers, or as ``None`` for nullable arguments.  ``Context`` wraps a
``dil_ctx`` and adds allocating conveniences built on the same calls.

There is no fallback: if ``libdil.so`` cannot be loaded (or built with nvcc),
every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EITER, ECANCELED = 0, -1, -2, -3, -4, -5, -6
SIZES = {2: (1312, 2528, 2420), 3: (1952, 4000, 3293), 5: (2592, 4864, 4595)}
PARAMS = {2: dict(k=4, l=4), 3: dict(k=6, l=5), 5: dict(k=8, l=7)}

_lock = threading.Lock()
_lib = None


class DilError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Loads libdil.so (building it with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libdil.so missing at {path}")
            L = ctypes.CDLL(path)
            P, S, I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
            sigs = {
                "dil_sizes": [I, P, P, P],
                "dil_ctx_create": [I, S, P],
                "dil_ctx_destroy": [P],
                "dil_set_max_iter": [P, I],
                "dil_set_tuning": [P, I, I, I, I],
                "dil_keygen": [P, I, S, P, P, P, P],
                "dil_sign": [P, I, S, P, P, P, P, P, P],
                "dil_sign_ex": [P, I, S, P, P, P, P, P, P, P],
                "dil_verify": [P, I, S, P, P, P, P, P, P],
                "dil_sign_noalloc": [I, S, P, P, P, P, P, P],
                "dil_expand_a": [P, I, S, P, S, P, P],
                "dil_sign_a": [P, I, S, P, P, P, P, P, P, P, P],
                "dil_verify_a": [P, I, S, P, P, P, P, P, P, P],
                "dil_keygen_host": [P, I, S, P, P, P, P],
                "dil_sign_host": [P, I, S, P, P, P, P, P, P],
                "dil_verify_host": [P, I, S, P, P, P, P, P, P],
                "dil_test_shake": [P, I, S, P, P, P, S, P],
                "dil_test_ntt": [P, S, P, P, I, P],
                "dil_test_keccak_f": [P, I, S, P, P, P],
                "dil_test_k16_rider": [P, S, P, P, P, P, P],
                "dil_test_k16_chain_rider": [P, S, P, P, P, P, P, P],
                "dil_test_t0_ntt": [P, I, I, S, P, P, P],
                "dil_test_sample_in_ball_stream": [P, I, S, P, I, P, P],
                "dil_test_expand_a": [P, I, S, P, P, P],
                "dil_test_expand_s": [P, I, S, P, P, P],
                "dil_test_expand_mask": [P, I, S, P, P, P, P],
                "dil_test_sample_in_ball": [P, I, S, P, P, P],
                "dil_test_rounding": [P, I, S, P, P, P, P, P],
                "dil_test_issue_rate": [P, I, P],
                "dil_test_keccak_rate": [P, I, P],
                "dil_test_sign_split": [P, I, S, P, P, P, P, P, P, P, P],
                "dil_test_bounded_wait": [P, I, I, P],
                "dil_test_set_spin_limit": [P, I],
                "dil_sign_persistent": [P, I, P, P],
                "dil_set_persistent_tuning": [P, I, I, I, I, I],
                "dil_persistent_status": [P, P],
                "dil_persistent_cancel": [P],
                "dil_keystore_create": [P, I, S, P, P, P, P],
                "dil_keystore_destroy": [P],
                "dil_sign_keyed": [P, P, S, P, P, P, P, P, P],
                "dil_verify_keyed": [P, P, S, P, P, P, P, P, P],
                "dil_server_create": [I, S, I, I, P],
                "dil_server_destroy": [P],
                "dil_server_limits": [P, P, P],
                "dil_server_set_batching": [P, I, ctypes.c_double],
                "dil_server_set_tuning": [P, I, I, I, I],
                "dil_server_add_keys": [P, I, S, P, P],
                "dil_server_submit": [P, I, I, ctypes.c_int32, P, S, P, P],
                "dil_server_poll": [P, P, S, P, I],
                "dil_server_cancel": [P, ctypes.c_uint64],
                "dil_server_replay": [P, S, P, P, P, P, P, P, P, P, P, P, P, P],
                "dil_server_stats": [P, P, P, P],
                "dil_test_server_mu_hashed": [P, P],
            }
            for name, args in sigs.items():
                f = getattr(L, name)
                f.restype = I
                f.argtypes = args
            L.dil_status_string.restype = ctypes.c_char_p
            L.dil_status_string.argtypes = [I]
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return load().dil_status_string(status).decode()


def _ptr(x):
    """Device or host address of a tensor / array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc: int, what: str) -> int:
    if rc != OK:
        raise DilError(rc, what)
    return rc


# ----------------------------------------------------------------- C names
def dil_sizes(level: int) -> tuple[int, int, int]:
    pk, sk, sig = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().dil_sizes(level, ctypes.byref(pk), ctypes.byref(sk), ctypes.byref(sig)), "dil_sizes")
    return pk.value, sk.value, sig.value


def dil_ctx_create(device: int = 0, workspace_budget: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().dil_ctx_create(device, workspace_budget, ctypes.byref(h)), "dil_ctx_create")
    return h.value


def dil_ctx_destroy(ctx: int) -> None:
    _check(load().dil_ctx_destroy(ctx), "dil_ctx_destroy")


def dil_set_max_iter(ctx: int, max_iter: int) -> None:
    _check(load().dil_set_max_iter(ctx, max_iter), "dil_set_max_iter")


def dil_set_tuning(ctx: int, op: int, warps_per_cta: int, warps_per_task: int = 1, level: int = 0) -> None:
    _check(load().dil_set_tuning(ctx, op, level, warps_per_cta, warps_per_task), "dil_set_tuning")


def dil_keygen(ctx, level, n, seeds, pk, sk, stream=None):
    return _check(load().dil_keygen(ctx, level, n, _ptr(seeds), _ptr(pk), _ptr(sk), _stream(stream)), "dil_keygen")


def dil_sign(ctx, level, n, sk, msg, msg_off, sig, task_status=None, stream=None):
    return _check(load().dil_sign(ctx, level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                  _ptr(task_status), _stream(stream)), "dil_sign")


def dil_sign_ex(ctx, level, n, sk, msg, msg_off, sig, task_status=None, iterations=None, stream=None):
    return _check(load().dil_sign_ex(ctx, level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                     _ptr(task_status), _ptr(iterations), _stream(stream)), "dil_sign_ex")


def dil_verify(ctx, level, n, pk, msg, msg_off, sig, ok, stream=None):
    return _check(load().dil_verify(ctx, level, n, _ptr(pk), _ptr(msg), _ptr(msg_off), _ptr(sig), _ptr(ok),
                                    _stream(stream)), "dil_verify")


def dil_expand_a(ctx, level, n, rho, rho_stride, ahat, stream=None):
    """A^ = ExpandA(rho) of n keys into ahat (n x k x l x 256 words)."""
    return _check(load().dil_expand_a(ctx, level, n, _ptr(rho), rho_stride, _ptr(ahat), _stream(stream)),
                  "dil_expand_a")


def dil_sign_a(ctx, level, n, sk, msg, msg_off, ahat, sig, task_status=None, iterations=None, stream=None):
    """dil_sign_ex with each task's A^ taken from ahat (None: dil_sign_ex)."""
    return _check(load().dil_sign_a(ctx, level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(ahat), _ptr(sig),
                                    _ptr(task_status), _ptr(iterations), _stream(stream)), "dil_sign_a")


def dil_verify_a(ctx, level, n, pk, msg, msg_off, sig, ahat, ok, stream=None):
    """dil_verify with each task's A^ taken from ahat (None: dil_verify)."""
    return _check(load().dil_verify_a(ctx, level, n, _ptr(pk), _ptr(msg), _ptr(msg_off), _ptr(sig), _ptr(ahat),
                                      _ptr(ok), _stream(stream)), "dil_verify_a")


def dil_sign_noalloc(level, n, sk, msg, msg_off, sig, task_status=None, stream=None):
    """Sign on the library's static scratch (no allocation; see dil.h)."""
    return _check(load().dil_sign_noalloc(level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                          _ptr(task_status), _stream(stream)), "dil_sign_noalloc")


def _sign_scratch_polys(level: int) -> int:
    """Per-task scratch of the plain Sign kernel in polynomials: A^, s^1, s^2,
    t^0, then the mask ring (l + 15: masks are sampled sixteen nonces at a
    time), y^, w and z."""
    k, l = {2: (4, 4), 3: (6, 5), 5: (8, 7)}[level]
    return k * l + l + 2 * k + (l + 15) + l + k + l


# Largest batch dil_sign_noalloc accepts: its 64 MiB static scratch over the
# per-task scratch.
NOALLOC_MAX_TASKS = {lv: (64 << 20) // (_sign_scratch_polys(lv) * 1024) for lv in (2, 3, 5)}


def dil_keygen_host(ctx, level, n, seeds, pk, sk, stream=None):
    return _check(load().dil_keygen_host(ctx, level, n, _ptr(seeds), _ptr(pk), _ptr(sk), _stream(stream)),
                  "dil_keygen_host")


def dil_sign_host(ctx, level, n, sk, msg, msg_off, sig, task_status=None, stream=None):
    return _check(load().dil_sign_host(ctx, level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                       _ptr(task_status), _stream(stream)), "dil_sign_host")


def dil_verify_host(ctx, level, n, pk, msg, msg_off, sig, ok, stream=None):
    return _check(load().dil_verify_host(ctx, level, n, _ptr(pk), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                         _ptr(ok), _stream(stream)), "dil_verify_host")


def dil_test_shake(ctx, kind, n, inp, in_off, out, outlen, stream=None):
    return _check(load().dil_test_shake(ctx, kind, n, _ptr(inp), _ptr(in_off), _ptr(out), outlen,
                                        _stream(stream)), "dil_test_shake")


def dil_test_keccak_f(ctx, form, n, inp, out, stream=None):
    return _check(load().dil_test_keccak_f(ctx, int(form), n, _ptr(inp), _ptr(out), _stream(stream)),
                  "dil_test_keccak_f")


def dil_test_k16_rider(ctx, n, inp, in_off, perms, out, stream=None):
    return _check(load().dil_test_k16_rider(ctx, n, _ptr(inp), _ptr(in_off), _ptr(perms), _ptr(out),
                                            _stream(stream)), "dil_test_k16_rider")


def dil_test_k16_chain_rider(ctx, n, inp, in_off, perms, step, out, stream=None):
    return _check(load().dil_test_k16_chain_rider(ctx, n, _ptr(inp), _ptr(in_off), _ptr(perms), _ptr(step), _ptr(out),
                                                  _stream(stream)), "dil_test_k16_chain_rider")


def dil_test_sample_in_ball_stream(ctx, level, n, data, blocks, out, stream=None):
    return _check(load().dil_test_sample_in_ball_stream(ctx, int(level), n, _ptr(data), int(blocks), _ptr(out),
                                                        _stream(stream)), "dil_test_sample_in_ball_stream")


def dil_test_t0_ntt(ctx, level, variant, n, sk, out, stream=None):
    return _check(load().dil_test_t0_ntt(ctx, int(level), int(variant), n, _ptr(sk), _ptr(out), _stream(stream)),
                  "dil_test_t0_ntt")


def dil_test_ntt(ctx, n, inp, out, inverse, stream=None):
    return _check(load().dil_test_ntt(ctx, n, _ptr(inp), _ptr(out), int(inverse), _stream(stream)), "dil_test_ntt")


def dil_test_expand_a(ctx, level, n, rho, ahat, stream=None):
    return _check(load().dil_test_expand_a(ctx, level, n, _ptr(rho), _ptr(ahat), _stream(stream)),
                  "dil_test_expand_a")


def dil_test_expand_s(ctx, level, n, rhop, s, stream=None):
    return _check(load().dil_test_expand_s(ctx, level, n, _ptr(rhop), _ptr(s), _stream(stream)),
                  "dil_test_expand_s")


def dil_test_expand_mask(ctx, level, n, rhop, kappa, y, stream=None):
    return _check(load().dil_test_expand_mask(ctx, level, n, _ptr(rhop), _ptr(kappa), _ptr(y), _stream(stream)),
                  "dil_test_expand_mask")


def dil_test_sample_in_ball(ctx, level, n, ctilde, c, stream=None):
    return _check(load().dil_test_sample_in_ball(ctx, level, n, _ptr(ctilde), _ptr(c), _stream(stream)),
                  "dil_test_sample_in_ball")


def dil_test_rounding(ctx, level, n, r, z, h, out, stream=None):
    return _check(load().dil_test_rounding(ctx, level, n, _ptr(r), _ptr(z), _ptr(h), _ptr(out),
                                           _stream(stream)), "dil_test_rounding")


def dil_test_issue_rate(ctx, op: int) -> float:
    """Thread-ops per SM clock of one integer instruction class (see dil.h)."""
    r = ctypes.c_double()
    _check(load().dil_test_issue_rate(ctx, op, ctypes.byref(r)), "dil_test_issue_rate")
    return r.value


def dil_test_sign_split(ctx, level, n, sk, msg, msg_off, sig, task_status=None, iterations=None,
                        stream=None) -> int:
    """Sign split into kernels (fusion ablation; see dil.h); returns the rounds run."""
    r = ctypes.c_int()
    _check(load().dil_test_sign_split(ctx, level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                      _ptr(task_status), _ptr(iterations), ctypes.byref(r), _stream(stream)),
           "dil_test_sign_split")
    return r.value


def dil_test_keccak_rate(ctx, form: int) -> float:
    """SM clocks per state per round of a Keccak-f form (1, 2 or 6; see dil.h)."""
    r = ctypes.c_double()
    _check(load().dil_test_keccak_rate(ctx, form, ctypes.byref(r)), "dil_test_keccak_rate")
    return r.value


def dil_test_bounded_wait(ctx, flag_value: int, limit: int) -> int:
    r = ctypes.c_int()
    _check(load().dil_test_bounded_wait(ctx, flag_value, limit, ctypes.byref(r)), "dil_test_bounded_wait")
    return r.value


def dil_test_set_spin_limit(ctx, limit: int) -> None:
    """Polls per bounded device wait of later persistent launches (0 = default)."""
    _check(load().dil_test_set_spin_limit(ctx, int(limit)), "dil_test_set_spin_limit")


ISSUE_OPS = {"lop3": 0, "shf": 1, "imul": 2, "imul_hi": 3, "shfl": 4}


class SignJob(ctypes.Structure):
    """dil_sign_job: one batch of Sign tasks of one level (device pointers)."""
    _fields_ = [("level", ctypes.c_int), ("n", ctypes.c_size_t), ("sk", ctypes.c_void_p),
                ("msg", ctypes.c_void_p), ("msg_off", ctypes.c_void_p), ("sig", ctypes.c_void_p),
                ("task_status", ctypes.c_void_p), ("iterations", ctypes.c_void_p)]


def sign_job(level, n, sk, msg, msg_off, sig, task_status=None, iterations=None) -> SignJob:
    return SignJob(level, n, _ptr(sk), _ptr(msg), _ptr(msg_off), _ptr(sig), _ptr(task_status), _ptr(iterations))


def dil_sign_persistent(ctx, jobs, stream=None):
    arr = (SignJob * len(jobs))(*jobs)
    return _check(load().dil_sign_persistent(ctx, len(jobs), arr, _stream(stream)), "dil_sign_persistent")


def dil_set_persistent_tuning(ctx, warps_per_cta=8, warps_per_task=2, ctas_per_sm=0, chunk=1, speculation=4):
    return _check(load().dil_set_persistent_tuning(ctx, warps_per_cta, warps_per_task, ctas_per_sm, chunk,
                                                   speculation), "dil_set_persistent_tuning")


def dil_persistent_status(ctx, stream=None) -> int:
    return load().dil_persistent_status(ctx, _stream(stream))


def dil_persistent_cancel(ctx) -> int:
    return load().dil_persistent_cancel(ctx)


def dil_keystore_create(ctx, level, n_keys, pk, sk=None, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().dil_keystore_create(ctx, level, n_keys, _ptr(pk), _ptr(sk), ctypes.byref(h), _stream(stream)),
           "dil_keystore_create")
    return h.value


def dil_keystore_destroy(ks) -> None:
    _check(load().dil_keystore_destroy(ks), "dil_keystore_destroy")


def dil_sign_keyed(ctx, ks, n, key_idx, msg, msg_off, sig, task_status=None, stream=None):
    return _check(load().dil_sign_keyed(ctx, ks, n, _ptr(key_idx), _ptr(msg), _ptr(msg_off), _ptr(sig),
                                        _ptr(task_status), _stream(stream)), "dil_sign_keyed")


def dil_verify_keyed(ctx, ks, n, key_idx, msg, msg_off, sig, ok, stream=None):
    return _check(load().dil_verify_keyed(ctx, ks, n, _ptr(key_idx), _ptr(msg), _ptr(msg_off), _ptr(sig), _ptr(ok),
                                          _stream(stream)), "dil_verify_keyed")


class DilResult(ctypes.Structure):
    """dil_result: one completed serving request."""
    _fields_ = [("id", ctypes.c_uint64), ("op", ctypes.c_int32), ("level", ctypes.c_int32),
                ("status", ctypes.c_int32), ("ok", ctypes.c_uint8), ("sig", ctypes.c_uint8 * 4595),
                ("latency_s", ctypes.c_double)]


def dil_server_create(device=0, memory_budget=0, streams=4, max_batch=2048) -> int:
    h = ctypes.c_void_p()
    _check(load().dil_server_create(device, memory_budget, streams, max_batch, ctypes.byref(h)), "dil_server_create")
    return h.value


def dil_server_destroy(srv) -> None:
    _check(load().dil_server_destroy(srv), "dil_server_destroy")


def dil_server_limits(srv) -> tuple[int, int]:
    mb, mc = ctypes.c_int(), ctypes.c_size_t()
    _check(load().dil_server_limits(srv, ctypes.byref(mb), ctypes.byref(mc)), "dil_server_limits")
    return mb.value, mc.value


def dil_server_set_batching(srv, min_batch: int, max_wait_s: float) -> None:
    _check(load().dil_server_set_batching(srv, min_batch, max_wait_s), "dil_server_set_batching")


def dil_server_set_tuning(srv, op: int, level: int, warps_per_cta: int, warps_per_task: int) -> None:
    _check(load().dil_server_set_tuning(srv, op, level, warps_per_cta, warps_per_task), "dil_server_set_tuning")


def dil_server_add_keys(srv, level, n, pk, sk) -> None:
    _check(load().dil_server_add_keys(srv, level, n, _ptr(pk), _ptr(sk)), "dil_server_add_keys")


def dil_server_submit(srv, op, level, key, msg: bytes, sig: bytes | None = None) -> int:
    rid = ctypes.c_uint64()
    m = (ctypes.c_uint8 * max(len(msg), 1)).from_buffer_copy(msg or b"\0")
    sg = (ctypes.c_uint8 * len(sig)).from_buffer_copy(sig) if sig is not None else None
    _check(load().dil_server_submit(srv, op, level, key, m, len(msg), sg, ctypes.byref(rid)), "dil_server_submit")
    return rid.value


def dil_server_cancel(srv, rid: int) -> int:
    """DIL_OK when request `rid` was still pending and is now canceled, else
    DIL_EINVAL (unknown or already dispatched); does not raise."""
    return load().dil_server_cancel(srv, rid)


def dil_server_poll(srv, max_n=256, wait_us=1000) -> list:
    out = (DilResult * max_n)()
    n = ctypes.c_size_t()
    _check(load().dil_server_poll(srv, out, max_n, ctypes.byref(n), wait_us), "dil_server_poll")
    return [out[i] for i in range(n.value)]


def dil_server_replay(srv, n, arrival_s, op, level, key, msg, msg_off, sig_in, sig_out, status, ok, latency_s):
    wall = ctypes.c_double()
    _check(load().dil_server_replay(srv, n, _ptr(arrival_s), _ptr(op), _ptr(level), _ptr(key), _ptr(msg),
                                    _ptr(msg_off), _ptr(sig_in), _ptr(sig_out), _ptr(status), _ptr(ok),
                                    _ptr(latency_s), ctypes.byref(wall)), "dil_server_replay")
    return wall.value


def dil_server_stats(srv) -> tuple[int, int, int]:
    """(batches, requests, kernel launches) since the server was created."""
    b, r, k = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().dil_server_stats(srv, ctypes.byref(b), ctypes.byref(r), ctypes.byref(k)), "dil_server_stats")
    return b.value, r.value, k.value


def dil_test_server_mu_hashed(srv) -> int:
    """Requests served with a precomputed mu since the server was created."""
    c = ctypes.c_uint64()
    _check(load().dil_test_server_mu_hashed(srv, ctypes.byref(c)), "dil_test_server_mu_hashed")
    return c.value


# ----------------------------------------------------------------- wrapper
class Context:
    """Owns a dil_ctx.  Methods take and return torch CUDA tensors."""

    def __init__(self, device: int = 0, workspace_budget: int = 0):
        self.device = device
        self.handle = dil_ctx_create(device, workspace_budget)

    def close(self) -> None:
        if self.handle:
            dil_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, op: int, warps_per_cta: int, warps_per_task: int = 1, level: int = 0) -> None:
        dil_set_tuning(self.handle, op, warps_per_cta, warps_per_task, level)

    def apply_tuning(self, table: dict | None = None) -> None:
        """Applies an autotuner table (see autotune.py; the committed GB300
        table by default)."""
        from . import autotune
        autotune.apply(self, table)

    def set_max_iter(self, max_iter: int) -> None:
        dil_set_max_iter(self.handle, max_iter)

    def _dev(self):
        import torch
        return torch.device("cuda", self.device)

    def keygen(self, level: int, seeds, stream=None):
        import torch
        n = seeds.shape[0]
        pkb, skb, _ = SIZES[level]
        pk = torch.empty((n, pkb), dtype=torch.uint8, device=self._dev())
        sk = torch.empty((n, skb), dtype=torch.uint8, device=self._dev())
        dil_keygen(self.handle, level, n, seeds, pk, sk, stream)
        return pk, sk

    def sign(self, level: int, sk, msg, msg_off, stream=None, iterations: bool = False):
        import torch
        n = sk.shape[0]
        sig = torch.empty((n, SIZES[level][2]), dtype=torch.uint8, device=self._dev())
        status = torch.empty(n, dtype=torch.int32, device=self._dev())
        its = torch.empty(n, dtype=torch.int32, device=self._dev()) if iterations else None
        dil_sign_ex(self.handle, level, n, sk, msg if msg.numel() else None, msg_off, sig, status, its, stream)
        return (sig, status, its) if iterations else (sig, status)

    def verify(self, level: int, pk, msg, msg_off, sig, stream=None):
        import torch
        n = pk.shape[0]
        ok = torch.empty(n, dtype=torch.uint8, device=self._dev())
        dil_verify(self.handle, level, n, pk, msg if msg.numel() else None, msg_off, sig, ok, stream)
        return ok
