"""Helpers for the GPU parity tests: move numpy arrays to the device and run
the C-ABI entry points through the binding."""
import numpy as np
import torch

from paper_2211_12265_gb300 import dil


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def gpu_keygen(ctx, level, seeds):
    pk, sk = ctx.keygen(level, dev(seeds))
    return host(pk), host(sk)


def gpu_sign(ctx, level, sk, msg, off):
    sig, st, it = ctx.sign(level, dev(sk), dev(msg), dev(off.astype(np.uint64)), iterations=True)
    return host(sig), host(st), host(it)


def gpu_verify(ctx, level, pk, msg, off, sig):
    return host(ctx.verify(level, dev(pk), dev(msg), dev(off.astype(np.uint64)), dev(sig)))
