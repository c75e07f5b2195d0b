"""The paper's speedup breakdown of t^0 = NTT(t0) in Sign (section 5,
"Speedup Breakdown"), re-measured on this GPU: unpack and transform as two
kernels through global memory, then fused, then with t0 kept in registers,
then with the bank-conflict-free exchange layout (the form Sign uses).
Every variant is timed with CUDA events on the same keys, L2 flushed before
each launch, median of several.  Usage:
``python -m paper_2211_12265_gb300.breakdown [level] [tasks] [--once]``
(``--once``: each variant launched once, for a profiler capture).
"""
from __future__ import annotations

import json
import sys

VARIANTS = {0: "unpack kernel + NTT kernel, t0 through global memory",
            1: "one fused kernel, t0 still through global memory",
            2: "one kernel, t0 in registers, exchange with bank conflicts",
            3: "one kernel, t0 in registers, conflict-free exchange"}


def measure(level: int = 2, n: int = 100_000, reps: int = 9, device: int = 0) -> dict:
    import numpy as np
    import torch

    from . import dil
    from . import workload as W
    torch.cuda.set_device(device)
    k = {2: 4, 3: 6, 5: 8}[level]
    with dil.Context(device) as ctx:
        _, sk = ctx.keygen(level, torch.from_numpy(W.seeds(n, 70 + level)).cuda())
        out = torch.empty((n, k, 256), dtype=torch.int32, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        rows = {}
        for variant, what in VARIANTS.items():
            dil.dil_test_t0_ntt(ctx.handle, level, variant, n, sk, out)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                dil.dil_test_t0_ntt(ctx.handle, level, variant, n, sk, out)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = float(np.median(ts))
            rows[variant] = {"what": what, "ms": ms, "polys_per_s": n * k / (ms * 1e-3)}
    base = rows[0]["ms"]
    for r in rows.values():
        r["speedup_vs_0"] = base / r["ms"]
    return {"level": level, "tasks": n, "polynomials": n * k, "variants": rows}


def run_once(level: int, n: int, device: int = 0) -> None:
    """Each variant launched once, nothing else (for a profiler capture)."""
    import torch

    from . import dil
    from . import workload as W
    k = {2: 4, 3: 6, 5: 8}[level]
    with dil.Context(device) as ctx:
        _, sk = ctx.keygen(level, torch.from_numpy(W.seeds(n, 70 + level)).cuda())
        out = torch.empty((n, k, 256), dtype=torch.int32, device="cuda")
        for variant in VARIANTS:
            dil.dil_test_t0_ntt(ctx.handle, level, variant, n, sk, out)
        torch.cuda.synchronize()


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    lv = int(args[0]) if args else 2
    nn = int(args[1]) if len(args) > 1 else 100_000
    if "--once" in sys.argv:
        run_once(lv, nn)
    else:
        print(json.dumps(measure(lv, nn), indent=1))
