"""Project autotuner: launch shapes per security level.

For the plain kernels it sweeps, per level and operation, the warps per CTA
and the warps per task (32 x warps-per-task threads share one task's
polynomials: the paper's single-warp and four-warp forms, section 3.1); for
the persistent Sign it also sweeps CTAs per SM, the queue chunk (fresh tasks
per queue access) and the speculation slots (helper groups per unfinished
task, section 4.3).  Every candidate is timed with CUDA events on a probe
batch (L2 flushed before each timing, median of several) and the fastest is
kept.  The result is a JSON table keyed by GPU name; ``apply`` installs it on
a context.  ``tuning_gb300.json`` next to this file is the table measured on
GB300 and is applied by default.
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning_gb300.json")

PLAIN_SHAPES = [(1, 1), (2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (8, 2), (4, 4), (8, 4)]
PERSIST_SHAPES = [(4, 1, 0, 1, 4), (8, 1, 0, 1, 0), (8, 1, 0, 1, 4), (8, 1, 0, 1, 8), (8, 1, 0, 1, 16),
                  (8, 1, 0, 2, 8), (8, 2, 0, 1, 4), (8, 2, 0, 1, 8), (8, 4, 0, 1, 4), (8, 4, 0, 1, 8)]
OPS = {"keygen": 0, "sign": 1, "verify": 2}


def _timer(torch, flush):
    def timeit(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]
    return timeit


def _persistent_sweep(dil, ctx, jobs, timeit, n_tasks, label, log) -> dict:
    best = None
    for shape in PERSIST_SHAPES:
        dil.dil_set_persistent_tuning(ctx.handle, *shape)
        t = timeit(lambda: dil.dil_sign_persistent(ctx.handle, jobs))
        assert dil.dil_persistent_status(ctx.handle) == dil.OK
        log(f"{label} sign   persistent {shape}: {n_tasks / t * 1e3:11.0f}/s")
        if best is None or t < best[1]:
            best = (shape, t)
    s = best[0]
    return {"warps_per_cta": s[0], "warps_per_task": s[1], "ctas_per_sm": s[2], "chunk": s[3], "speculation": s[4],
            "ops_s": n_tasks / best[1] * 1e3}


def tune(levels=(2, 3, 5), n: int = 10000, device: int = 0, log=print, mixed_n: int = 100000) -> dict:
    """Measures every candidate shape; returns the table of the fastest.  The
    persistent Sign is tuned per level on n tasks and, as "mixed", on one
    launch of mixed_n Dilithium2 plus mixed_n Dilithium5 tasks."""
    import numpy as np
    import torch

    from . import dil
    from . import workload as W
    torch.cuda.set_device(device)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    timeit = _timer(torch, flush)
    table = {"gpu": torch.cuda.get_device_name(device), "probe_tasks": n, "plain": {}, "persistent": {}}
    with dil.Context(device) as ctx:
        for level in levels:
            w = W.workload(2 if level == 2 else 3, n)
            seeds = torch.from_numpy(w["seeds"]).cuda()
            msg = torch.from_numpy(w["msg"]).cuda()
            off = torch.from_numpy(w["msg_off"]).cuda()
            pk, sk = ctx.keygen(level, seeds)
            sig, st = ctx.sign(level, sk, msg, off)
            ok = torch.empty(n, dtype=torch.uint8, device="cuda")
            runs = {"keygen": lambda: dil.dil_keygen(ctx.handle, level, n, seeds, pk, sk),
                    "sign": lambda: dil.dil_sign(ctx.handle, level, n, sk, msg, off, sig, st),
                    "verify": lambda: dil.dil_verify(ctx.handle, level, n, pk, msg, off, sig, ok)}
            table["plain"][str(level)] = {}
            for name, fn in runs.items():
                best = None
                for shape in PLAIN_SHAPES:
                    ctx.set_tuning(OPS[name], shape[0], shape[1], level)
                    t = timeit(fn)
                    log(f"level {level} {name:6s} plain {shape}: {n / t * 1e3:11.0f}/s")
                    if best is None or t < best[1]:
                        best = (shape, t)
                ctx.set_tuning(OPS[name], best[0][0], best[0][1], level)
                table["plain"][str(level)][name] = {"warps_per_cta": best[0][0], "warps_per_task": best[0][1],
                                                    "ops_s": n / best[1] * 1e3}
            job = [dil.sign_job(level, n, sk, msg, off, sig, st)]
            table["persistent"][str(level)] = _persistent_sweep(dil, ctx, job, timeit, n, f"level {level}", log)
        if mixed_n and {2, 5} <= set(levels):
            jobs, keep = [], []
            for level in (2, 5):
                w = W.workload(4, mixed_n)
                seeds = torch.from_numpy(W.seeds(mixed_n, 4 + level)).cuda()
                msg = torch.from_numpy(w["msg"]).cuda()
                off = torch.from_numpy(w["msg_off"]).cuda()
                pk, sk = ctx.keygen(level, seeds)
                sig = torch.empty((mixed_n, dil.SIZES[level][2]), dtype=torch.uint8, device="cuda")
                st = torch.empty(mixed_n, dtype=torch.int32, device="cuda")
                keep.append((sk, msg, off, sig, st))
                jobs.append(dil.sign_job(level, mixed_n, sk, msg, off, sig, st))
            table["persistent"]["mixed"] = _persistent_sweep(dil, ctx, jobs, timeit, 2 * mixed_n, "levels 2+5", log)
    return table


def load(path: str | None = None) -> dict | None:
    path = path or DEFAULT_TABLE
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def save(table: dict, path: str | None = None) -> str:
    path = path or DEFAULT_TABLE
    with open(path, "w") as f:
        json.dump(table, f, indent=1)
    return path


def apply(ctx, table: dict | None = None, persistent_level: int | str | None = None) -> None:
    """Installs the plain shapes of every level and the persistent shape of
    `persistent_level` (a level, or "mixed" for launches that mix levels;
    default: "mixed" when tuned, else the slowest level) on a dil.Context."""
    from . import dil
    table = table or load()
    if not table:
        return
    for level, ops in table.get("plain", {}).items():
        for name, v in ops.items():
            ctx.set_tuning(OPS[name], v["warps_per_cta"], v["warps_per_task"], int(level))
    pers = table.get("persistent", {})
    if pers:
        if persistent_level and str(persistent_level) in pers:
            lv = str(persistent_level)
        elif "mixed" in pers:
            lv = "mixed"
        else:
            lv = max((k for k in pers if k.isdigit()), key=int)
        v = pers[lv]
        dil.dil_set_persistent_tuning(ctx.handle, v["warps_per_cta"], v["warps_per_task"], v["ctas_per_sm"],
                                      v["chunk"], v["speculation"])


if __name__ == "__main__":
    import sys
    out = sys.argv[1] if len(sys.argv) > 1 else None
    print(save(tune(), out))
