#!/usr/bin/env python3
"""Benchmark of the batched Dilithium engine on GB300.

Default workload (one "step"): Dilithium2, 10,000 independent tasks with
distinct seeded key pairs and 32-byte messages; Sign of the whole batch (one
launch) followed by Verify of the resulting signatures (one launch), plain
one-launch-per-phase form.  Inputs are resident in HBM when timing starts and
L2 is flushed (512 MiB write) before every step.  ``value`` is
(signs + verifies) per second over all ranks; ``e2e`` is the same through the
host-buffer C entry points with the copies inside the timed region.

The same line carries every other benchmark configuration, each measured
in the same run:
  * ``forms``: the persistent form of Sign on the same batch (device work
    queue, speculative nonces, CUDA graph), the split-kernel ablation,
    ``caller_ahat``: Sign and Verify of the batch reading the keys' A^ from
    dil_expand_a (and that expansion's rate), and
    ``level3`` / ``level5``: Dilithium3 and Dilithium5, 10,000 tasks each with
    messages of 32..4096 bytes, plain and persistent Sign, Verify, KeyGen;
    ``mixed_200k``: persistent Sign of 100,000 Dilithium2 + 100,000
    Dilithium5 tasks in one launch against the plain one-launch-per-level
    form;
  * ``served``: the continuous-batching server over 4096 resident keys per
    level (mixed 60% verify / 40% sign requests of all levels, messages
    32 B..16 KB, Poisson arrivals): saturated ops/s, an arrival-rate sweep
    with p50/p99 latency, at each rate the best p99 of the static-batching
    service over a grid of (min_batch, max_wait), and the plain kernels'
    rate on the same requests (one launch per operation and level).

``--workload level3|level5|mixed|serving`` runs one of those alone with its
own JSON line.

``--impl reference`` times the CPU oracle (test infrastructure) on a bounded
sample of the same workload on the host cores.

Multi-GPU: tasks are independent, so N ranks run N replicas of the workload
(weak scaling, no collective on the data path); the step time is the maximum
over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_12265_gb300 import work as WK  # noqa: E402
from paper_2211_12265_gb300 import workload as W  # noqa: E402

METRIC = "Dilithium2/3/5 sign & verify ops/s on 1 GB300; served p50/p99 latency"
PAPER_A100 = {2: {"sign_ops_s": 574953, "verify_ops_s": 1408703},
              3: {"sign_ops_s": 396360, "verify_ops_s": 982648},
              5: {"sign_ops_s": 315900, "verify_ops_s": 637299}}
SMS = 152
SM_MAX_MHZ = 2070.0
# Integer-issue ceiling of one SM: 4 SM sub-partitions, each issuing at most one
# warp instruction (32 thread-operations) per clock.  The ALU pipe alone (LOP3,
# shifts) takes 2 warp instructions per SM clock (64 thread-ops), as ncu's
# sm__inst_executed_pipe_alu.avg.peak_sustained reads on GB300.
ISSUE_THREAD_OPS_PER_SM_CLK = 128
L2_FLUSH_BYTES = 512 << 20

# static batching (the plain one-launch-per-batch service): grid searched per arrival rate
STATIC_GRID = [(mb, w) for mb in (128, 512, 2048) for w in (0.0005, 0.002, 0.008)]
SERVED_FRACTIONS = (0.25, 0.5, 0.75, 0.9)
SERVED_REPLAYS = 3   # continuous batching: median of this many replays of each trace

WORKLOADS = {
    "level2": dict(level=2, n=10000, config=2),
    "level3": dict(level=3, n=10000, config=3),
    "level5": dict(level=5, n=10000, config=3),
    "mixed": dict(level=5, n=100000, config=4),
    "serving": dict(level=5, n=60000, config=5),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="level2")
    ap.add_argument("--n", type=int, default=0, help="override the task count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-served", action="store_true",
                    help="leave out the served measurement (its kernel waits on copies made while it runs, which "
                         "a profiler that serialises work would hold back)")
    return ap.parse_args()


# ----------------------------------------------------------------- ranks
class Ranks:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [s for t, s in self.samples if self.t0 and self.t1 and self.t0 <= t <= self.t1 + 0.2]
        if not rows:
            rows = [s for _, s in self.samples]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- oracle
def cpu_baseline(level: int, wl: dict, budget_s: float = 10.0) -> dict:
    """Times the CPU oracle (as it stands) on a bounded sample of the workload:
    Sign then Verify of `sample` tasks on all host cores."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    n_all = wl["seeds"].shape[0]
    # keys for the sample are generated outside the timed region
    sample = min(n_all, max(cores * 4, 64))
    seeds = wl["seeds"][:sample]
    lens = wl["lengths"][:sample]
    off = wl["msg_off"][: sample + 1]
    msg = wl["msg"][: int(off[-1]) + 1]
    pk, sk = oracle.keygen_batch(level, seeds, nthreads=cores)
    done, t_total = 0, 0.0
    while t_total < budget_s:
        t0 = time.perf_counter()
        sig, st, _ = oracle.sign_batch(level, sk, msg, off, nthreads=cores)
        ok = oracle.verify_batch(level, pk, msg, off, sig, nthreads=cores)
        t_total += time.perf_counter() - t0
        done += sample
        assert ok.all()
    # one host thread on a smaller sample (a few seconds)
    one = min(sample, 16)
    t0 = time.perf_counter()
    sig1, _, _ = oracle.sign_batch(level, sk[:one], msg, off[: one + 1], nthreads=1)
    ok1 = oracle.verify_batch(level, pk[:one], msg, off[: one + 1], sig1, nthreads=1)
    t1 = time.perf_counter() - t0
    assert ok1.all()
    return {"value": 2 * done / t_total, "unit": "ops/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} Dilithium{level} sign+verify tasks ({sample} distinct, messages "
                      f"{int(lens.min())}-{int(lens.max())} B) in {t_total:.1f} s",
            "single_thread": {"value": 2 * one / t1, "unit": "ops/s", "sample": f"{one} sign+verify tasks"}}


# ----------------------------------------------------------------- ours
def run_ours(args, ranks: Ranks) -> dict | None:
    import torch

    from paper_2211_12265_gb300 import dil

    spec = WORKLOADS[args.workload]
    level, n = spec["level"], (args.n or spec["n"])
    dev = ranks.local if torch.cuda.device_count() > ranks.local else 0
    torch.cuda.set_device(dev)
    wl = W.workload(spec["config"], n)
    # per-rank replicas draw distinct keys
    if ranks.rank:
        wl["seeds"] = W.seeds(n, spec["config"], offset=ranks.rank * n)
    ctx = dil.Context(dev)
    ctx.apply_tuning()
    seeds = torch.from_numpy(wl["seeds"]).cuda()
    msg = torch.from_numpy(wl["msg"]).cuda()
    off = torch.from_numpy(wl["msg_off"]).cuda()
    pk, sk = ctx.keygen(level, seeds)                     # untimed key generation
    sig, status, its = ctx.sign(level, sk, msg, off, iterations=True)
    ok = ctx.verify(level, pk, msg, off, sig)
    torch.cuda.synchronize()
    assert bool((status == 0).all()) and bool(ok.all()), "warm-up batch failed"
    iters = its.cpu().numpy()

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    n_ops = 2 * n

    def step(ev):
        flush.fill_(1)                                   # evict L2 between steps
        ev[0].record(stream)
        dil.dil_sign(ctx.handle, level, n, sk, msg, off, sig, status, stream)
        ev[1].record(stream)
        dil.dil_verify(ctx.handle, level, n, pk, msg, off, sig, ok, stream)
        ev[2].record(stream)

    for _ in range(args.warmup):
        step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
    torch.cuda.synchronize()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clk = ClockSampler(dev)
    clk.start()
    time.sleep(0.5)
    ranks.barrier()
    torch.cuda.synchronize()
    clk.mark(True)
    wall0 = time.perf_counter()
    for ev in events:
        step(ev)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ranks.barrier()
    clk.mark(False)
    clocks = clk.stop()
    sign_ms = [e[0].elapsed_time(e[1]) for e in events]
    ver_ms = [e[1].elapsed_time(e[2]) for e in events]
    step_ms = float(np.mean(np.add(sign_ms, ver_ms)))
    step_ms_max = ranks.max(step_ms)
    assert bool((status == 0).all()) and bool(ok.all())

    # persistent form of the same Sign batch (graph-captured launch)
    from paper_2211_12265_gb300 import autotune
    autotune.apply(ctx, persistent_level=level)
    job = [dil.sign_job(level, n, sk, msg, off, sig, status)]
    p_steps = max(1, min(args.steps, 100))
    for _ in range(max(args.warmup, 3)):
        dil.dil_sign_persistent(ctx.handle, job, stream)
    torch.cuda.synchronize()
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(p_steps)]
    ranks.barrier()
    for ev in pev:
        flush.fill_(1)
        ev[0].record(stream)
        dil.dil_sign_persistent(ctx.handle, job, stream)
        ev[1].record(stream)
    torch.cuda.synchronize()
    assert dil.dil_persistent_status(ctx.handle, stream) == dil.OK
    assert bool((status == 0).all())
    p_sign_ms = ranks.max(float(np.mean([e[0].elapsed_time(e[1]) for e in pev])))

    # fusion ablation: the same Sign batch split into kernels (precompute + two per repetition round)
    split_ms, rounds = [], 0
    for i in range(2 + 5):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        rounds = dil.dil_test_sign_split(ctx.handle, level, n, sk, msg, off, sig, status, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            split_ms.append(ev[0].elapsed_time(ev[1]))
    assert bool((status == 0).all())
    s_sign_ms = ranks.max(float(np.mean(split_ms)))

    # KeyGen of the batch's seeds (plain form, outside the timed step; the
    # keys come out byte-identical to those signed and verified above)
    kg_ms = []
    for i in range(2 + 5):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        dil.dil_keygen(ctx.handle, level, n, seeds, pk, sk, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            kg_ms.append(ev[0].elapsed_time(ev[1]))
    k_gen_ms = ranks.max(float(np.mean(kg_ms)))

    # the other configurations, each in its own launch configuration
    timed = _timer(torch, flush, stream, ranks)
    extra = max(1, min(args.steps, 10))
    # caller-owned A^: expanded once per key (timed alone), then Sign and
    # Verify of the same batch reading it instead of sampling it
    kl = {2: 16, 3: 30, 5: 56}[level]
    ahat = torch.empty((n, kl * 256), dtype=torch.int32, device="cuda")
    t_exp = timed(lambda: dil.dil_expand_a(ctx.handle, level, n, pk, pk.shape[1], ahat, stream), extra)
    sig_a = torch.empty_like(sig)
    st_a = torch.empty_like(status)
    ok_a = torch.empty(n, dtype=torch.uint8, device="cuda")
    t_sign_a = timed(lambda: dil.dil_sign_a(ctx.handle, level, n, sk, msg, off, ahat, sig_a, st_a, stream=stream), extra)
    t_ver_a = timed(lambda: dil.dil_verify_a(ctx.handle, level, n, pk, msg, off, sig, ahat, ok_a, stream), extra)
    assert bool(torch.equal(sig_a, sig)) and bool((st_a == 0).all()) and bool(ok_a.all())
    ahat_forms = {"expand_a_keys_s": ranks.world * n / (t_exp * 1e-3),
                  "sign_ops_s": ranks.world * n / (t_sign_a * 1e-3),
                  "verify_ops_s": ranks.world * n / (t_ver_a * 1e-3),
                  "note": "dil_sign_a / dil_verify_a with the keys' A^ from dil_expand_a (one warp per task)"}
    del ahat
    other_levels = {f"level{lv}": level_forms(ctx, lv, timed, stream, ranks, extra) for lv in (3, 5) if lv != level}
    mixed = mixed_forms(ctx, timed, stream, ranks, max(1, min(args.steps, 5)))
    ctx.apply_tuning()
    served = served_measure(dev) if ranks.world == 1 and not args.skip_served else None

    # e2e: host buffers through the host-form C entry points
    h_sk = torch.empty_like(sk, device="cpu").pin_memory()
    h_sk.copy_(sk)
    h_pk = torch.empty_like(pk, device="cpu").pin_memory()
    h_pk.copy_(pk)
    h_msg = torch.from_numpy(wl["msg"]).pin_memory()
    h_off = torch.from_numpy(wl["msg_off"]).pin_memory()
    h_sig = torch.empty(sig.shape, dtype=torch.uint8).pin_memory()
    h_st = torch.empty(n, dtype=torch.int32).pin_memory()
    h_ok = torch.empty(n, dtype=torch.uint8).pin_memory()
    e2e_steps = max(1, min(args.steps, 50))

    def e2e_step():
        dil.dil_sign_host(ctx.handle, level, n, h_sk, h_msg, h_off, h_sig, h_st, stream)
        dil.dil_verify_host(ctx.handle, level, n, h_pk, h_msg, h_off, h_sig, h_ok, stream)

    for _ in range(2):
        e2e_step()
    ranks.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_ms = ranks.max((time.perf_counter() - t0) * 1e3 / e2e_steps)
    assert bool((h_st == 0).all()) and bool(h_ok.all())
    mlen = int(wl["msg_off"][-1])
    h2d = sk.numel() + mlen + 8 * (n + 1) + pk.numel() + mlen + 8 * (n + 1) + sig.numel()
    d2h = sig.numel() + 4 * n + n

    # roofline of the dominant kernel (Sign): algorithmic integer ops / its time
    sw = WK.sign_work(level, iters, wl["lengths"])
    ops = WK.int_ops(sw)
    sign_mean_ms = float(np.mean(sign_ms))
    achieved = ops / (sign_mean_ms * 1e-3) / 1e12
    lop3_rate = dil.dil_test_issue_rate(ctx.handle, dil.ISSUE_OPS["lop3"])   # thread-ops / SM / clk
    shfl_rate = dil.dil_test_issue_rate(ctx.handle, dil.ISSUE_OPS["shfl"])
    keccak_forms = {name: dil.dil_test_keccak_rate(ctx.handle, form)
                    for name, form in (("one_state_25_lanes", 1), ("two_states_interleaved", 2),
                                       ("six_states_row_layout", 6), ("sixteen_states_two_threads", 16))}
    peak = SMS * ISSUE_THREAD_OPS_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    alu_peak = SMS * lop3_rate * SM_MAX_MHZ * 1e6 / 1e12
    for r in other_levels.values():
        r["roofline_frac"] = r["sign_int_ops"] / (r["sign_ms"] * 1e-3) / 1e12 / peak
    traffic = load_traffic(level, n)
    hbm = measured_hbm_gbs()
    table = autotune.load() or {}
    sign_p = table.get("plain", {}).get(str(level), {}).get("sign", {}).get("warps_per_task", 2)

    res = {
        "metric": METRIC,
        "value": ranks.world * n_ops / (step_ms_max * 1e-3),
        "unit": "ops/s",
        "n_gpus": ranks.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded PCG64 keys and messages)",
        "config": {"workload": f"dilithium{level}-sign+verify-{n}", "level": level, "n_tasks_per_gpu": n,
                   "msg_bytes": f"{int(wl['lengths'].min())}-{int(wl['lengths'].max())}",
                   "form": "plain, one launch per phase", "l2": "flushed before every step (512 MiB write)",
                   "parallelism": f"replicas x{ranks.world}"},
        "forms": {"plain_sign_ops_s": ranks.world * n / (ranks.max(sign_mean_ms) * 1e-3),
                  "persistent_sign_ops_s": ranks.world * n / (p_sign_ms * 1e-3),
                  "persistent_step_ops_s": ranks.world * n_ops / ((p_sign_ms + ranks.max(float(np.mean(ver_ms))))
                                                                  * 1e-3),
                  "persistent_sign_ms": p_sign_ms,
                  "split_sign_ops_s": ranks.world * n / (s_sign_ms * 1e-3), "split_sign_rounds": rounds,
                  "split_note": "fusion ablation: precompute kernel + two kernels per repetition round",
                  "caller_ahat": ahat_forms, **other_levels, "mixed_200k": mixed},
        "served": served,
        "breakdown": {"sign_ops_s": ranks.world * n / (ranks.max(sign_mean_ms) * 1e-3),
                      "verify_ops_s": ranks.world * n / (ranks.max(float(np.mean(ver_ms))) * 1e-3),
                      "sign_ms": sign_mean_ms, "verify_ms": float(np.mean(ver_ms)),
                      "keygen_ops_s": ranks.world * n / (k_gen_ms * 1e-3), "keygen_ms": k_gen_ms,
                      "mean_sign_repetitions": float(iters.mean()),
                      "sign_repetitions_histogram": {str(k): int((iters == k).sum()) for k in range(1, 16)} |
                                                    {">15": int((iters > 15).sum())},
                      "wall_s_timed_region": wall},
        "e2e": {"value": ranks.world * n_ops / (e2e_ms * 1e-3), "unit": "ops/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
        "gpu_launches": 2 * args.steps,
        "gpu_launches_note": "plain timed region: one Sign and one Verify kernel per step",
        "roofline": {"bound": "alu", "kernel": f"k_sign<{level}, {sign_p}>", "achieved": achieved,
                     "peak": peak, "unit": "Tops/s (32-bit integer)", "frac": achieved / peak,
                     "traffic": traffic, "ops_per_sign": ops / n,
                     "dram_gbs": traffic / (sign_mean_ms * 1e-3) / 1e9 if traffic else None,
                     "dram_frac_of_measured_hbm": (traffic / (sign_mean_ms * 1e-3) / 1e9 / hbm
                                                   if traffic and hbm else None),
                     "peak_basis": f"{SMS} SMs x 4 sub-partitions x one 32-thread warp instruction per clock "
                                   f"({ISSUE_THREAD_OPS_PER_SM_CLK} thread-ops/SM/clk) x {SM_MAX_MHZ:.0f} MHz max SM clock",
                     "alu_pipe": {"lop3_thread_ops_per_sm_clk": lop3_rate, "peak": alu_peak,
                                  "frac": achieved / alu_peak,
                                  "basis": "LOP3 rate measured live (per-SM clock64 spans) x SMs x max SM clock"},
                     "shfl_thread_ops_per_sm_clk": shfl_rate,
                     "keccak_sm_clk_per_state_round": keccak_forms},
        "clocks": clocks,
        "tuning": {"plain": table.get("plain", {}).get(str(level)),
                   "persistent": table.get("persistent", {}).get(str(level)),
                   "source": "paper_2211_12265_gb300/tuning_gb300.json (autotune.py)"},
        "paper_context_a100": PAPER_A100[level],
    }
    ctx.close()
    if ranks.rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(level, wl)
    return res


def _timer(torch, flush, stream, ranks):
    """Mean CUDA-event time (ms) of fn over `steps` runs, L2 flushed before
    each, after `warm` untimed runs; maximum over ranks."""
    def timed(fn, steps, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        ranks.barrier()
        for ev in evs:
            flush.fill_(1)
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
        torch.cuda.synchronize()
        return ranks.max(float(np.mean([e[0].elapsed_time(e[1]) for e in evs])))
    return timed


def level_forms(ctx, level: int, timed, stream, ranks, steps: int, n: int = 10000) -> dict:
    """Config 3 at one level: 10,000 tasks with messages of 32..4096 bytes;
    plain Sign, Verify and KeyGen (one launch each) and the persistent Sign."""
    import torch

    from paper_2211_12265_gb300 import autotune, dil
    wl = W.workload(3, n)
    if ranks.rank:
        wl["seeds"] = W.seeds(n, 3, offset=ranks.rank * n)
    seeds = torch.from_numpy(wl["seeds"]).cuda()
    msg = torch.from_numpy(wl["msg"]).cuda()
    off = torch.from_numpy(wl["msg_off"]).cuda()
    pk, sk = ctx.keygen(level, seeds)
    sig, st, its = ctx.sign(level, sk, msg, off, iterations=True)
    ok = ctx.verify(level, pk, msg, off, sig)
    torch.cuda.synchronize()
    assert bool((st == 0).all()) and bool(ok.all())
    t_sign = timed(lambda: dil.dil_sign(ctx.handle, level, n, sk, msg, off, sig, st, stream), steps)
    t_ver = timed(lambda: dil.dil_verify(ctx.handle, level, n, pk, msg, off, sig, ok, stream), steps)
    t_kg = timed(lambda: dil.dil_keygen(ctx.handle, level, n, seeds, pk, sk, stream), steps)
    autotune.apply(ctx, persistent_level=level)
    job = [dil.sign_job(level, n, sk, msg, off, sig, st)]
    t_p = timed(lambda: dil.dil_sign_persistent(ctx.handle, job, stream), steps)
    assert dil.dil_persistent_status(ctx.handle, stream) == dil.OK and bool((st == 0).all())
    assert bool(ok.all())
    iters = its.cpu().numpy()
    w = ranks.world
    return {"workload": f"dilithium{level}-{n}", "msg_bytes": f"{int(wl['lengths'].min())}-{int(wl['lengths'].max())}",
            "plain_sign_ops_s": w * n / (t_sign * 1e-3), "persistent_sign_ops_s": w * n / (t_p * 1e-3),
            "verify_ops_s": w * n / (t_ver * 1e-3), "keygen_ops_s": w * n / (t_kg * 1e-3),
            "plain_step_ops_s": w * 2 * n / ((t_sign + t_ver) * 1e-3),
            "persistent_step_ops_s": w * 2 * n / ((t_p + t_ver) * 1e-3),
            "sign_ms": t_sign, "persistent_sign_ms": t_p, "verify_ms": t_ver, "keygen_ms": t_kg,
            "mean_sign_repetitions": float(iters.mean()),
            "sign_int_ops": WK.int_ops(WK.sign_work(level, iters, wl["lengths"])),
            "paper_context_a100": PAPER_A100[level]}


def mixed_forms(ctx, timed, stream, ranks, steps: int, n: int = 100000) -> dict:
    """Config 4: persistent Sign of n Dilithium2 + n Dilithium5 tasks (one
    graph-captured launch) against the plain form (one launch per level)."""
    import torch

    from paper_2211_12265_gb300 import autotune, dil
    autotune.apply(ctx, persistent_level="mixed")
    data = {}
    for level in (2, 5):
        wl = W.workload(4, n)
        seeds = torch.from_numpy(W.seeds(n, 4 + level, offset=ranks.rank * n)).cuda()
        msg = torch.from_numpy(wl["msg"]).cuda()
        off = torch.from_numpy(wl["msg_off"]).cuda()
        pk, sk = ctx.keygen(level, seeds)
        sig = torch.empty((n, dil.SIZES[level][2]), dtype=torch.uint8, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        data[level] = (sk, msg, off, sig, st)
    jobs = [dil.sign_job(2, n, *data[2]), dil.sign_job(5, n, *data[5])]
    t_p = timed(lambda: dil.dil_sign_persistent(ctx.handle, jobs, stream), steps)
    assert dil.dil_persistent_status(ctx.handle, stream) == dil.OK
    assert all(bool((data[lv][4] == 0).all()) for lv in (2, 5))
    t_plain = timed(lambda: (dil.dil_sign(ctx.handle, 2, n, *data[2], stream=stream),
                             dil.dil_sign(ctx.handle, 5, n, *data[5], stream=stream)), steps)
    assert all(bool((data[lv][4] == 0).all()) for lv in (2, 5))
    w = ranks.world
    return {"workload": f"sign-{n}-dilithium2+{n}-dilithium5, 32 B messages",
            "persistent_ops_s": w * 2 * n / (t_p * 1e-3), "plain_ops_s": w * 2 * n / (t_plain * 1e-3),
            "persistent_ms": t_p, "plain_ms": t_plain, "steps": steps}


def plain_replay(dev: int, keys: dict, req: dict, reps: int = 5) -> dict:
    """The requests of a served trace run by the plain kernels, one launch per
    (operation, level) over the whole trace: the plain one-launch-per-batch
    form at its largest batch.  Timed twice: with the requests resident on
    the device, and with what a service moves per request inside the timed
    region (messages and signatures to verify in from pinned host memory,
    signatures and results out; keys resident, as for the server)."""
    import torch

    from paper_2211_12265_gb300 import dil
    groups = []
    stream = torch.cuda.current_stream()
    with dil.Context(dev) as ctx:
        ctx.apply_tuning()
        for op in (0, 1):
            for lv in sorted(keys):
                idx = np.nonzero((req["op"] == op) & (req["level"] == lv))[0]
                if idx.size == 0:
                    continue
                parts = [req["msg"][req["msg_off"][i]:req["msg_off"][i + 1]] for i in idx]
                o = np.zeros(idx.size + 1, dtype=np.uint64)
                o[1:] = np.cumsum([p.size for p in parts])
                g = {"op": op, "lv": lv, "k": idx.size,
                     "h_msg": torch.from_numpy(np.concatenate(parts + [np.zeros(1, np.uint8)])).pin_memory(),
                     "h_off": torch.from_numpy(o).pin_memory()}
                g["msg"] = g["h_msg"].cuda()
                g["off"] = g["h_off"].cuda()
                kidx = req["key"][idx]
                sigb = dil.SIZES[lv][2]
                if op == 0:
                    g["key"] = torch.from_numpy(np.ascontiguousarray(keys[lv][1][kidx])).cuda()
                    g["out"] = torch.empty((idx.size, sigb), dtype=torch.uint8, device="cuda")
                    g["st"] = torch.empty(idx.size, dtype=torch.int32, device="cuda")
                    g["h_out"] = torch.empty((idx.size, sigb), dtype=torch.uint8).pin_memory()
                    g["h_st"] = torch.empty(idx.size, dtype=torch.int32).pin_memory()
                else:
                    g["key"] = torch.from_numpy(np.ascontiguousarray(keys[lv][0][kidx])).cuda()
                    g["h_sig"] = torch.from_numpy(np.ascontiguousarray(req["sig_in"][idx, :sigb])).pin_memory()
                    g["sig"] = g["h_sig"].cuda()
                    g["out"] = torch.empty(idx.size, dtype=torch.uint8, device="cuda")
                    g["h_out"] = torch.empty(idx.size, dtype=torch.uint8).pin_memory()
                groups.append(g)

        def run(copies: bool):
            for g in groups:
                if copies:
                    g["msg"].copy_(g["h_msg"], non_blocking=True)
                    g["off"].copy_(g["h_off"], non_blocking=True)
                    if g["op"] == 1:
                        g["sig"].copy_(g["h_sig"], non_blocking=True)
                if g["op"] == 0:
                    dil.dil_sign(ctx.handle, g["lv"], g["k"], g["key"], g["msg"], g["off"], g["out"], g["st"], stream)
                else:
                    dil.dil_verify(ctx.handle, g["lv"], g["k"], g["key"], g["msg"], g["off"], g["sig"], g["out"],
                                   stream)
                if copies:
                    g["h_out"].copy_(g["out"], non_blocking=True)
                    if g["op"] == 0:
                        g["h_st"].copy_(g["st"], non_blocking=True)

        def timed(copies: bool) -> float:
            run(copies)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run(copies)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return float(np.median(ts))
        t_dev = timed(False)
        t_e2e = timed(True)
    n = int(req["op"].size)
    return {"ops_s": n / (t_dev * 1e-3), "ms": t_dev, "e2e_ops_s": n / (t_e2e * 1e-3), "e2e_ms": t_e2e,
            "requests": n, "launches": len(groups),
            "form": "plain kernels, one launch per (operation, level); ops_s with the requests resident on the "
                    "device, e2e_ops_s with messages / signatures copied in and results copied out"}


def served_measure(dev: int, n: int = 80000, fractions=SERVED_FRACTIONS) -> dict:
    """Config 5: the served mix on the continuous-batching server: saturated
    ops/s, an arrival-rate sweep with p50/p99, and at each rate the best p99
    of static batching over STATIC_GRID; beside it the plain kernels' rate on
    the saturated trace's requests."""
    from paper_2211_12265_gb300 import serving
    keys = serving.make_keys((2, 3, 5), n_keys=4096, device=dev)
    with serving.Server(dev, memory_budget=8 << 30, streams=4, max_batch=4096) as srv:
        for lv in keys:
            srv.add_keys(lv, *keys[lv])
        srv.replay(serving.serving_workload(keys, n, rate=1e9, seed=100))         # warm-up (host buffers touched)
        sat_req = serving.serving_workload(keys, n, rate=1e9, seed=101)

        def median_of(req, key, runs=SERVED_REPLAYS):
            # the replay with the median `key` of `runs` replays of one trace
            rs = sorted((serving.summarize(req, srv.replay(req)) for _ in range(runs)), key=lambda r: r[key])
            out = dict(rs[len(rs) // 2])
            out["replays"] = runs
            return out
        sat = median_of(sat_req, "ops_s")
        rows, static_rows = [], []
        for i, f in enumerate(fractions):
            rq = serving.serving_workload(keys, n, rate=f * sat["ops_s"], seed=102 + i)
            srv.set_batching(1, 0.0)
            r = median_of(rq, "p99_ms")
            r["offered_fraction"] = f
            rows.append(r)
            best = None
            for mb, wait in STATIC_GRID:
                srv.set_batching(mb, wait)
                sr = serving.summarize(rq, srv.replay(rq))
                sr.update({"min_batch": mb, "max_wait_s": wait})
                if best is None or sr["p99_ms"] < best["p99_ms"]:
                    best = sr
            best["offered_fraction"] = f
            best["grid_points"] = len(STATIC_GRID)
            static_rows.append(best)
        srv.set_batching(1, 0.0)
        batches, carried, launches = srv.stats()
    plain = plain_replay(dev, keys, sat_req)
    return {"saturated_ops_s": sat["ops_s"], "saturated": sat,
            "mix": "60% verify / 40% sign, levels 2/3/5, msg 32 B-16 KB log-uniform, 4096 resident keys per level, "
                   "Poisson arrivals", "streams": 4, "sweep": rows,
            "static_batching_best_p99": static_rows,
            "static_grid": {"min_batch": sorted({g[0] for g in STATIC_GRID}),
                            "max_wait_s": sorted({g[1] for g in STATIC_GRID})},
            "plain_kernels_same_requests": plain,
            "served_over_plain": sat["ops_s"] / plain["ops_s"],
            "served_over_plain_e2e": sat["ops_s"] / plain["e2e_ops_s"],
            "server_batches": batches, "server_requests": carried, "server_launches": launches}


def run_mixed(args, ranks: Ranks) -> dict:
    """Config 4 alone (``--workload mixed``)."""
    import torch

    from paper_2211_12265_gb300 import dil
    dev = ranks.local if torch.cuda.device_count() > ranks.local else 0
    torch.cuda.set_device(dev)
    ctx = dil.Context(dev)
    ctx.apply_tuning()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    steps = max(1, min(args.steps, 20))
    r = mixed_forms(ctx, _timer(torch, flush, stream, ranks), stream, ranks, steps, n=args.n or 100000)
    ctx.close()
    return {"metric": METRIC, "value": r["persistent_ops_s"], "unit": "ops/s", "n_gpus": ranks.world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": r["persistent_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded PCG64 keys and messages)",
            "config": {"workload": r["workload"], "form": "persistent, one graph-captured launch",
                       "l2": "flushed before every step", "parallelism": f"replicas x{ranks.world}"},
            "forms": {"mixed_200k": r}, "gpu_launches": steps}


def run_level(args, ranks: Ranks) -> dict:
    """Config 3 at one level alone (``--workload level3|level5``)."""
    import torch

    from paper_2211_12265_gb300 import dil
    spec = WORKLOADS[args.workload]
    dev = ranks.local if torch.cuda.device_count() > ranks.local else 0
    torch.cuda.set_device(dev)
    ctx = dil.Context(dev)
    ctx.apply_tuning()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    steps = max(1, min(args.steps, 50))
    r = level_forms(ctx, spec["level"], _timer(torch, flush, stream, ranks), stream, ranks, steps,
                    n=args.n or spec["n"])
    ctx.close()
    return {"metric": METRIC, "value": r["plain_step_ops_s"], "unit": "ops/s", "n_gpus": ranks.world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": r["sign_ms"] + r["verify_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded PCG64 keys and messages)",
            "config": {"workload": r["workload"] + "-sign+verify", "msg_bytes": r["msg_bytes"],
                       "form": "plain, one launch per phase", "l2": "flushed before every step",
                       "parallelism": f"replicas x{ranks.world}"},
            "forms": {f"level{spec['level']}": r}, "gpu_launches": 2 * steps}


def run_serving(args, ranks: Ranks) -> dict | None:
    """Config 5 alone (``--workload serving``): a finer sweep, 10% to 120%."""
    import torch
    dev = ranks.local if torch.cuda.device_count() > ranks.local else 0
    torch.cuda.set_device(dev)
    r = served_measure(dev, n=args.n or 60000, fractions=(0.1, 0.3, 0.5, 0.7, 0.9, 1.1, 1.2))
    best = max(r["sweep"] + [r["saturated"]], key=lambda x: x["ops_s"])
    return {"metric": METRIC, "value": ranks.world * best["ops_s"], "unit": "ops/s", "n_gpus": ranks.world,
            "steps": len(r["sweep"]) + 1, "warmup": 1, "ms_per_step": 1e3 * r["saturated"]["wall_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Poisson arrivals)",
            "config": {"workload": "served-mix", "mix": r["mix"], "requests_per_point": args.n or 60000,
                       "streams": 4, "parallelism": f"replicas x{ranks.world}"},
            "served": r, "gpu_launches": r["server_launches"],
            "gpu_launches_note": "keyed kernel launches of the server over the whole run"}


def measured_hbm_gbs():
    """Measured HBM copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def load_traffic(level: int, n: int):
    """DRAM bytes per Sign launch, scaled from the committed ncu capture of a
    smaller batch; None when the kernel sources changed since the capture."""
    from paper_2211_12265_gb300 import build
    path = os.path.join(ROOT, "profiles", f"k_sign_level{level}_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_digest") != build.source_digest():
            return None
        return d["dram_bytes_per_task"] * n
    except (OSError, KeyError, ValueError):
        return None


def run_reference(args, ranks: Ranks) -> dict | None:
    if ranks.rank != 0:
        return None
    from oracle import oracle
    spec = WORKLOADS[args.workload]
    level = spec["level"]
    cores = os.cpu_count() or 1
    sample = 64 * cores            # 64 tasks per host thread: the repetition counts average out per thread
    wl = W.workload(spec["config"], sample)
    pk, sk = oracle.keygen_batch(level, wl["seeds"], nthreads=cores)
    off, msg = wl["msg_off"], wl["msg"]

    def step():
        sig, st, _ = oracle.sign_batch(level, sk, msg, off, nthreads=cores)
        ok = oracle.verify_batch(level, pk, msg, off, sig, nthreads=cores)
        assert ok.all()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = 2 * sample * args.steps / dt
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ops/s", "n_gpus": ranks.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded PCG64 keys and messages)",
        "config": {"workload": f"dilithium{level}-sign+verify-{spec['n']}", "level": level,
                   "n_tasks_per_step": sample, "form": "CPU oracle (plain C, -O2) on host threads"},
        "cpu_baseline": {"value": value, "unit": "ops/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} tasks per step x {args.steps} steps"},
        "e2e": {"value": value, "unit": "ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    ranks = Ranks()
    try:
        if args.impl == "reference":
            res = run_reference(args, ranks)
        elif args.workload == "mixed":
            res = run_mixed(args, ranks)
        elif args.workload in ("level3", "level5"):
            res = run_level(args, ranks)
        elif args.workload == "serving":
            res = run_serving(args, ranks)
        else:
            res = run_ours(args, ranks)
        if res is not None and ranks.rank == 0:
            print(json.dumps(res), flush=True)
    finally:
        ranks.close()


if __name__ == "__main__":
    main()
