"""Driver of the continuous-batching server (``dil_server_*`` in include/dil.h).

``Server`` wraps the C server; ``serving_workload`` builds the serving mix
(Poisson arrivals, 60% verify / 40% sign, levels 2/3/5 in equal shares,
messages log-uniform in [32, 16384] bytes, keys drawn from resident key pairs;
verify requests carry valid signatures made beforehand); ``sweep`` replays it
at a list of arrival rates and reports ops/s with p50/p99 latency.  All the
cryptographic work runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import dil
from . import workload as W

SIG_STRIDE = 4595


class Server:
    def __init__(self, device: int = 0, memory_budget: int = 0, streams: int = 4, max_batch: int = 2048):
        self.handle = dil.dil_server_create(device, memory_budget, streams, max_batch)
        self.max_batch, self.msg_capacity = dil.dil_server_limits(self.handle)

    def close(self):
        if self.handle:
            dil.dil_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_batching(self, min_batch: int = 1, max_wait_s: float = 0.0) -> None:
        """Continuous batching on the device when max_wait_s is 0 (the
        default); max_wait_s > 0 selects static batching, where a batch starts
        with min_batch pending requests or once the oldest waited max_wait_s."""
        dil.dil_server_set_batching(self.handle, min_batch, max_wait_s)

    def set_tuning(self, op: int, level: int, warps_per_cta: int, warps_per_task: int) -> None:
        dil.dil_server_set_tuning(self.handle, op, level, warps_per_cta, warps_per_task)

    def add_keys(self, level: int, pk: np.ndarray, sk: np.ndarray) -> None:
        pk = np.ascontiguousarray(pk, dtype=np.uint8)
        sk = np.ascontiguousarray(sk, dtype=np.uint8)
        dil.dil_server_add_keys(self.handle, level, pk.shape[0], pk, sk)

    def submit(self, op: int, level: int, key: int, msg: bytes, sig: bytes | None = None) -> int:
        return dil.dil_server_submit(self.handle, op, level, key, msg, sig)

    def cancel(self, rid: int) -> bool:
        """Withdraws a still-pending request; True when it was canceled."""
        return dil.dil_server_cancel(self.handle, rid) == dil.OK

    def poll(self, max_n: int = 256, wait_us: int = 1000) -> list:
        return dil.dil_server_poll(self.handle, max_n, wait_us)

    def replay(self, req: dict) -> dict:
        """Open-loop replay of a request set built by serving_workload()."""
        n = req["op"].size
        # output buffers written before the replay starts, so that storing a
        # result does not take a page fault inside the measured interval
        sig_out = np.empty((n, SIG_STRIDE), dtype=np.uint8)
        sig_out.fill(0)
        status = np.full(n, 0, dtype=np.int32)
        ok = np.full(n, 0, dtype=np.uint8)
        lat = np.full(n, 0.0, dtype=np.float64)
        wall = dil.dil_server_replay(self.handle, n, req["arrival"], req["op"], req["level"], req["key"],
                                     req["msg"], req["msg_off"], req["sig_in"], sig_out, status, ok, lat)
        return {"sig": sig_out, "status": status, "ok": ok, "latency": lat, "wall": wall}

    def stats(self) -> tuple[int, int, int]:
        """(batches, requests, kernel launches) since creation."""
        return dil.dil_server_stats(self.handle)


def make_keys(levels=(2, 3, 5), n_keys: int = 4096, device: int = 0) -> dict:
    """Key pairs per level generated on the GPU from seeded seeds (host arrays)."""
    import torch
    keys = {}
    with dil.Context(device) as ctx:
        for lv in levels:
            seeds = torch.from_numpy(W.seeds(n_keys, 50 + lv)).cuda()
            pk, sk = ctx.keygen(lv, seeds)
            keys[lv] = (pk.cpu().numpy(), sk.cpu().numpy())
    return keys


def serving_workload(keys: dict, n: int, rate: float, seed: int = 7, device: int = 0,
                     lo: int = 32, hi: int = 16384) -> dict:
    """The serving mix at `rate` requests/s; verify requests carry signatures
    produced (untimed) by dil_sign on the same keys."""
    import torch
    mix = W.request_mix(n, min(v[0].shape[0] for v in keys.values()), seed=seed,
                        levels=tuple(sorted(keys)))
    lens = W.message_lengths(n, 5, "loguniform", lo, hi)
    msg, off = W.messages(lens, 5)
    arrival = W.arrivals(n, rate, seed=seed + 1)
    arrival -= arrival[0]
    sig_in = np.zeros((n, SIG_STRIDE), dtype=np.uint8)
    with dil.Context(device) as ctx:
        for lv in keys:
            idx = np.nonzero((mix["level"] == lv) & (mix["op"] == 1))[0]
            if idx.size == 0:
                continue
            sk = torch.from_numpy(keys[lv][1][mix["key"][idx]]).cuda()
            m = np.concatenate([msg[off[i]:off[i + 1]] for i in idx] + [np.zeros(1, np.uint8)])
            o = np.zeros(idx.size + 1, dtype=np.uint64)
            o[1:] = np.cumsum(lens[idx])
            sig, st = ctx.sign(lv, sk, torch.from_numpy(m).cuda(), torch.from_numpy(o).cuda())
            sig_in[idx, :sig.shape[1]] = sig.cpu().numpy()
    return {"arrival": np.ascontiguousarray(arrival), "op": mix["op"].astype(np.int32),
            "level": mix["level"].astype(np.int32), "key": mix["key"].astype(np.int32),
            "msg": msg, "msg_off": off, "sig_in": sig_in, "lengths": lens}


def summarize(req: dict, out: dict) -> dict:
    lat = out["latency"]
    return {"requests": int(req["op"].size), "ops_s": req["op"].size / out["wall"],
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3), "wall_s": out["wall"]}


def sweep(server: Server, keys: dict, rates, n_per_rate: int = 20000, seed: int = 11) -> list:
    """Replays the serving mix at each arrival rate; returns one summary each."""
    rows = []
    for i, rate in enumerate(rates):
        req = serving_workload(keys, n_per_rate, rate, seed=seed + i)
        out = server.replay(req)
        row = summarize(req, out)
        row["offered_rate"] = rate
        rows.append(row)
    return rows
