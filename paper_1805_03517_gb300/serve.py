"""Request loop around the continuous-batching server (``ff_server_*`` in include/ff.h).

Frame pairs arrive on a timeline; each is submitted when its arrival time has passed, the native server admits
what fits its device-memory budget and advances every admitted request by one merged tick per ``step()``, and
completed requests hand back their device outputs (forward/inverse flow and consistency mask of FlowFields++
Sec. 3.1).  Latency is measured on the host from the scheduled arrival time to the poll that reports completion.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np


@dataclass
class ServeStats:
    n: int
    wall_s: float
    mpx: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    ticks: int
    launches: int

    @property
    def mpx_per_s(self) -> float:
        return self.mpx / self.wall_s

    def as_dict(self):
        return {"requests": self.n, "wall_s": self.wall_s, "value": self.mpx_per_s, "unit": "Mpx/s",
                "p50_ms": self.p50_ms, "p99_ms": self.p99_ms, "mean_ms": self.mean_ms, "ticks": self.ticks,
                "gpu_launches": self.launches}


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given mean rate (requests/s)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def serve(matcher, frames, arrivals, mem_budget_bytes=60 << 30, max_active=256, keep_outputs=False):
    """Serve requests i = 0..n-1 with inputs frames[i] = (img_a, img_b) (uint8 [h][w][3] CUDA tensors) arriving at
    arrivals[i] seconds after the start.  Returns ServeStats (and the outputs per request if keep_outputs)."""
    import torch

    from . import ff

    srv = ff.Server(matcher, mem_budget_bytes, max_active)
    n = len(frames)
    pools = {}  # (h, w) -> free output dicts

    def take(h, w):
        free = pools.setdefault((h, w), [])
        if free:
            return free.pop()
        with torch.cuda.stream(matcher.stream):
            return {"flow_fwd": torch.empty((h, w, 2), dtype=torch.int16, device=matcher.device),
                    "flow_bwd": torch.empty((h, w, 2), dtype=torch.int16, device=matcher.device),
                    "mask": torch.empty((h, w), dtype=torch.uint8, device=matcher.device)}

    outs, kept = {}, {}
    lat = np.zeros(n)
    mpx = sum(int(a.shape[0]) * int(a.shape[1]) for a, _ in frames) / 1e6
    submitted = completed = 0
    in_flight = 0
    matcher.stream.synchronize()
    t0 = time.perf_counter()
    while completed < n:
        now = time.perf_counter() - t0
        while submitted < n and arrivals[submitted] <= now:
            a, b = frames[submitted]
            o = take(int(a.shape[0]), int(a.shape[1]))
            outs[submitted] = o
            srv.submit(submitted, a, b, o)
            submitted += 1
            in_flight += 1
        if in_flight:
            srv.step()
        for rid in srv.poll(wait=False):
            lat[rid] = time.perf_counter() - t0 - arrivals[rid]
            o = outs.pop(rid)
            if keep_outputs:
                kept[rid] = {k: v.clone() for k, v in o.items()}
            else:
                pools[(int(o["mask"].shape[0]), int(o["mask"].shape[1]))].append(o)
            completed += 1
            in_flight -= 1
        if not in_flight and submitted < n:
            wait = arrivals[submitted] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.002))
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    stats = ServeStats(n, wall, mpx, float(np.percentile(lat, 50) * 1e3), float(np.percentile(lat, 99) * 1e3),
                       float(lat.mean() * 1e3), st["ticks"], st["launches"])
    return (stats, kept) if keep_outputs else stats
