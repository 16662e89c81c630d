"""Serving loop: render requests of mixed size and (a, i) with continuous
batching over a resident device pool.

Requests (one image each) arrive over time.  The pool is one state buffer of
a fixed number of ray slots; a request is admitted when a contiguous free
range large enough for its pixels exists (admission by device memory), its
rays are set up there, and from then on they are traced together with every
other request in flight: each round is one ``gray_trace`` over the pool with
a step budget (finished and empty slots are skipped), after which requests
whose rays are all done are rendered, copied to the host and their slots
cleared, and newly arrived requests are admitted into the freed space.  A
request therefore never waits for a batch to fill or drain; its rays overlap
on the device with everyone else's.  Because a ray's result is independent of
batching and of how its trace is split over calls, a request's image is the
same alone and in the mix.

Latency of a request = time its result reaches the host - its arrival time.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import gray


@dataclass
class Slot:
    first: int
    n: int


class PoolAllocator:
    """First-fit allocator of contiguous ray ranges in [0, capacity)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free = [Slot(0, self.capacity)]

    def alloc(self, n: int):
        for k, s in enumerate(self.free):
            if s.n >= n:
                out = Slot(s.first, n)
                if s.n == n:
                    self.free.pop(k)
                else:
                    self.free[k] = Slot(s.first + n, s.n - n)
                return out
        return None

    def release(self, slot: Slot):
        self.free.append(Slot(slot.first, slot.n))
        self.free.sort(key=lambda s: s.first)
        merged = []
        for s in self.free:
            if merged and merged[-1].first + merged[-1].n == s.first:
                merged[-1] = Slot(merged[-1].first, merged[-1].n + s.n)
            else:
                merged.append(s)
        self.free = merged

    def free_rays(self):
        return sum(s.n for s in self.free)


@dataclass
class Result:
    rid: int
    t_arrive: float
    t_admit: float
    t_done: float
    pixels: np.ndarray  # gray_pixel32 records
    steps: int = 0

    @property
    def latency(self):
        return self.t_done - self.t_arrive


@dataclass
class ServerStats:
    results: list = field(default_factory=list)
    rounds: int = 0
    steps: int = 0
    wall: float = 0.0

    def latencies(self):
        return np.array([r.latency for r in self.results])

    def summary(self):
        lat = self.latencies()
        return {"requests": len(self.results), "rounds": self.rounds, "photon_steps": self.steps,
                "wall_s": self.wall, "photon_steps_per_s": self.steps / self.wall if self.wall > 0 else 0.0,
                "p50_ms": 1000.0 * float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": 1000.0 * float(np.percentile(lat, 99)) if lat.size else None,
                "max_ms": 1000.0 * float(lat.max()) if lat.size else None}


class Server:
    """Continuous-batching render server over one resident pool.

    capacity: ray slots in the pool (device memory = gray_state_bytes).
    round_budget: steps each in-flight ray may take per round."""

    def __init__(self, opt: gray.Options, capacity: int, round_budget: int = 256, device="cuda"):
        import torch
        self.opt = opt
        self.capacity = int(capacity)
        self.round_budget = int(round_budget)
        self.tracer = gray.Tracer(opt, self.capacity, device=device)
        gray.gray_clear(self.tracer.ctx, self.tracer.state, self.capacity, 0, self.capacity)
        self.alloc = PoolAllocator(self.capacity)
        self.out_dev = torch.empty(16 * self.capacity, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream()

    def close(self):
        self.tracer.close()

    def _admit(self, req, now, inflight):
        slot = self.alloc.alloc(req.image.nx * req.image.ny)
        if slot is None:
            return False
        self.tracer.setup([req.image], first_ray=slot.first)
        inflight.append((req, slot, now))
        return True

    def _finish(self, req, slot, t_admit, stats):
        tr = self.tracer
        out = self.out_dev[16 * slot.first: 16 * (slot.first + slot.n)]
        gray.gray_render(tr.ctx, tr.state, tr.n, gray.RENDER_PIXELS32, first_ray=slot.first, n=slot.n, out=out)
        host = out.cpu()  # waits for the stream
        px = host.numpy().view(gray.PIXEL32_DTYPE)
        gray.gray_clear(tr.ctx, tr.state, tr.n, slot.first, slot.n)
        self.alloc.release(slot)
        stats.results.append(Result(req.rid, req.t_arrive, t_admit, time.perf_counter() - self._t0, px))

    def run(self, requests, realtime: bool = True, max_wall: float = None):
        """Serve `requests` (objects with rid, t_arrive seconds, image).  With
        realtime, arrivals follow the wall clock from the start of the call;
        otherwise every request is available at once.  Returns ServerStats."""
        pending = sorted(requests, key=lambda r: r.t_arrive)
        if not realtime:
            for r in pending:
                r.t_arrive = 0.0
        waiting = []  # arrived, not admitted (FIFO)
        inflight = []  # (request, slot, t_admit)
        stats = ServerStats()
        self._t0 = time.perf_counter()
        k = 0
        while k < len(pending) or waiting or inflight:
            now = time.perf_counter() - self._t0
            if max_wall is not None and now > max_wall:
                break
            while k < len(pending) and pending[k].t_arrive <= now:
                waiting.append(pending[k])
                k += 1
            # admission by device memory, first come first served
            while waiting and self._admit(waiting[0], now, inflight):
                waiting.pop(0)
            if waiting and not inflight:
                raise RuntimeError("request of %d rays does not fit a pool of %d" %
                                   (waiting[0].image.nx * waiting[0].image.ny, self.capacity))
            if not inflight:
                if k < len(pending):
                    time.sleep(max(0.0, min(0.002, pending[k].t_arrive - now)))
                continue
            # one round over the pool
            rc, n_active, st = self.tracer.trace(step_budget=self.round_budget, wait=True)
            stats.rounds += 1
            stats.steps += st[0]
            counts = gray.gray_count_active(self.tracer.ctx, self.tracer.state, self.tracer.n,
                                            [(s.first, s.n) for (_, s, _) in inflight])
            still = []
            for (req, slot, t_admit), c in zip(inflight, counts):
                if c == 0:
                    self._finish(req, slot, t_admit, stats)
                else:
                    still.append((req, slot, t_admit))
            inflight = still
        stats.wall = time.perf_counter() - self._t0
        return stats


def render_alone(image, opt: gray.Options):
    """One request traced by itself in its own buffer (for comparison)."""
    import torch
    tr = gray.Tracer(opt, image.nx * image.ny)
    tr.setup([image])
    while True:
        rc, n_active, _ = tr.trace()
        if n_active == 0:
            break
    out = tr.render(gray.RENDER_PIXELS32)
    torch.cuda.synchronize()
    px = out.cpu().numpy().view(gray.PIXEL32_DTYPE)
    tr.close()
    return px
