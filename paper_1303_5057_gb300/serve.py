"""Serving loop: render requests of mixed size and (a, i) with continuous
batching over a resident device pool.

Requests (one image each) arrive over time.  The pool is one state buffer of
a fixed number of ray slots; a request is admitted when a contiguous free
range large enough for its pixels exists (admission by device memory), its
rays are set up there (large requests also planned longest-first into the
pool's work queue), and from then on they are traced together with every
other request in flight: each round is one ``gray_trace`` over the pool's
queue with a step budget (finished and empty slots are skipped).  A request
therefore never waits for a batch to fill or drain; its rays overlap on the
device with everyone else's.  Because a ray's result is independent of
batching, of the queue order and of how its trace is split over calls, a
request's image is the same alone and in the mix.

The host never waits for the device inside the loop.  Each round enqueues,
on the pool's stream, the trace, ``gray_range_stats`` over the requests in
flight (active rays and steps per request), a copy of those counts to pinned
host memory and an event; the next round is enqueued while it runs.  When a
round's event has completed, the requests it shows finished are rendered
into their slots of a device image buffer, copied on a side stream into a
pinned host buffer of their own and cleared; their ranges return to the allocator once the copy
is done, and arrived requests are admitted into the free space.

Latency of a request = the host time at which its image is in host memory
(its copy's event observed complete) - its arrival time.
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
    busy: float = 0.0  # wall time with at least one request in flight

    def latencies(self):
        return np.array([r.latency for r in self.results])

    def summary(self):
        lat = self.latencies()
        return {"requests": len(self.results), "rounds": self.rounds, "photon_steps": self.steps,
                "wall_s": self.wall, "busy_s": self.busy,
                "photon_steps_per_s": self.steps / self.wall if self.wall > 0 else 0.0,
                "photon_steps_per_busy_s": self.steps / self.busy if self.busy > 0 else 0.0,
                "p50_ms": 1000.0 * float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": 1000.0 * float(np.percentile(lat, 99)) if lat.size else None,
                "max_ms": 1000.0 * float(lat.max()) if lat.size else None}


@dataclass
class _Flight:
    req: object
    slot: Slot
    t_admit: float
    steps: int = 0
    done_event: object = None  # copy of its image complete
    host: object = None        # its image in pinned host memory


class Server:
    """Continuous-batching render server over one resident pool.

    capacity: ray slots in the pool (device memory = gray_state_bytes).
    round_budget: steps each in-flight ray may take per round (measured on the
    config-5 mix at 30 req/s: p99 195 ms at 1024, 143 ms at 4096; the same
    saturated rate).
    depth: rounds enqueued ahead of the host.
    plan_min_rays: requests of at least this many rays are planned
    longest-first (gray_setup_plan) into the pool's queue; smaller ones keep
    their natural order (0: plan every request, None: plan none)."""

    def __init__(self, opt: gray.Options, capacity: int, round_budget: int = 4096, device="cuda", depth: int = 2,
                 plan_min_rays=1 << 16, probe_stride: int = 6, probe_budget: int = 400, max_requests: int = 4096):
        import torch
        self.torch = torch
        self.opt = opt
        self.capacity = int(capacity)
        self.round_budget = int(round_budget)
        self.depth = max(1, int(depth))
        self.plan_min_rays = plan_min_rays
        self.probe_stride, self.probe_budget = int(probe_stride), int(probe_budget)
        self.max_requests = int(max_requests)
        self.tracer = gray.Tracer(opt, self.capacity, device=device)
        gray.gray_clear(self.tracer.ctx, self.tracer.state, self.capacity, 0, self.capacity)
        self.alloc = PoolAllocator(self.capacity)
        self.queue = torch.arange(self.capacity, dtype=torch.int32, device=device)
        self.out_dev = torch.empty(16 * self.capacity, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream()
        self.copy_stream = torch.cuda.Stream()
        self.rings = []  # per round in flight: (ranges pinned, ranges dev, stats dev, stats pinned, event, requests)
        for _ in range(self.depth):
            self.rings.append({
                "rh": torch.empty(2 * self.max_requests, dtype=torch.int64, pin_memory=True),
                "rd": torch.empty(2 * self.max_requests, dtype=torch.int64, device=device),
                "sd": torch.empty(2 * self.max_requests, dtype=torch.int64, device=device),
                "sh": torch.empty(2 * self.max_requests, dtype=torch.int64, pin_memory=True),
                "ev": torch.cuda.Event(), "flights": None})
        self.free_rings = list(range(self.depth))
        torch.cuda.synchronize()

    def close(self):
        self.torch.cuda.synchronize()
        self.tracer.close()

    # ---- steps of the loop (all asynchronous on the pool's stream) ----

    def _admit(self, req, now, inflight):
        n = req.image.nx * req.image.ny
        if len(inflight) >= self.max_requests:
            return False
        slot = self.alloc.alloc(n)
        if slot is None:
            return False
        tr = self.tracer
        if self.plan_min_rays is not None and n >= self.plan_min_rays:
            tr.setup_plan([req.image], first_ray=slot.first, probe_stride=self.probe_stride,
                          probe_budget=self.probe_budget, order=self.queue[slot.first:slot.first + n],
                          stream=self.stream)
        else:
            tr.setup([req.image], first_ray=slot.first, stream=self.stream)
            self.queue[slot.first:slot.first + n].copy_(
                self.torch.arange(slot.first, slot.first + n, dtype=self.torch.int32, device=self.queue.device),
                non_blocking=True)
        inflight.append(_Flight(req, slot, now))
        return True

    def _enqueue_round(self, flights):
        torch = self.torch
        k = self.free_rings.pop(0)
        ring = self.rings[k]
        m = len(flights)
        rh = ring["rh"].numpy()
        for j, f in enumerate(flights):
            rh[2 * j], rh[2 * j + 1] = f.slot.first, f.slot.n
        tr = self.tracer
        # the queue up to the end of the highest range in flight (first-fit
        # keeps the ranges low in the pool)
        hi = max(f.slot.first + f.slot.n for f in flights)
        gray.gray_trace(tr.ctx, tr.state, tr.n, self.round_budget, wait=False, stream=self.stream,
                        order=self.queue[:hi])
        ring["rd"][:2 * m].copy_(ring["rh"][:2 * m], non_blocking=True)
        gray.gray_range_stats(tr.ctx, tr.state, tr.n, ring["rd"], ring["sd"], n_ranges=m, stream=self.stream)
        ring["sh"][:2 * m].copy_(ring["sd"][:2 * m], non_blocking=True)
        ring["ev"].record(self.stream)
        ring["flights"] = list(flights)
        return k

    def _finish(self, f):
        """Render the request's rays, copy its image to pinned host memory on
        the side stream, clear its slots."""
        tr, s = self.tracer, f.slot
        out = self.out_dev[16 * s.first: 16 * (s.first + s.n)]
        gray.gray_render(tr.ctx, tr.state, tr.n, gray.RENDER_PIXELS32, first_ray=s.first, n=s.n, out=out,
                         stream=self.stream)
        rendered = self.torch.cuda.Event()
        rendered.record(self.stream)
        gray.gray_clear(tr.ctx, tr.state, tr.n, s.first, s.n, stream=self.stream)
        self.copy_stream.wait_event(rendered)
        with self.torch.cuda.stream(self.copy_stream):
            # the request's own pinned buffer (from torch's caching host
            # allocator): the image is handed over without a host-side copy
            f.host = self.torch.empty(16 * s.n, dtype=self.torch.uint8, pin_memory=True)
            f.host.copy_(out, non_blocking=True)
            f.done_event = self.torch.cuda.Event()
            f.done_event.record(self.copy_stream)

    def run(self, requests, realtime: bool = True, max_wall: float = None):
        """Serve `requests` (objects with rid, t_arrive seconds, image).  With
        realtime, arrivals follow the wall clock from the start of the call;
        otherwise every request is available at once.  Returns ServerStats."""
        pending = sorted(requests, key=lambda r: r.t_arrive)
        if not realtime:
            for r in pending:
                r.t_arrive = 0.0
        waiting = []   # arrived, not admitted (FIFO)
        inflight = []  # admitted, not yet seen finished
        copying = []   # finished, image on its way to the host
        rounds = []    # ring indices of rounds in flight, oldest first
        stats = ServerStats()
        t0 = time.perf_counter()
        k = 0
        busy_since = None
        while k < len(pending) or waiting or inflight or copying or rounds:
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                break
            while k < len(pending) and pending[k].t_arrive <= now:
                waiting.append(pending[k])
                k += 1
            progressed = False
            # the oldest round: requests it shows finished
            if rounds and self.rings[rounds[0]]["ev"].query():
                kr = rounds.pop(0)
                ring = self.rings[kr]
                sh = ring["sh"].numpy()
                done_ids = set()
                for j, f in enumerate(ring["flights"]):
                    f.steps = int(sh[2 * j + 1])
                    if sh[2 * j] == 0:
                        done_ids.add(id(f))
                still = []
                for f in inflight:
                    if id(f) in done_ids:
                        self._finish(f)
                        copying.append(f)
                    else:
                        still.append(f)
                inflight = still
                self.free_rings.append(kr)
                stats.rounds += 1
                progressed = True
            # images that reached the host: done; their ranges are free again
            still = []
            for f in copying:
                if f.done_event.query():
                    t_done = time.perf_counter() - t0
                    s = f.slot
                    px = f.host.numpy().view(gray.PIXEL32_DTYPE)
                    stats.results.append(Result(f.req.rid, f.req.t_arrive, f.t_admit, t_done, px, f.steps))
                    stats.steps += f.steps
                    self.alloc.release(s)
                    progressed = True
                else:
                    still.append(f)
            copying = still
            # admission by device memory, first come first served
            while waiting and self._admit(waiting[0], now, inflight):
                waiting.pop(0)
                progressed = True
            if waiting and not inflight and not copying and not rounds:
                raise RuntimeError("request of %d rays does not fit a pool of %d" %
                                   (waiting[0].image.nx * waiting[0].image.ny, self.capacity))
            busy = bool(inflight or copying or rounds)
            if busy and busy_since is None:
                busy_since = now
            elif not busy and busy_since is not None:
                stats.busy += now - busy_since
                busy_since = None
            # keep `depth` rounds enqueued while requests are in flight
            if inflight and self.free_rings:
                # requests admitted after the last round are traced by this one
                rounds.append(self._enqueue_round(inflight))
                progressed = True
            if not progressed:
                if rounds or copying:
                    time.sleep(5e-5)
                elif k < len(pending):
                    time.sleep(max(0.0, min(0.002, pending[k].t_arrive - now)))
        end = time.perf_counter() - t0
        if busy_since is not None:
            stats.busy += end - busy_since
        self.torch.cuda.synchronize()
        stats.wall = end
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
