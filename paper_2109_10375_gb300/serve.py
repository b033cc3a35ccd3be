"""Serving form of the z_re(x) path: a continuous-batching request loop.

Parameter studies (Sec. 5 of the paper varies z_mid, dz, Az, the source
threshold and l_mfp over one realisation) reuse most of the work.  The server
keeps, per realisation and grid, the density field on the device, and two
levels of cached results:

* per (realisation, grid, delta_c): the transformed source field
  (amber_source_spectrum: the x and y passes of the forward transform) and
  the cell masses;
* per (realisation, grid, l_mfp, delta_c): the rank order and the rank-order
  masses that the solve leaves behind.

A request that changes only the history (z_mid, dz, Az) runs only the
abundance matching (amber_assign_zre_ranked).  One that changes l_mfp starts
from the cached spectrum (amber_solve_spectrum: the z pass with the new
kernel, the inverse passes, ranking and matching).  One that changes the
source threshold reruns the source field and both forward passes first.

Continuous batching: each slot is a library context with its own CUDA
stream.  Requests that arrive while others are on the GPU are admitted as
slots free up and as free HBM allows their cache entries; their work overlaps
on the device.  All GPU work is libamber's; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np
import torch

from . import binding as B
from . import synth

BOX_PER_CELL = {128: 100.0 / 128, 256: 200.0 / 256, 512: 400.0 / 512}


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds from the start of the run
    realisation: int
    n: int
    l_mfp: float
    delta_c: float
    history: tuple            # (z_mid, dz, Az)
    # filled by the server
    start: float = math.nan
    done: float = math.nan
    hit: bool = False         # history-only: the rank order was cached
    spec_hit: bool = False    # l_mfp change: the transformed source was cached
    z: torch.Tensor | None = None

    @property
    def latency_ms(self):
        return 1e3 * (self.done - self.arrival)


def poisson_requests(n_requests: int, rate: float, seed: int = 7, sizes=(128, 256, 512),
                     size_p=(0.6, 0.3, 0.1), n_realisations: int = 20, hit_fraction: float = 0.7):
    """Seeded request stream: Poisson arrivals; a fraction changes only the history."""
    g = np.random.default_rng(seed)
    t = 0.0
    current = {}  # (realisation, n) -> (l_mfp, delta_c) last used
    out = []
    for i in range(n_requests):
        t += g.exponential(1.0 / rate)
        n = int(g.choice(sizes, p=size_p))
        r = int(g.integers(n_realisations))
        hist = (float(g.uniform(6.5, 9.0)), float(g.uniform(2.0, 6.0)), float(g.uniform(1.5, 5.0)))
        key = (r, n)
        if key in current and g.random() < hit_fraction:
            l, dc = current[key]
        else:
            l, dc = current.get(key, (5.0, 1.686))
            if key in current:
                if g.random() < 0.5:
                    l = float(g.uniform(1.0, 20.0))
                else:
                    dc = float(g.uniform(1.5, 2.0))
            current[key] = (l, dc)
        out.append(Request(i, t, r, n, l, dc, hist))
    return out


class _Slot:
    def __init__(self, max_cells: int, device: int):
        self.ctx = B.Context(max_cells, device)
        self.stream = torch.cuda.Stream(device=device)
        self.event = torch.cuda.Event()
        self.req: Request | None = None
        # per-slot source and output scratch, so concurrent requests never share them
        self.S = torch.empty(max_cells, device=f"cuda:{device}")
        self.z = torch.empty(max_cells, device=f"cuda:{device}")
        self.held = []


class Server:
    """Continuous-batching server over n_slots contexts on one GPU.

    free_bytes: a callable returning the device's free bytes (default
    torch.cuda.mem_get_info); admission keeps that above hbm_reserve after a
    request's new cache entries, evicting unused entries (least recently used
    first) and otherwise leaving the request queued until running ones end."""

    def __init__(self, n_slots: int = 6, max_n: int = 512, cache_bytes: float = 40e9, device: int = 0,
                 hbm_reserve: float = 8e9, keep_outputs: bool = False, free_bytes=None):
        self.device = device
        self.slots = [_Slot(max_n ** 3, device) for _ in range(n_slots)]
        # key -> [tensors, bytes, running users, event recorded after it was written]
        # ("order", r, n, l, dc): (order, mass_rank); ("spec", r, n, dc): (spectrum, mass)
        self.cache = collections.OrderedDict()
        self.cache_bytes = cache_bytes
        self.cached = 0
        self.fields = {}  # (realisation, n) -> density field on the device
        self.hbm_reserve = hbm_reserve
        self.keep_outputs = keep_outputs
        self.free_bytes = free_bytes or self._device_free_bytes
        self.waited = set()  # requests that had to wait for HBM at least once
        self.evictions = 0

    def _device_free_bytes(self) -> int:
        """Free device memory: the driver's free bytes plus what torch's caching
        allocator holds reserved but unused (evicted entries return there)."""
        free, _ = torch.cuda.mem_get_info(self.device)
        return free + torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)

    # --- inputs ---------------------------------------------------------------
    def _field(self, r: int, n: int):
        key = (r, n)
        if key not in self.fields:
            box = BOX_PER_CELL[n] * n if n in BOX_PER_CELL else 100.0 * n / 128
            self.fields[key] = synth.gaussian_density(n, box, 1000 + r, device=f"cuda:{self.device}").float()
        return self.fields[key]

    def prepare(self, requests):
        """Make the density fields the requests use (outside any timed region)."""
        for q in requests:
            self._field(q.realisation, q.n)
        torch.cuda.synchronize()

    # --- admission --------------------------------------------------------------
    @staticmethod
    def _order_key(q: Request):
        return ("order", q.realisation, q.n, q.l_mfp, q.delta_c)

    @staticmethod
    def _spec_key(q: Request):
        return ("spec", q.realisation, q.n, q.delta_c)

    @staticmethod
    def _order_bytes(n):
        return 8 * n ** 3  # order + rank-order masses

    @staticmethod
    def _spec_bytes(n):
        return B.spectrum_bytes(n) + 4 * n ** 3  # transformed source + masses

    def _need(self, q: Request) -> int:
        """Bytes of the cache entries q would add."""
        if self._order_key(q) in self.cache:
            return 0
        need = self._order_bytes(q.n) + (4 * q.n ** 3 if self.keep_outputs else 0)
        if self._spec_key(q) not in self.cache:
            need += self._spec_bytes(q.n)
        return need

    def _admissible(self, q: Request) -> bool:
        need = self._need(q)
        if need == 0:
            return True
        protect = {self._order_key(q), self._spec_key(q)}
        while self.cached + need > self.cache_bytes or self.free_bytes() - need < self.hbm_reserve:
            if not self._evict_one(protect):
                return False
        return True

    def _evict_one(self, protect=()) -> bool:
        for k, v in self.cache.items():
            if v[2] == 0 and k not in protect:  # not in use by a running request
                self.cache.pop(k)
                self.cached -= v[1]
                self.evictions += 1
                return True
        return False

    def _put(self, key, tensors, nbytes, stream):
        ready = torch.cuda.Event()
        ready.record(stream)
        self.cache[key] = [tensors, nbytes, 1, ready]
        self.cached += nbytes

    def _use(self, key, stream):
        ent = self.cache[key]
        self.cache.move_to_end(key)
        ent[2] += 1
        stream.wait_event(ent[3])  # the entry may still be being written by another slot
        return ent[0]

    # --- execution --------------------------------------------------------------
    def _launch(self, slot: _Slot, q: Request, now: float):
        n = q.n
        box = BOX_PER_CELL.get(n, 100.0 / 128) * n
        h = B.history(*q.history)
        okey, skey = self._order_key(q), self._spec_key(q)
        dev = f"cuda:{self.device}"
        z = torch.empty((n, n, n), device=dev) if self.keep_outputs else None
        zbuf = z if z is not None else slot.z[: n ** 3].view(n, n, n)
        held = []
        with torch.cuda.stream(slot.stream):
            if okey in self.cache:
                # history only: the matching over the cached ranking
                order, mrank = self._use(okey, slot.stream)
                held.append(okey)
                slot.ctx.assign_zre_ranked(order, mrank, h, zbuf.view(-1), stream=slot.stream)
                q.hit = True
            else:
                if skey in self.cache:
                    # a new l_mfp: the z pass onward from the cached spectrum
                    spec, m = self._use(skey, slot.stream)
                    q.spec_hit = True
                else:
                    # a new threshold: source field and the two forward passes, kept
                    S = slot.S[: n ** 3].view(n, n, n)
                    m = torch.empty((n, n, n), device=dev)
                    slot.ctx.source_field(self._field(q.realisation, n), q.delta_c, 0.7, out=S, mass_out=m,
                                          stream=slot.stream)
                    spec = slot.ctx.source_spectrum(S, stream=slot.stream)
                    self._put(skey, (spec, m), self._spec_bytes(n), slot.stream)
                held.append(skey)
                order = torch.empty(n ** 3, dtype=torch.int32, device=dev)
                mrank = torch.empty(n ** 3, device=dev)
                slot.ctx.solve_spectrum(spec, m, box, q.l_mfp, h, zbuf, order, mrank, stream=slot.stream)
                self._put(okey, (order, mrank), self._order_bytes(n), slot.stream)
                held.append(okey)
            slot.event.record(slot.stream)
        q.start = now
        q.z = z
        slot.req = q
        slot.held = held

    def _finish(self, slot: _Slot, now: float):
        q = slot.req
        q.done = now
        for k in slot.held:
            if k in self.cache:
                self.cache[k][2] = max(0, self.cache[k][2] - 1)
        slot.req = None

    def run(self, requests, realtime: bool = True):
        """Serve the requests; returns them with start/done times filled in."""
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        queue = collections.deque()
        t0 = time.perf_counter()
        while pending or queue or any(s.req is not None for s in self.slots):
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                queue.append(pending.popleft())
            for s in self.slots:
                if s.req is not None and s.event.query():
                    self._finish(s, time.perf_counter() - t0)
            for s in self.slots:
                if s.req is None and queue:
                    if not self._admissible(queue[0]):
                        if all(x.req is None for x in self.slots):
                            raise RuntimeError(f"request {queue[0].rid} ({queue[0].n}^3) does not fit the HBM "
                                               "budget even with every cache entry evicted")
                        self.waited.add(queue[0].rid)  # queued until a running request ends
                        break
                    self._launch(s, queue.popleft(), time.perf_counter() - t0)
            if not queue and pending and realtime:
                dt = pending[0].arrival - (time.perf_counter() - t0)
                if dt > 0 and all(s.req is None for s in self.slots):
                    time.sleep(min(dt, 0.002))
        torch.cuda.synchronize()
        for s in self.slots:
            st = s.ctx.sync_status(s.stream)
            if st != 0:
                raise RuntimeError(f"device status {B.status_string(st)}")
        return requests

    @property
    def waiting_hbm(self) -> int:
        return len(self.waited)

    def close(self):
        for s in self.slots:
            s.ctx.close()
        self.cache.clear()
        self.fields.clear()


def summarize(requests) -> dict:
    lat = np.array([q.latency_ms for q in requests])
    cells = sum(q.n ** 3 for q in requests)
    span = max(q.done for q in requests) - min(q.arrival for q in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "cells_per_s": cells / span, "hit_rate": float(np.mean([q.hit for q in requests])),
            "spectrum_hit_rate": float(np.mean([q.spec_hit for q in requests])),
            "makespan_s": span}
