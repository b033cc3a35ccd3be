"""Serving form of the z_re(x) path: a continuous-batching request loop.

Parameter studies (Sec. 5 of the paper varies z_mid, dz, Az, the source
threshold and l_mfp over one realisation) reuse most of the work.  The server
keeps, per realisation and grid, the density field on the device and, per
(realisation, grid, l_mfp, delta_c), the rank order and the rank-order masses
that amber_solve_ex leaves behind.  A request that changes only the history
(z_mid, dz, Az) then runs only the abundance matching
(amber_assign_zre_ranked); one that changes l_mfp or the threshold reruns the
source field, the radiation field and the ranking.

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
    hit: bool = False
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
        # per-slot source and mass scratch, so concurrent misses never share them
        self.S = torch.empty(max_cells, device=f"cuda:{device}")
        self.m = torch.empty(max_cells, device=f"cuda:{device}")
        self.z = torch.empty(max_cells, device=f"cuda:{device}")


class Server:
    """Continuous-batching server over n_slots contexts on one GPU."""

    def __init__(self, n_slots: int = 6, max_n: int = 512, cache_bytes: float = 40e9, device: int = 0,
                 hbm_reserve: float = 8e9, keep_outputs: bool = False):
        self.device = device
        self.slots = [_Slot(max_n ** 3, device) for _ in range(n_slots)]
        # key -> [order, mass_rank, bytes, running users, event recorded after it was written]
        self.cache = collections.OrderedDict()
        self.cache_bytes = cache_bytes
        self.cached = 0
        self.fields = {}  # (realisation, n) -> density field on the device
        self.hbm_reserve = hbm_reserve
        self.keep_outputs = keep_outputs
        self.waiting_hbm = 0

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
    def _entry_bytes(self, n):
        return 8 * n ** 3  # order + rank-order masses

    def _admissible(self, q: Request) -> bool:
        key = (q.realisation, q.n, q.l_mfp, q.delta_c)
        if key in self.cache:
            return True
        need = self._entry_bytes(q.n) + 4 * q.n ** 3
        free, _ = torch.cuda.mem_get_info(self.device)
        while self.cached + need > self.cache_bytes or free - need < self.hbm_reserve:
            if not self._evict_one():
                return False
            free, _ = torch.cuda.mem_get_info(self.device)
        return True

    def _evict_one(self) -> bool:
        for k, v in self.cache.items():
            if v[3] == 0:  # not in use by a running request
                self.cache.pop(k)
                self.cached -= v[2]
                return True
        return False

    # --- execution --------------------------------------------------------------
    def _launch(self, slot: _Slot, q: Request, now: float):
        n = q.n
        box = BOX_PER_CELL.get(n, 100.0 / 128) * n
        h = B.history(*q.history)
        key = (q.realisation, n, q.l_mfp, q.delta_c)
        d = self._field(q.realisation, n)
        z = torch.empty((n, n, n), device=f"cuda:{self.device}") if self.keep_outputs else None
        zbuf = z if z is not None else slot.z[: n ** 3].view(n, n, n)
        with torch.cuda.stream(slot.stream):
            if key in self.cache:
                ent = self.cache[key]
                self.cache.move_to_end(key)
                ent[3] += 1
                slot.stream.wait_event(ent[4])  # the entry may still be being written by another slot
                slot.ctx.assign_zre_ranked(ent[0], ent[1], h, zbuf.view(-1), stream=slot.stream)
                q.hit = True
            else:
                # a new l_mfp or threshold: source field, radiation field, rank
                S = slot.S[: n ** 3].view(n, n, n)
                m = slot.m[: n ** 3].view(n, n, n)
                slot.ctx.source_field(d, q.delta_c, 0.7, out=S, mass_out=m, stream=slot.stream)
                order = torch.empty(n ** 3, dtype=torch.int32, device=f"cuda:{self.device}")
                mrank = torch.empty(n ** 3, device=f"cuda:{self.device}")
                slot.ctx.solve_ex(S, m, box, q.l_mfp, h, zbuf, order, mrank, stream=slot.stream)
                ready = torch.cuda.Event()
                ready.record(slot.stream)
                nbytes = self._entry_bytes(n)
                self.cache[key] = [order, mrank, nbytes, 1, ready]
                self.cached += nbytes
            slot.event.record(slot.stream)
        q.start = now
        q.z = z
        slot.req = q
        slot.key = key

    def _finish(self, slot: _Slot, now: float):
        q = slot.req
        q.done = now
        k = slot.key
        if k in self.cache:
            self.cache[k][3] = max(0, self.cache[k][3] - 1)
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
                        self.waiting_hbm += 1
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
            "makespan_s": span}
