"""Continuous-batching request loop over the egb C ABI.

Requests (a medium plus a source description) arrive over time.  The loop admits them while the
library accepts new solves (egb_source refuses with EGB_E_NOMEM when free device memory is short;
the request then waits), keeps every admitted solve resident on the device, and advances all of
them together in chunks of pseudo-time steps with egb_evolve_batch, so requests that arrive while
others are on the GPU join at the next chunk boundary and their work overlaps on the device.  When a
solve has taken all its steps it is superposed, its results are copied out and its memory is freed,
which admits waiting requests.  Latency = completion time - arrival time.  A request can be cancelled
at any time (Request.cancel, e.g. from another thread): the loop drops it if it is still waiting, or
releases its solve at the next chunk boundary if it is on the GPU.

The loop only schedules; every step of the method runs in the CUDA library.  `Backend` wraps the
library calls so that the scheduling logic can also be driven by a fake backend on the CPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds since the start of the stream
    problem: object         # synthmedia.Problem2D
    kmax: int = 8
    # filled by the loop
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: object = None
    steps_left: int = 0
    medium: object = None   # backend's handle of the request's medium
    solve: int = 0
    cancelled: bool = False

    def cancel(self):
        """Ask the loop to drop this request (honoured before admission or between chunks)."""
        self.cancelled = True


class NoMemory(Exception):
    """The backend refused a new solve for lack of device memory."""


class Backend:
    """The egb library behind the loop (one context, one CUDA stream).

    Requests whose problems share a stiffness array share one uploaded medium, and with it the
    characteristic velocities the library keeps per medium and angle count; a medium stays
    resident while a request uses it, and up to `keep_media` idle media are kept for later
    requests (released first when the device runs short of memory)."""

    def __init__(self, device=0, stream=0, keep_media=8):
        import paper_2006_11945_gb300 as egb
        self.egb = egb
        self.ctx = egb.Context(device, stream)
        self.keep_media = keep_media
        self.media = {}    # key -> [medium id, users, stiffness array (kept alive so its id stays unique)]
        self.idle = []     # keys of media without users, oldest first

    @staticmethod
    def _key(p):
        return (id(p.c21), p.nx, p.nz, p.hx, p.hz)

    def _release_idle(self, keep):
        while len(self.idle) > keep:
            key = self.idle.pop(0)
            mid = self.media.pop(key)[0]
            self.egb.egb_release(self.ctx.h, mid)

    def _medium(self, p):
        key = self._key(p)
        if key in self.media:
            ent = self.media[key]
            if ent[1] == 0:
                self.idle.remove(key)
            ent[1] += 1
            return key, ent[0]
        try:
            m = self.ctx.medium_2d(p)
        except self.egb.EgbError as e:
            if e.status != self.egb.EGB_E_NOMEM or not self.idle:
                raise
            self._release_idle(0)
            m = self.ctx.medium_2d(p)
        self.media[key] = [m, 1, p.c21]
        return key, m

    def _unuse(self, key):
        ent = self.media[key]
        ent[1] -= 1
        if ent[1] == 0:
            self.idle.append(key)
            self._release_idle(self.keep_media)

    def admit(self, req: Request):
        egb = self.egb
        p = req.problem
        try:
            key, m = self._medium(p)
        except egb.EgbError as e:
            if e.status == egb.EGB_E_NOMEM:
                raise NoMemory() from e
            raise
        try:
            s = self.ctx.source_2d(m, p)
        except egb.EgbError as e:
            if e.status == egb.EGB_E_NOMEM and self.idle:
                self._release_idle(0)
                try:
                    s = self.ctx.source_2d(m, p)
                except egb.EgbError as e2:
                    self._unuse(key)
                    if e2.status == egb.EGB_E_NOMEM:
                        raise NoMemory() from e2
                    raise
            else:
                self._unuse(key)
                if e.status == egb.EGB_E_NOMEM:
                    raise NoMemory() from e
                raise
        req.medium, req.solve = key, s

    def evolve(self, reqs: List[Request], steps: List[int], cfl: float):
        self.egb.egb_evolve_batch(self.ctx.h, [r.solve for r in reqs], steps, cfl)

    def finish(self, req: Request):
        p = req.problem
        res = self.ctx.superpose(req.solve, len(p.freqs), p.nz, p.nx, req.kmax)
        self.egb.egb_sync(self.ctx.h)
        self.egb.egb_release(self.ctx.h, req.solve)
        self._unuse(req.medium)
        return res

    def cancel(self, req: Request):
        """Free the solve of a request cancelled while on the device (no superposition)."""
        self.egb.egb_sync(self.ctx.h)
        self.egb.egb_release(self.ctx.h, req.solve)
        self._unuse(req.medium)

    def close(self):
        self.ctx.close()


@dataclass
class ServeStats:
    completed: List[Request] = field(default_factory=list)
    cancelled: List[Request] = field(default_factory=list)
    unfinished: List[Request] = field(default_factory=list)   # on the device when wall_limit hit
    not_admitted: List[Request] = field(default_factory=list)  # still queued when admission closed
    refused_admissions: int = 0
    chunks: int = 0
    work: float = 0.0       # cell-updates advanced on the device (finished or not)
    max_active: int = 0
    wall: float = 0.0

    def summary(self, offered: int):
        lat = np.array([r.finished - r.arrival for r in self.completed]) if self.completed else np.zeros(0)
        cells = sum(r.problem.cells * r.problem.steps for r in self.completed)
        return {
            'offered': offered, 'completed': len(self.completed), 'cancelled': len(self.cancelled),
            'unfinished': len(self.unfinished), 'not_admitted': len(self.not_admitted),
            'solves_per_s': len(self.completed) / self.wall if self.wall > 0 else 0.0,
            'cell_updates_per_s': cells / self.wall if self.wall > 0 else 0.0,
            'device_cell_updates_per_s': self.work / self.wall if self.wall > 0 else 0.0,
            'p50_latency_s': float(np.percentile(lat, 50)) if lat.size else None,
            'p99_latency_s': float(np.percentile(lat, 99)) if lat.size else None,
            'max_active': self.max_active, 'chunks': self.chunks,
            'refused_admissions': self.refused_admissions, 'wall_s': self.wall,
        }


def _chunk_steps(req: Request, chunk_steps: int, chunk_work: Optional[float]) -> int:
    """Steps a request takes in one chunk: chunk_steps, or with a work budget, the steps worth
    about chunk_work cell-updates (at least chunk_steps), never more than it has left."""
    n = chunk_steps
    if chunk_work is not None:
        n = max(n, int(chunk_work // max(1, req.problem.cells)))
    return min(n, req.steps_left if req.steps_left > 0 else req.problem.steps)


def serve(requests: List[Request], backend, chunk_steps: int = 30, cfl: float = 0.5,
          time_limit: Optional[float] = None, clock: Callable[[], float] = time.perf_counter,
          max_active: Optional[int] = None, wall_limit: Optional[float] = None,
          chunk_work: Optional[float] = None, max_chunk_work: Optional[float] = None) -> ServeStats:
    """Run the request stream through the backend; returns the statistics.

    Arrival times are honoured against `clock` (requests become visible once the wall time since
    the start reaches their arrival).  With `time_limit`, no request is admitted after that time
    and the loop returns once the admitted ones are done.  With `wall_limit`, the loop stops at the
    first chunk boundary after that time: requests still on the device are released unfinished.

    Scheduling.  By default every active request advances chunk_steps steps per chunk and waiting
    requests are admitted in arrival order.  With `chunk_work` (cell-updates) a request advances
    about that much work per chunk instead, so a small solve finishes in one chunk; with
    `max_chunk_work` waiting requests are admitted shortest-remaining-work first while the work of
    the next chunk stays within that bound (one request is always admitted into an idle device), so
    chunks, and with them the latency of small requests, stay short under load.
    """
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    waiting: deque = deque()
    active: List[Request] = []
    stats = ServeStats()
    t0 = clock()
    while pending or waiting or active:
        now = clock() - t0
        if wall_limit is not None and now >= wall_limit:
            for r in active:
                backend.cancel(r)
                stats.unfinished.append(r)
            active = []
            stats.not_admitted.extend(waiting)
            stats.not_admitted.extend(pending)
            break
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        admitting = time_limit is None or now < time_limit
        if not admitting:
            stats.not_admitted.extend(waiting)
            stats.not_admitted.extend(pending)
            pending.clear()
            waiting.clear()
        # cancellations: waiting requests are dropped, solves on the device released
        for r in [r for r in waiting if r.cancelled]:
            waiting.remove(r)
            stats.cancelled.append(r)
        for r in [r for r in active if r.cancelled]:
            active.remove(r)
            backend.cancel(r)
            stats.cancelled.append(r)
        # admission by free device memory (and, with max_chunk_work, by the next chunk's work)
        if max_chunk_work is not None:
            waiting = deque(sorted(waiting, key=lambda r: (r.problem.cells * r.problem.steps, r.arrival)))
        work = sum(r.problem.cells * _chunk_steps(r, chunk_steps, chunk_work) for r in active)
        while admitting and waiting and (max_active is None or len(active) < max_active):
            req = waiting[0]
            add = req.problem.cells * _chunk_steps(req, chunk_steps, chunk_work)
            if max_chunk_work is not None and active and work + add > max_chunk_work:
                break
            try:
                backend.admit(req)
            except NoMemory:
                stats.refused_admissions += 1
                break
            waiting.popleft()
            req.admitted = clock() - t0
            req.steps_left = req.problem.steps
            active.append(req)
            work += add
        stats.max_active = max(stats.max_active, len(active))
        if not active:
            if pending:
                # idle until the next arrival
                nxt = pending[0].arrival
                while clock() - t0 < nxt:
                    time.sleep(min(1e-3, max(0.0, nxt - (clock() - t0))))
            continue
        steps = [_chunk_steps(r, chunk_steps, chunk_work) for r in active]
        backend.evolve(active, steps, cfl)
        stats.chunks += 1
        stats.work += sum(r.problem.cells * n for r, n in zip(active, steps))
        for r, s in zip(active, steps):
            r.steps_left -= s
        done = [r for r in active if r.steps_left <= 0]
        active = [r for r in active if r.steps_left > 0]
        for r in done:
            r.result = backend.finish(r)
            r.finished = clock() - t0
            stats.completed.append(r)
    stats.wall = clock() - t0
    return stats
