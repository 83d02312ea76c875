"""Serving loop: continuous batching of Dirac solves over resident hierarchies.

Requests (lattice L, gauge field k, bare mass m0, R right-hand sides) arrive
over time.  Every (L, k) pair has one resident SM-AMG hierarchy (setup once,
at the field's lowest serving mass) and one slot batch of the C library
(amamg_batch_*).  A worker thread per pair, on its own CUDA stream, loops:

  admit waiting right-hand sides into free slots -> one FGMRES restart cycle
  over all occupied slots -> retire the slots whose right-hand side is done.

So right-hand sides that arrive while others are on the GPU join at the next
restart cycle, and the pairs' cycles overlap on the device.  Each slot carries
its own mass (the library shifts the fine operator per slot).  Slot counts come
from a device-memory budget (amamg_query_bytes): the resident hierarchies are
charged first, then each pair gets as many slots as its share allows.

Everything numeric runs in the C library; this module only schedules.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import amamg as A

# status of a request withdrawn by Server.cancel (a serving-level status, not a
# library code)
CANCELLED = -100
FAILED = -101          # the worker of the request's hierarchy stopped on a library error


def aggregates_for(L: int) -> List[int]:
    """Tile sides: 4 while the coarse lattice stays above 64^2, then 2 down to 32^2."""
    aggs, n = [], L
    while n > 64 and n // 4 >= 32:
        aggs.append(4)
        n //= 4
    while n > 32:
        aggs.append(2)
        n //= 2
    if not aggs:
        aggs = [4] if L >= 16 else [2]
    return aggs


@dataclass
class Request:
    rid: int
    L: int
    field: int
    m0: float
    R: int
    arrival: float                     # seconds after the start of the stream
    rhs_seed: int
    done_units: int = 0
    status: int = 0
    iterations: List[int] = field(default_factory=list)
    relres: List[float] = field(default_factory=list)
    finish: Optional[float] = None
    cancelled: bool = False


class Group:
    """One resident hierarchy and its slot batch, served by one thread."""

    def __init__(self, server, key, U, m_setup, slots, precision, restart, tol, max_iter, autotune=False):
        import torch
        self.server = server
        self.key = key
        self.L = key[0]
        self.stream = torch.cuda.Stream()
        self.params = A.make_params(aggregates_for(self.L), precision=precision, restart=restart, tol=tol,
                                    max_iter=max_iter, autotune=autotune)
        with torch.cuda.stream(self.stream):
            self.hier = A.setup(U, m_setup, self.params, stream=self.stream)
            self.batch = A.Batch(self.hier, slots)
        self.slots = slots
        self.setup_s = A.setup_seconds(self.hier)
        self.queue: List[Tuple[Request, int]] = []       # (request, rhs index)
        self.where: Dict[int, Tuple[Request, int]] = {}
        self.free = list(range(slots))
        self.cv = threading.Condition()
        self.cycles = 0
        self.busy_s = 0.0
        self.cancelling: List[Request] = []
        self.error: Optional[str] = None

    def submit(self, req: Request):
        with self.cv:
            if self.error is not None:
                req.status = FAILED
                req.finish = time.perf_counter() - self.server.t0
                return
            for i in range(req.R):
                self.queue.append((req, i))
            self.cv.notify()

    def cancel(self, req: Request):
        """Withdraws req: its queued right-hand sides are dropped now, the slots
        it holds are freed after the restart cycle in flight (if any)."""
        with self.cv:
            req.cancelled = True
            self.queue = [(r, i) for (r, i) in self.queue if r is not req]
            self.cv.notify()

    def _finish_cancelled(self):
        """Retires the slots of cancelled requests (no copy of the iterate) and
        closes requests that hold no slot any more.  Called between cycles by
        the worker, on its stream."""
        for slot, (req, i) in list(self.where.items()):
            if req.cancelled:
                self.batch.retire(slot, None, stream=self.stream)
                del self.where[slot]
                self.free.append(slot)
        for req in list(self.cancelling):
            if not any(r is req for (r, _) in self.where.values()):
                req.status = CANCELLED
                req.finish = time.perf_counter() - self.server.t0
                self.cancelling.remove(req)

    def run(self):
        """Worker loop; an exception (a library error) fails every request this
        group holds or will receive, so that no caller waits forever."""
        try:
            self._run()
        except Exception as exc:                        # noqa: BLE001 - reported through the requests
            with self.cv:
                self.error = repr(exc)
                pending = [r for (r, _) in self.queue] + [r for (r, _) in self.where.values()]
                self.queue.clear()
                self.where.clear()
            now = time.perf_counter() - self.server.t0
            for r in pending:
                if r.finish is None:
                    r.status = FAILED
                    r.finish = now

    def _run(self):
        import torch
        from . import fixtures as fx
        torch.cuda.set_device(self.server.device)
        L = self.L
        x = torch.empty(2, L, L, dtype=torch.complex128, device=self.server.device)
        while True:
            with self.cv:
                while (not self.queue and not self.where and not self.server.closing
                       and not self._pending_cancel()):
                    self.cv.wait(timeout=0.05)
                for r in self._pending_cancel():
                    self.cancelling.append(r)
                with torch.cuda.stream(self.stream):
                    self._finish_cancelled()
                if self.server.closing and not self.queue and not self.where:
                    return
                admit = []
                while self.free and self.queue:
                    admit.append((self.free.pop(0), self.queue.pop(0)))
            if not admit and not self.where:
                continue
            t0 = time.perf_counter()
            with torch.cuda.stream(self.stream):
                for slot, (req, i) in admit:
                    dpsi = fx.gaussian_rhs_device(L, L, req.rhs_seed + i, self.server.device)
                    self.batch.admit(slot, dpsi, req.m0, stream=self.stream)
                    self.where[slot] = (req, i)
                info = self.batch.cycle(stream=self.stream)
                self.cycles += 1
                for slot, (req, i) in list(self.where.items()):
                    active, done, status, iters, relres = info[slot]
                    if not done or req.cancelled:
                        continue
                    self.batch.retire(slot, x, stream=self.stream)
                    del self.where[slot]
                    self.free.append(slot)
                    req.iterations.append(iters)
                    req.relres.append(relres)
                    if status != A.OK:
                        req.status = status
                    req.done_units += 1
                    if req.done_units == req.R:
                        self.stream.synchronize()
                        req.finish = time.perf_counter() - self.server.t0
            self.busy_s += time.perf_counter() - t0

    def _pending_cancel(self) -> List[Request]:
        """Cancelled requests that still hold slots here and are not yet being closed."""
        seen = []
        for (r, _) in self.where.values():
            if r.cancelled and r.finish is None and r not in self.cancelling and r not in seen:
                seen.append(r)
        return seen


class Server:
    """Resident hierarchies for a set of gauge fields and one worker per field."""

    def __init__(self, fields: Dict[Tuple[int, int], Tuple[object, float]], mem_budget_bytes: int,
                 max_slots: int = 16, precision: int = A.SOLVE_MIXED, restart: int = 30, tol: float = 1e-10,
                 max_iter: int = 3000, device=None, autotune: bool = True):
        """fields[(L, k)] = (U on the device, setup mass); autotune: each
        hierarchy's coarse smoother is timed and picked at its first batch
        cycle (amamg_params.autotune)."""
        import torch
        self.device = device or torch.device("cuda:0")
        self.closing = False
        self.t0 = time.perf_counter()
        # memory admission: hierarchies first, then slots in proportion to the budget left
        need = {}
        total_setup = 0
        for key in fields:
            L = key[0]
            p = A.make_params(aggregates_for(L), precision=precision, restart=restart)
            sb, rb = A.query_bytes(p, L, L, 1)
            need[key] = (sb, rb)
            total_setup += sb
        left = mem_budget_bytes - total_setup
        if left <= 0:
            raise MemoryError("the resident hierarchies alone exceed the memory budget")
        per_group = left / len(fields)
        self.groups: Dict[Tuple[int, int], Group] = {}
        for key, (U, m_setup) in fields.items():
            sb, rb = need[key]
            slots = int(max(1, min(max_slots, per_group // rb)))
            self.groups[key] = Group(self, key, U, m_setup, slots, precision, restart, tol, max_iter, autotune)
        self.threads = []

    def start(self):
        """Starts one worker per resident hierarchy (again after close(): the
        hierarchies stay resident between request streams)."""
        self.closing = False
        self.stalled = False
        self.t0 = time.perf_counter()
        self.threads = [threading.Thread(target=g.run, daemon=True) for g in self.groups.values()]
        for t in self.threads:
            t.start()

    def submit(self, req: Request):
        self.groups[(req.L, req.field)].submit(req)

    def cancel(self, req: Request):
        """Withdraws a submitted request (its right-hand sides stop at the end of
        the restart cycle in flight; status CANCELLED)."""
        g = self.groups[(req.L, req.field)]
        g.cancel(req)
        with g.cv:
            if req.finish is None and not any(r is req for (r, _) in g.where.values()):
                req.status = CANCELLED                  # nothing admitted yet: done at once
                req.finish = time.perf_counter() - self.t0

    def close(self):
        """Stops the workers after the work they hold (a stalled stream's workers
        are left to finish on their own: daemon threads)."""
        self.closing = True
        for g in self.groups.values():
            with g.cv:
                g.cv.notify()
        for t in self.threads:
            t.join(timeout=None if not getattr(self, "stalled", False) else 1.0)


def serve(server: Server, requests: List[Request], time_scale: float = 1.0, max_idle_s: float = 900.0) -> dict:
    """Releases requests at their arrival times, waits for all, returns metrics.
    If no request finishes for max_idle_s seconds while some are open, the
    open ones are marked FAILED (a watchdog: the caller never waits forever)."""
    server.start()
    for req in sorted(requests, key=lambda r: r.arrival):
        delay = req.arrival * time_scale - (time.perf_counter() - server.t0)
        if delay > 0:
            time.sleep(delay)
        req.arrival = time.perf_counter() - server.t0
        server.submit(req)
    last_done, last_t = -1, time.perf_counter()
    while True:
        open_ = [r for r in requests if r.finish is None]
        if not open_:
            break
        done = len(requests) - len(open_)
        if done != last_done:
            last_done, last_t = done, time.perf_counter()
        elif time.perf_counter() - last_t > max_idle_s:
            now = time.perf_counter() - server.t0
            for r in open_:
                r.status = FAILED
                r.finish = now
            server.stalled = True
            break
        time.sleep(0.005)
    wall = time.perf_counter() - server.t0
    server.close()
    lat = np.array([r.finish - r.arrival for r in requests])
    solves = sum(r.R for r in requests)
    return {
        "requests": len(requests), "solves": solves, "wall_s": wall,
        "solves_per_s": solves / wall, "requests_per_s": len(requests) / wall,
        "latency_p50_ms": float(np.percentile(lat, 50) * 1e3), "latency_p99_ms": float(np.percentile(lat, 99) * 1e3),
        "not_converged": sum(1 for r in requests if r.status not in (A.OK, CANCELLED, FAILED)),
        "failed": sum(1 for r in requests if r.status == FAILED),
        "errors": sorted({g.error for g in server.groups.values() if g.error is not None}),
        "cancelled": sum(1 for r in requests if r.status == CANCELLED),
        "max_true_relres": float(max([max(r.relres) for r in requests if r.relres], default=0.0)),
        "slots": {f"{k[0]}/{k[1]}": g.slots for k, g in server.groups.items()},
        "cycles": sum(g.cycles for g in server.groups.values()),
    }


def poisson_requests(n: int, rate: float, pairs, mcrit, seed: int = 100, max_rhs: int = 16,
                     dm=(0.005, 0.1)) -> List[Request]:
    """n requests with exponential inter-arrival times (rate per second); each draws
    its (lattice, field) pair uniformly from `pairs` (the resident hierarchies),
    its mass offset m0 - m_crit ~ U[dm] and R ~ U{1..max_rhs}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = sorted(pairs)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        L, k = pairs[int(rng.integers(0, len(pairs)))]
        m0 = mcrit[(L, k)] + rng.uniform(*dm)
        R = int(rng.integers(1, max_rhs + 1))
        out.append(Request(i, L, k, float(m0), R, t, rhs_seed=1_000_000 + 100 * i))
    return out
