"""Continuous-batching request loop for parameter-scan simulations.

Requests (grid size N, S_csr, Pi, steps per period, number of periods) arrive
over time.  The loop keeps every admitted simulation's psi resident on the
device inside one vfps_batch and never blocks on the GPU while it waits:

* a chunk of up to `chunk_steps` steps of all active slots is queued
  (slots of the same grid size share one launch per step; different sizes
  run on their own streams and overlap), and the loop then polls the batch
  (vfps_batch_idle, no synchronisation) while it moves arrivals into the
  queue and admits them -- a new slot's upload and set-up run on the
  batch's admission stream beside the chunk in flight;
* admission takes queued requests in arrival order while a slot and the
  device-memory budget allow (the library refuses with EBUSY otherwise); a
  request that does not fit is passed over so that smaller ones behind it
  can start, but once it has been passed over `max_skips` times it holds
  the queue: nothing behind it is admitted until it fits (no starvation of
  large grids);
* when the chunk has finished, finished slots are read out and freed, and
  the next chunk starts with everything admitted meanwhile.

A request's result is its final psi, profile and CSR-power series; its
time-to-result is completion minus arrival.  All step arithmetic runs in the
library's kernels; this module only decides admission order and timing.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import vfps as V


@dataclass
class Result:
    rid: int
    n: int
    steps: int
    arrival_s: float
    admitted_s: float
    done_s: float
    psi: np.ndarray | None
    rho: np.ndarray
    power: np.ndarray

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class Stats:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    max_active: int = 0
    max_queue: int = 0
    rejected_admissions: int = 0   # admission attempts refused (slots or memory)
    passed_over: int = 0           # requests admitted ahead of an older one that did not fit
    admitted_in_flight: int = 0    # admissions made while a chunk was running on the GPU
    chunks: int = 0

    def summary(self) -> dict:
        lat = np.array([r.latency_s for r in self.results]) if self.results else np.zeros(1)
        cells = sum(r.n * r.n * r.steps for r in self.results)
        return {"requests": len(self.results), "wall_s": self.wall_s,
                "cell_updates_per_s": cells / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "max_active": self.max_active, "max_queue": self.max_queue,
                "deferred_admissions": self.rejected_admissions, "passed_over": self.passed_over,
                "admitted_while_gpu_busy": self.admitted_in_flight, "chunks": self.chunks}


class Server:
    """Serve simulation requests on one GPU with a bounded set of slots.

    max_slots: concurrent simulations; budget_bytes: device memory the slots
    may hold (0 = only the free-memory check); chunk_steps: steps between
    completion checks; keep_psi: return final psi with each result;
    max_skips: how often a request that does not fit may be passed over
    before it holds the queue; poll_s: sleep between polls of a busy GPU;
    autotune: let the library time launch shapes for the served groups (off
    by default: a served mix changes every few chunks, tuning it costs
    steps, and a shape timed under a mixed load would be cached for the
    process and reused by later pure batches of that configuration).
    """

    def __init__(self, max_slots: int = 64, budget_bytes: int = 0, chunk_steps: int = 500,
                 beta: float = 1e-2, stream=None, keep_psi: bool = True, max_skips: int = 8,
                 poll_s: float = 2e-4, autotune: bool = False):
        self.batch = V.Batch(max_slots, budget_bytes, stream)
        self.batch.autotune(autotune)
        self.chunk = chunk_steps
        self.beta = beta
        self.keep_psi = keep_psi
        self.max_skips = max_skips
        self.poll_s = poll_s
        self.active = {}  # slot -> (request, admitted time)

    def params_for(self, req) -> V.Params:
        return V.Params(n=req.n, steps_per_period=req.steps_per_period, beta=self.beta)

    def _admit(self, req, psi0, now) -> bool:
        slot = self.batch.try_add(self.params_for(req), psi0, V.IMPEDANCE_PARALLEL_PLATES, req.Pi,
                                  req.s_csr, nsteps=req.nsteps)
        if slot is None:
            return False
        self.active[slot] = (req, now)
        return True

    def _admit_queue(self, queue, skips, psi0_for, now, stats, busy):
        """Admit from the queue in arrival order; returns the requests left."""
        left = []
        blocked = False
        for req in queue:
            if blocked:
                left.append(req)
                continue
            psi0 = psi0_for(req) if psi0_for else None
            if self._admit(req, psi0, now()):
                if left:
                    stats.passed_over += 1
                if busy:
                    stats.admitted_in_flight += 1
                continue
            stats.rejected_admissions += 1
            if not self.active:
                raise V.VfpsError(V.EBUSY, f"request {req.rid} (N={req.n}) does not fit an empty batch")
            skips[req.rid] = skips.get(req.rid, 0) + 1
            left.append(req)
            if skips[req.rid] > self.max_skips:
                blocked = True  # it holds the queue until it fits
        return left

    def _collect(self, now, stats):
        for slot in self.batch.poll():
            req, t_adm = self.active.pop(slot)
            r = self.batch.take(slot, psi=self.keep_psi, rho=True)
            self.batch.remove(slot)
            stats.results.append(Result(req.rid, req.n, r["steps"], req.arrival_s, t_adm, now,
                                        r["psi"], r["rho"], r["power"]))

    def run(self, requests, psi0_for=None, realtime: bool = True) -> Stats:
        """Serve `requests` (arrival_s offsets from the start).  With realtime,
        a request is only admitted once its arrival time has passed."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        queue = []
        skips = {}
        stats = Stats()
        t0 = time.perf_counter()
        in_flight = False

        def now():
            return time.perf_counter() - t0

        while pending or queue or self.active:
            t = now()
            while pending and (not realtime or pending[0].arrival_s <= t):
                queue.append(pending.popleft())
            stats.max_queue = max(stats.max_queue, len(queue))
            if queue:
                queue = self._admit_queue(queue, skips, psi0_for, now, stats, in_flight)
            stats.max_active = max(stats.max_active, len(self.active))
            if in_flight:
                if not self.batch.idle():
                    time.sleep(self.poll_s)
                    continue
                in_flight = False
                self._collect(now(), stats)
                continue  # freed slots and memory: admit before the next chunk
            if self.active:
                self.batch.run(self.chunk)
                stats.chunks += 1
                in_flight = True
            elif pending and realtime:
                time.sleep(max(0.0, min(0.05, pending[0].arrival_s - now())))
        stats.wall_s = now()
        return stats

    def close(self):
        self.batch.close()
