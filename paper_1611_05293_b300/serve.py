"""Continuous-batching request loop for parameter-scan simulations.

Requests (grid size N, S_csr, Pi, steps per period, number of periods) arrive
over time.  The loop keeps every admitted simulation's psi resident on the
device inside one vfps_batch: at each chunk boundary it admits queued
requests while a slot and the device-memory budget allow (the library
refuses with EBUSY otherwise), advances all active slots together by up to
`chunk_steps` steps (slots of the same grid size share one launch per step;
different sizes run on their own streams and overlap), then reads out and
frees the slots that have finished.  A request's result is its final psi,
profile and CSR-power series; its time-to-result is completion minus arrival.

All step arithmetic runs in the library's kernels; this module only decides
admission order and timing.
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
    rejected_admissions: int = 0

    def summary(self) -> dict:
        lat = np.array([r.latency_s for r in self.results]) if self.results else np.zeros(1)
        cells = sum(r.n * r.n * r.steps for r in self.results)
        return {"requests": len(self.results), "wall_s": self.wall_s,
                "cell_updates_per_s": cells / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "max_active": self.max_active, "max_queue": self.max_queue,
                "deferred_admissions": self.rejected_admissions}


class Server:
    """Serve simulation requests on one GPU with a bounded set of slots.

    max_slots: concurrent simulations; budget_bytes: device memory the slots
    may hold (0 = only the free-memory check); chunk_steps: steps between
    admission/completion checks; keep_psi: return final psi with each result.
    """

    def __init__(self, max_slots: int = 64, budget_bytes: int = 0, chunk_steps: int = 500,
                 beta: float = 1e-2, stream=None, keep_psi: bool = True):
        self.batch = V.Batch(max_slots, budget_bytes, stream)
        self.chunk = chunk_steps
        self.beta = beta
        self.keep_psi = keep_psi
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
        queue = collections.deque()
        stats = Stats()
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while pending or queue or self.active:
            t = now()
            while pending and (not realtime or pending[0].arrival_s <= t):
                queue.append(pending.popleft())
            stats.max_queue = max(stats.max_queue, len(queue))
            while queue:
                req = queue[0]
                psi0 = psi0_for(req) if psi0_for else None
                if not self._admit(req, psi0, now()):
                    if not self.active:
                        raise V.VfpsError(V.EBUSY, f"request {req.rid} (N={req.n}) does not fit an empty batch")
                    stats.rejected_admissions += 1
                    break
                queue.popleft()
            stats.max_active = max(stats.max_active, len(self.active))
            if self.active:
                self.batch.run(self.chunk)
                self._collect(now(), stats)
            elif pending and realtime:
                time.sleep(max(0.0, min(0.05, pending[0].arrival_s - now())))
        stats.wall_s = now()
        return stats

    def close(self):
        self.batch.close()
