"""Continuous-batching solve server on one GPU.

Requests (a chain, a tolerance, an arrival time) are admitted first come,
first served while the device memory they need fits an HBM budget and a
slot is free. Each admitted request gets its own context and CUDA stream:
its chain and its cash and history stay resident on the device, and its
whole solve (Alg. 1 to its own tolerance) runs as one device-side loop
(rlgl_solve_async). The solves of all admitted requests run at the same
time on the GPU. The host loop only admits, polls for completions
(rlgl_query), reads each finished estimate and frees the slot and its
memory, so requests that arrive while others are running start as soon as
memory and a slot allow, not when a batch ends.

Because every request runs in its own context, its result does not depend
on what else is running: the same request alone or in the mix follows the
same arithmetic (up to the order of floating-point atomic additions).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Iterable, List, Optional

import numpy as np

from . import rlgl


@dataclasses.dataclass
class Request:
    id: int
    arrival: float            # seconds after the start of the run
    csr: object               # synth.CSR (host arrays, ideally pinned)
    tol: float
    schedule: str = "link_threshold"
    max_steps: int = 100000


@dataclasses.dataclass
class Result:
    id: int
    status: str
    moves: int
    edges_pushed: int
    pi: Optional[np.ndarray]
    arrival: float
    start: float              # admitted (context creation began)
    finish: float             # estimate read back
    n: int

    @property
    def latency(self) -> float:
        return self.finish - self.arrival

    @property
    def queue_wait(self) -> float:
        return self.start - self.arrival


class Server:
    """Admission by HBM budget and slot count; one context per request."""

    def __init__(self, hbm_budget_bytes: float, max_active: int = 32, precision: str = "mixed",
                 theta_scale: float = 0.5, keep_pi: bool = True):
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.precision = precision
        self.theta_scale = theta_scale
        self.keep_pi = keep_pi
        self.stats = {}
        rlgl.load()

    def footprint(self, req: Request) -> int:
        c = req.csr
        return rlgl.footprint(c.n, int(c.row_ptr[-1]), c.w is not None, self.precision)

    def run(self, requests: Iterable[Request], realtime: bool = True) -> List[Result]:
        """Serves the requests; with realtime, each becomes visible at its
        arrival time (else all are queued at once). Returns the results in
        completion order."""
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for r in todo:
            if self.footprint(r) > self.budget:
                raise ValueError(f"request {r.id} needs more than the whole HBM budget")
        queue: collections.deque = collections.deque()
        active = {}
        used = 0
        max_used = 0
        max_active = 0
        results: List[Result] = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while todo or queue or active:
            t = now()
            while todo and (not realtime or todo[0].arrival <= t):
                queue.append(todo.popleft())
            # admit in arrival order while memory and slots allow
            while queue and len(active) < self.max_active:
                r = queue[0]
                need = self.footprint(r)
                if used + need > self.budget:
                    break
                queue.popleft()
                start = now()
                ch = rlgl.Chain(r.csr, precision=self.precision)
                # Solves run side by side here: the persistent sweep (a
                # cooperative kernel that takes the whole GPU) is for a
                # solve that has the device to itself.
                ch.set_params(theta_scale=self.theta_scale, persistent=0)
                ch.solve_async(r.schedule, 0.0, r.tol, r.max_steps)
                active[r.id] = (r, ch, need, start)
                used += need
                max_used = max(max_used, used)
                max_active = max(max_active, len(active))
            # retire finished solves
            done = [rid for rid, (r, ch, need, start) in active.items() if ch.query()]
            for rid in done:
                r, ch, need, start = active.pop(rid)
                info = ch.wait(raise_on_noconv=False)
                pi = None
                if info["status"] != "RLGL_EDEGENERATE":
                    pi = ch.estimate()
                ch.close()
                used -= need
                results.append(Result(r.id, info["status"], info["moves"], info["edges_pushed"],
                                      pi if self.keep_pi else None, r.arrival, start, now(), r.csr.n))
            if not done:
                # nothing finished: wait a little (or until the next arrival)
                nxt = todo[0].arrival - now() if (realtime and todo and not queue) else 0.0
                time.sleep(min(max(nxt, 0.0), 0.002) if nxt > 0 else 0.0002)
        self.stats = {"max_used_bytes": max_used, "max_active": max_active}
        rlgl.release_retired()  # nothing runs any more
        return results


def summary(results: List[Result]) -> dict:
    """Latency percentiles (s) and throughput of a finished run."""
    lat = np.array([r.latency for r in results])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    return {
        "requests": len(results),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "solves_per_s": len(results) / span if span > 0 else float("inf"),
        "span_s": span,
        "edge_pushes": int(sum(r.edges_pushed for r in results)),
        "not_ok": int(sum(r.status != "RLGL_OK" for r in results)),
    }
