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

BatchServer gives every solve the whole device, one at a time: a large
request runs alone through the persistent sweep; whenever the device is
free and the oldest request is small, every queued small request that fits
the HBM budget (and the chain cap) is stacked into one block-diagonal batch
and solved in one persistent launch, each chain to its own tolerance, and
all of them retire when that launch completes. Requests that arrive
meanwhile wait for the next solve. Each chain of a batch runs Alg. 1 on its
own statistics, threshold and stop, so its result does not depend on the
rest of the batch either.
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
        # Solves that run side by side take the phase kernels: the persistent
        # sweep (a cooperative kernel that takes the whole GPU) is for a
        # solve that has the device to itself.
        self.persistent = 1 if self.max_active == 1 else 0
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
                ch.set_params(theta_scale=self.theta_scale, persistent=self.persistent)
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


def _stack(chains):
    """Block-diagonal stack (device tensors when the chains hold them)."""
    from . import synth
    if all(rlgl._is_torch(c.row_ptr) for c in chains):
        return synth.stack_chains_device(chains)
    return synth.stack_chains(chains)


class BatchServer:
    """One solve on the device at a time, each with the whole GPU: a request
    of at least `alone_nodes` nodes runs alone through the persistent sweep;
    the small requests queued when the device is free (up to the chain cap
    and the HBM budget, in arrival order) run together as one persistent
    batch launch, each chain to its own tolerance."""

    def __init__(self, hbm_budget_bytes: float, max_chains: int = 1024, precision: str = "mixed",
                 theta_scale: float = 0.5, keep_pi: bool = True, batch_block: int = 256,
                 alone_nodes: int = 1 << 17, theta_lag: int = 1):
        self.budget = int(hbm_budget_bytes)
        self.max_chains = int(max_chains)
        self.precision = precision
        self.theta_scale = theta_scale
        self.keep_pi = keep_pi
        self.batch_block = int(batch_block)
        self.alone_nodes = int(alone_nodes)
        self.theta_lag = int(theta_lag)  # the stale threshold of a solve alone (the batch has none)
        self.stats = {}
        rlgl.load()

    def footprint(self, req: Request) -> int:
        c = req.csr
        return rlgl.footprint(c.n, int(c.row_ptr[-1]), c.w is not None, self.precision)

    def _take(self, queue: collections.deque) -> List[Request]:
        """The next solve's requests: the head alone when it is large, else
        every small queued request that fits, in arrival order."""
        if queue[0].csr.n >= self.alone_nodes:
            return [queue.popleft()]
        take, keep, used = [], collections.deque(), 0
        while queue:
            r = queue.popleft()
            need = self.footprint(r)
            if r.csr.n < self.alone_nodes and len(take) < self.max_chains and used + need <= self.budget:
                take.append(r)
                used += need
            else:
                keep.append(r)
        queue.extend(keep)
        return take

    def _start(self, take: List[Request]):
        if len(take) == 1:
            r = take[0]
            ch = rlgl.Chain(r.csr, precision=self.precision)
            ch.set_params(theta_scale=self.theta_scale, theta_lag=self.theta_lag)
            ch.solve_async(r.schedule, 0.0, r.tol, r.max_steps)
            return ch, None
        csr, node_ptr = _stack([r.csr for r in take])
        ch = rlgl.Chain(csr, precision=self.precision, node_ptr=node_ptr)
        ch.set_params(theta_scale=self.theta_scale, persistent=1, theta_lag=0, batch_block=self.batch_block)
        ch.set_chain_tol(np.array([r.tol for r in take]))
        ch.solve_async(take[0].schedule, 0.0, -1.0, max(r.max_steps for r in take))
        return ch, node_ptr

    def run(self, requests: Iterable[Request], realtime: bool = True) -> List[Result]:
        """Serves the requests; with realtime, each becomes visible at its
        arrival time (else all are queued at once). Returns the results in
        completion order."""
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for r in todo:
            if self.footprint(r) > self.budget:
                raise ValueError(f"request {r.id} needs more than the whole HBM budget")
        queue: collections.deque = collections.deque()
        active = None
        results: List[Result] = []
        batches, alone, max_used, max_chains = 0, 0, 0, 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while todo or queue or active:
            t = now()
            while todo and (not realtime or todo[0].arrival <= t):
                queue.append(todo.popleft())
            if active is None and queue:
                take = self._take(queue)
                start = now()
                ch, node_ptr = self._start(take)
                active = (take, ch, node_ptr, start)
                if len(take) > 1:
                    batches += 1
                else:
                    alone += 1
                max_used = max(max_used, sum(self.footprint(r) for r in take))
                max_chains = max(max_chains, len(take))
            if active is not None and active[1].query():
                take, ch, node_ptr, start = active
                info = ch.wait(raise_on_noconv=False)
                if node_ptr is None:
                    statuses, moves, edges = [info["status"]], [info["moves"]], [info["edges_pushed"]]
                else:
                    st, mv, _ = ch.chains()
                    statuses = [rlgl.status_name(int(x)) for x in st]
                    moves = [int(x) for x in mv]
                    edges = [0] * len(take)  # (the batch counts its links in all)
                pi = None
                try:
                    pi = ch.estimate()
                except rlgl.RLGLError:
                    pass  # a degenerate chain: no estimate
                ch.close()
                fin = now()
                for k, r in enumerate(take):
                    seg = None
                    if pi is not None and self.keep_pi:
                        seg = pi if node_ptr is None else pi[int(node_ptr[k]):int(node_ptr[k + 1])]
                    results.append(Result(r.id, statuses[k], moves[k], edges[k], seg, r.arrival, start, fin,
                                          r.csr.n))
                active = None
                continue
            if active is not None or (realtime and todo and not queue):
                nxt = todo[0].arrival - now() if (realtime and todo and not queue and active is None) else 0.0
                time.sleep(min(max(nxt, 0.0), 0.002) if nxt > 0 else 0.0002)
        self.stats = {"batches": batches, "alone": alone, "max_used_bytes": max_used, "max_chains": max_chains}
        rlgl.release_retired()
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
