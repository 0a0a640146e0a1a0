"""Continuous-batching server for finite cell Stokes solves on one GPU.

Requests (a problem and its arrival time) are admitted first-come first-served
as soon as a slot is free and the request's device footprint
(``fc_footprint_estimate``) fits into what is left of the HBM budget.  Each
slot is a host thread with its own CUDA stream: it sets the problem up
(``fc_setup``: operator, patch caches, coarse solve stay resident while the
request is in flight), solves it with FGMRES-GMG and releases its memory.
Requests that arrive while others run are admitted as slots and memory free
up, and their kernels overlap on the device (separate streams; the library's
allocations are stream-ordered, so one request's setup or teardown does not
stall the others).  Every solve is deterministic and uses only its own
handle, so a result does not depend on what else is in flight.

The numerical work is all in libfc; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import heapq
import statistics
import threading
import time
from typing import Callable, List, Optional


@dataclasses.dataclass
class Request:
    rid: int
    problem: object
    arrival: float                 # seconds from the start of the run


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    iterations: int
    relres: float
    setup_s: float
    solve_s: float
    footprint: int
    solution: Optional[object] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def latency_stats(results: List[Result]) -> dict:
    lat = sorted(r.latency for r in results)
    if not lat:
        return {}
    def pct(q):
        k = max(0, min(len(lat) - 1, int(round(q * (len(lat) - 1)))))
        return lat[k]
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"requests": len(lat), "p50_s": pct(0.50), "p99_s": pct(0.99), "mean_s": statistics.mean(lat),
            "solves_per_s": len(lat) / span if span > 0 else float("inf")}


class Server:
    """FIFO admission by footprint into ``budget_bytes`` with ``slots`` slots.

    ``solve_fn(problem, stream) -> (iterations, relres, setup_s, solve_s,
    solution or None)`` and ``footprint_fn(problem) -> bytes`` make the
    scheduler testable without a GPU; ``Server.gpu(...)`` wires libfc in."""

    def __init__(self, solve_fn: Callable, footprint_fn: Callable, budget_bytes: float, slots: int,
                 make_stream: Callable = lambda: None, clock: Callable = time.perf_counter):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.solve_fn = solve_fn
        self.footprint_fn = footprint_fn
        self.budget = float(budget_bytes)
        self.slots = slots
        self.make_stream = make_stream
        self.clock = clock

    @classmethod
    def gpu(cls, budget_bytes: float = 150e9, slots: int = 8, cache: str = "inverse", prec: str = "fp32",
            dedup: int = 1, keep_solutions: bool = False, rtol: Optional[float] = None):
        import torch
        from . import fc

        def footprint(p):
            return fc.footprint_estimate(p, cache=cache, prec=prec)

        def solve(p, stream):
            with torch.cuda.stream(stream):
                t0 = time.perf_counter()
                s = fc.Solver(p, cache=cache, prec=prec, stream=stream, dedup=dedup)
                b = s.rhs()
                stream.synchronize()
                t1 = time.perf_counter()
                x, its, rr = s.solve(b, rtol=rtol if rtol is not None else p.rtol, maxit=400)
                t2 = time.perf_counter()
                sol = x.cpu().numpy() if keep_solutions else None
                s.close()
                return its, rr, t1 - t0, t2 - t1, sol

        return cls(solve, footprint, budget_bytes, slots, make_stream=lambda: torch.cuda.Stream())

    def run(self, requests: List[Request]) -> List[Result]:
        """Serve ``requests`` (arrival times relative to the call) to completion."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if self.footprint_fn(r.problem) > self.budget:
                raise ValueError(f"request {r.rid} needs more than the whole budget")
        lock = threading.Condition()
        state = {"used": 0.0, "free_slots": list(range(self.slots)), "results": [], "errors": []}
        streams = [self.make_stream() for _ in range(self.slots)]
        t0 = self.clock()
        queue: List = []   # heap of (arrival, rid, request) that have arrived
        threads = []

        def worker(slot, req, fp, admitted):
            try:
                its, rr, ts, tsol, sol = self.solve_fn(req.problem, streams[slot])
                res = Result(req.rid, req.arrival, admitted, self.clock() - t0, its, rr, ts, tsol, fp, sol)
                with lock:
                    state["results"].append(res)
            except Exception as e:  # a failed request is reported, the server keeps running
                with lock:
                    state["errors"].append((req.rid, repr(e)))
            finally:
                with lock:
                    state["used"] -= fp
                    state["free_slots"].append(slot)
                    lock.notify_all()

        i = 0
        with lock:
            while i < len(pending) or queue or len(state["free_slots"]) < self.slots:
                now = self.clock() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    heapq.heappush(queue, (pending[i].arrival, pending[i].rid, pending[i]))
                    i += 1
                # admit in arrival order while a slot and the memory allow
                while queue and state["free_slots"]:
                    req = queue[0][2]
                    fp = self.footprint_fn(req.problem)
                    if state["used"] + fp > self.budget:
                        break
                    heapq.heappop(queue)
                    slot = state["free_slots"].pop()
                    state["used"] += fp
                    th = threading.Thread(target=worker, args=(slot, req, fp, now), daemon=True)
                    threads.append(th)
                    th.start()
                if i >= len(pending) and not queue and len(state["free_slots"]) == self.slots:
                    break
                wait = None
                if i < len(pending):
                    wait = max(0.0, pending[i].arrival - (self.clock() - t0))
                lock.wait(timeout=wait if wait is not None else 0.05)
        for th in threads:
            th.join()
        if state["errors"]:
            raise RuntimeError(f"{len(state['errors'])} requests failed: {state['errors'][:3]}")
        return sorted(state["results"], key=lambda r: r.rid)
