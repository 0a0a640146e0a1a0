"""Continuous-batching servers for finite cell Stokes solves on one GPU.

Requests (a problem and its arrival time) are admitted first-come first-served
as soon as a slot is free and the request's device footprint
(``fc_footprint_estimate``) fits into what is left of the HBM budget.  An
admitted request is set up on a host thread with its own CUDA stream
(``fc_setup``: operator, patch caches and coarse solve stay resident while
the request is in flight); the library's allocations are stream-ordered, so
one request's setup or teardown does not stall the others.

``BatchServer`` batches the smoother sweeps of the requests in flight: one
driver thread takes every request whose setup has finished and solves them
together as one ``fc_batch`` (each V-cycle phase one persistent launch over
the patches of all of them, each Arnoldi step one CUDA graph, every problem
with its own FGMRES and stopping test).  In rounds (the default), requests
whose setup finishes while a round runs join the next round, while setups
keep overlapping the round on their own streams.  Live (``live=True``), the
driver runs one FGMRES restart cycle at a time over the requests in flight:
requests whose setup finished join at the next cycle boundary (starting from
x = 0), converged ones leave after the cycle that converged them, and the
others continue from their current iterate, which is exactly the restart of
FGMRES(restart).  The batch is built with a fixed patch-apply tile, so a
request's result is bit-identical alone and in any mix.

``Server`` is the unbatched form: each slot sets up and solves its own
request on its own stream, so requests only overlap as independent streams.

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


@dataclasses.dataclass
class BatchResult(Result):
    round_id: int = -1
    round_size: int = 0


class BatchServer:
    """FIFO admission by footprint into ``budget_bytes`` with ``slots``
    requests in flight (setting up, waiting for a round or solving), and one
    driver that solves the set-up requests in rounds of at most
    ``max_batch``.

    ``setup_fn(problem, stream) -> handle``, ``round_fn([handles], stream) ->
    [(iterations, relres, solution or None)]`` (one batched solve of the
    round), ``release_fn(handle)`` and ``footprint_fn(problem) -> bytes``
    make the scheduler testable without a GPU; ``BatchServer.gpu(...)`` wires
    libfc in.  ``gather_s``: once a request is ready, how long the driver
    may wait for setups still running to join the same round (0: start the
    round at once).

    With ``cycle_fn([(handle, state)], stream) -> [(iterations, relres,
    state, converged)]`` the driver runs live: one restart cycle per call
    over the requests in flight (state None for a request that has just
    joined), new requests joining and converged ones (or ones past
    ``max_iters`` iterations) leaving between cycles; a request's result
    holds ``final_fn(state)`` of its last cycle as its solution."""

    def __init__(self, setup_fn: Callable, round_fn: Callable, release_fn: Callable, footprint_fn: Callable,
                 budget_bytes: float, slots: int, max_batch: int = 64, make_stream: Callable = lambda: None,
                 clock: Callable = time.perf_counter, gather_s: float = 0.0, cycle_fn: Optional[Callable] = None,
                 max_iters: int = 400, final_fn: Callable = lambda state: state):
        if slots < 1 or max_batch < 1:
            raise ValueError("slots and max_batch must be >= 1")
        self.setup_fn = setup_fn
        self.round_fn = round_fn
        self.cycle_fn = cycle_fn
        self.max_iters = max_iters
        self.final_fn = final_fn
        self.release_fn = release_fn
        self.footprint_fn = footprint_fn
        self.budget = float(budget_bytes)
        self.slots = slots
        self.max_batch = max_batch
        self.make_stream = make_stream
        self.clock = clock
        self.gather_s = gather_s

    @classmethod
    def gpu(cls, budget_bytes: float = 150e9, slots: int = 8, prec: str = "fp32", dedup: int = 1,
            tc: str = "none", tile=(16, 256, 8), keep_solutions: bool = False, rtol: Optional[float] = None,
            max_batch: int = 64, gather_s: float = 0.0, live: bool = False, cycle_iters: int = 30):
        """libfc form.  ``live``: one FGMRES restart cycle of ``cycle_iters``
        iterations (the solvers' restart length) per batched call, requests
        joining and leaving between cycles; the batch is rebuilt only when
        its membership changes."""
        import torch
        from . import fc

        def footprint(p):
            return fc.footprint_estimate(p, cache="inverse", prec=prec)

        def setup(p, stream):
            with torch.cuda.stream(stream):
                s = fc.Solver(p, prec=prec, stream=stream, dedup=dedup, tc=tc)
                b = s.rhs()
                stream.synchronize()
            return (s, b, p)

        def solve_round(items, stream):
            with torch.cuda.stream(stream):
                B = fc.Batch([s for s, _, _ in items], stream=stream, tile=tile)
                try:
                    bp = B.pack([b for _, b, _ in items])
                    tol = rtol if rtol is not None else items[0][2].rtol
                    x, its, rr = B.solve(bp, rtol=tol, maxit=400)
                    sols = [v.cpu().numpy() for v in B.unpack(x)] if keep_solutions else [None] * len(items)
                finally:
                    B.close()
            return [(int(i), float(r), sol) for i, r, sol in zip(its, rr, sols)]

        cache = {"key": None, "batch": None}

        def solve_cycle(items, stream):
            # items: [((solver, b, problem), x or None)]
            with torch.cuda.stream(stream):
                key = tuple(id(h[0]) for h, _ in items)
                if cache["key"] != key:
                    if cache["batch"] is not None:
                        cache["batch"].close()
                    cache["batch"] = fc.Batch([h[0] for h, _ in items], stream=stream, tile=tile)
                    cache["key"] = key
                B = cache["batch"]
                bp = B.pack([h[1] for h, _ in items])
                xp = B.pack([x if x is not None else torch.zeros_like(h[1]) for h, x in items])
                tol = rtol if rtol is not None else items[0][0][2].rtol
                x, its, rr = B.solve(bp, x0=xp, rtol=tol, maxit=cycle_iters)
                xs = [v.clone() for v in B.unpack(x)]
            return [(int(i), float(r), xv, float(r) <= tol) for i, r, xv in zip(its, rr, xs)]

        def release(item):
            if cache["key"] is not None and id(item[0]) in cache["key"]:
                cache["batch"].close()  # the batch refers to the handle being released
                cache["key"], cache["batch"] = None, None
            item[0].close()

        def final(x):
            return x.cpu().numpy() if (keep_solutions and x is not None) else None

        return cls(setup, solve_round, release, footprint, budget_bytes, slots, max_batch,
                   make_stream=lambda: torch.cuda.Stream(), gather_s=gather_s,
                   cycle_fn=solve_cycle if live else None, final_fn=final)

    def run(self, requests: List[Request]) -> List[BatchResult]:
        """Serve ``requests`` (arrival times relative to the call) to completion."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if self.footprint_fn(r.problem) > self.budget:
                raise ValueError(f"request {r.rid} needs more than the whole budget")
        lock = threading.Condition()
        st = {"used": 0.0, "free_slots": list(range(self.slots)), "ready": [], "results": [], "errors": [],
              "setting_up": 0, "solving": 0, "done_admitting": False, "rounds": 0}
        streams = [self.make_stream() for _ in range(self.slots)]
        driver_stream = self.make_stream()
        t0 = self.clock()
        threads = []

        def finish(slot, fp):
            st["used"] -= fp
            st["free_slots"].append(slot)

        def setup_worker(slot, req, fp, admitted):
            try:
                t1 = self.clock()
                h = self.setup_fn(req.problem, streams[slot])
                ts = self.clock() - t1
                with lock:
                    st["ready"].append((req, h, slot, fp, admitted, ts))
                    st["setting_up"] -= 1
                    lock.notify_all()
            except Exception as e:  # a failed setup is reported; its slot is freed
                with lock:
                    st["errors"].append((req.rid, repr(e)))
                    st["setting_up"] -= 1
                    finish(slot, fp)
                    lock.notify_all()

        def driver():
            while True:
                with lock:
                    while not st["ready"] and not (st["done_admitting"] and st["setting_up"] == 0):
                        lock.wait(timeout=0.05)
                    if not st["ready"]:
                        return
                    deadline = self.clock() + self.gather_s
                    while (st["setting_up"] > 0 and len(st["ready"]) < self.max_batch
                           and self.clock() < deadline):
                        lock.wait(timeout=min(0.01, max(0.0, deadline - self.clock())))
                    batch = st["ready"][: self.max_batch]
                    del st["ready"][: len(batch)]
                    rid_round = st["rounds"]
                    st["rounds"] += 1
                t1 = self.clock()
                try:
                    outs = self.round_fn([h for _, h, _, _, _, _ in batch], driver_stream)
                    err = None
                except Exception as e:
                    outs, err = None, repr(e)
                t_end = self.clock()
                for k, (req, h, slot, fp, admitted, ts) in enumerate(batch):
                    try:
                        self.release_fn(h)
                    except Exception:
                        pass
                    with lock:
                        if err is None:
                            its, rr, sol = outs[k]
                            st["results"].append(BatchResult(req.rid, req.arrival, admitted, t_end - t0, its, rr, ts,
                                                             t_end - t1, fp, sol, rid_round, len(batch)))
                        else:
                            st["errors"].append((req.rid, err))
                        finish(slot, fp)
                        lock.notify_all()

        def live_driver():
            active = []  # requests in flight: [req, h, slot, fp, admitted, ts, state, iterations, joined, first]
            while True:
                with lock:
                    while not st["ready"] and not active and not (st["done_admitting"] and st["setting_up"] == 0):
                        lock.wait(timeout=0.05)
                    room = self.max_batch - len(active)
                    joining = st["ready"][:room]
                    del st["ready"][: len(joining)]
                    if not active and not joining:
                        return
                    cyc = st["rounds"]
                    st["rounds"] += 1
                for (req, h, slot, fp, admitted, ts) in joining:
                    active.append([req, h, slot, fp, admitted, ts, None, 0, self.clock(), cyc])
                try:
                    outs = self.cycle_fn([(a[1], a[6]) for a in active], driver_stream)
                    err = None
                except Exception as e:
                    outs, err = None, repr(e)
                t_end = self.clock()
                keep = []
                for k, a in enumerate(active):
                    req, h, slot, fp, admitted, ts = a[:6]
                    if err is None:
                        its, rr, state, conv = outs[k]
                        a[6] = state
                        a[7] += int(its)
                        if not conv and a[7] < self.max_iters:
                            keep.append(a)
                            continue
                    try:
                        self.release_fn(h)
                    except Exception:
                        pass
                    with lock:
                        if err is None:
                            st["results"].append(BatchResult(req.rid, req.arrival, admitted, t_end - t0, a[7],
                                                             float(rr), ts, t_end - a[8], fp,
                                                             self.final_fn(a[6]), a[9], len(active)))
                        else:
                            st["errors"].append((req.rid, err))
                        finish(slot, fp)
                        lock.notify_all()
                active = keep

        drv = threading.Thread(target=live_driver if self.cycle_fn is not None else driver, daemon=True)
        drv.start()
        queue: List = []
        i = 0
        with lock:
            while True:
                now = self.clock() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    heapq.heappush(queue, (pending[i].arrival, pending[i].rid, pending[i]))
                    i += 1
                while queue and st["free_slots"]:
                    req = queue[0][2]
                    fp = self.footprint_fn(req.problem)
                    if st["used"] + fp > self.budget:
                        break
                    heapq.heappop(queue)
                    slot = st["free_slots"].pop()
                    st["used"] += fp
                    st["setting_up"] += 1
                    th = threading.Thread(target=setup_worker, args=(slot, req, fp, now), daemon=True)
                    threads.append(th)
                    th.start()
                if i >= len(pending) and not queue:
                    break
                wait = max(0.0, pending[i].arrival - (self.clock() - t0)) if i < len(pending) else None
                lock.wait(timeout=wait if wait is not None else 0.05)
            st["done_admitting"] = True
            lock.notify_all()
        for th in threads:
            th.join()
        drv.join()
        if st["errors"]:
            raise RuntimeError(f"{len(st['errors'])} requests failed: {st['errors'][:3]}")
        return sorted(st["results"], key=lambda r: r.rid)
