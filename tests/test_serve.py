"""Scheduling logic of the continuous-batching server (CPU, fake solver) and,
on the GPU, that every result is the same alone and in the mix."""
import threading
import time

import numpy as np
import pytest

from paper_2403_11636_gb300 import inputs
from paper_2403_11636_gb300.serve import BatchServer, Request, Server, latency_stats


class FakeProblem:
    def __init__(self, fp, dur):
        self.fp, self.dur = fp, dur


def make_fake(log):
    lock = threading.Lock()
    active = {"mem": 0, "n": 0, "max_mem": 0, "max_n": 0}

    def solve(p, stream):
        with lock:
            active["mem"] += p.fp
            active["n"] += 1
            active["max_mem"] = max(active["max_mem"], active["mem"])
            active["max_n"] = max(active["max_n"], active["n"])
        time.sleep(p.dur)
        with lock:
            active["mem"] -= p.fp
            active["n"] -= 1
        log.append(p)
        return 3, 1e-9, 0.0, p.dur, None

    return solve, active


def test_admission_respects_budget_and_slots():
    log = []
    solve, active = make_fake(log)
    reqs = [Request(k, FakeProblem(fp=40 + 10 * (k % 3), dur=0.02), arrival=0.001 * k) for k in range(12)]
    srv = Server(solve, lambda p: p.fp, budget_bytes=100, slots=3)
    res = srv.run(reqs)
    assert [r.rid for r in res] == list(range(12))
    assert active["max_mem"] <= 100 and active["max_n"] <= 3
    assert active["max_n"] >= 2          # work overlapped
    assert all(r.admitted >= r.arrival - 1e-9 and r.finished >= r.admitted for r in res)


def test_fifo_order_and_arrivals_wait():
    log = []
    solve, _ = make_fake(log)
    reqs = [Request(0, FakeProblem(90, 0.05), 0.0), Request(1, FakeProblem(90, 0.01), 0.01),
            Request(2, FakeProblem(5, 0.01), 0.02)]
    res = Server(solve, lambda p: p.fp, budget_bytes=100, slots=4).run(reqs)
    # request 2 fits next to request 0 but arrives after request 1, which
    # does not fit: first come, first served keeps it waiting
    assert res[2].admitted >= res[1].admitted
    assert res[1].admitted >= res[0].finished - 1e-3


def test_oversized_request_rejected():
    solve, _ = make_fake([])
    with pytest.raises(ValueError):
        Server(solve, lambda p: p.fp, budget_bytes=10, slots=1).run([Request(0, FakeProblem(11, 0.0), 0.0)])


def test_failed_request_is_reported_and_frees_its_slot():
    """A request whose solve raises (an FcError from setup, for instance)
    frees its slot and memory; every other request is still served, and
    run() reports the failure at the end."""
    log = []
    solve, active = make_fake(log)

    def flaky(p, stream):
        if p.fp == 77:
            raise RuntimeError("setup failed")
        return solve(p, stream)

    reqs = [Request(k, FakeProblem(fp=77 if k == 2 else 30, dur=0.01), arrival=0.002 * k) for k in range(8)]
    with pytest.raises(RuntimeError) as e:
        Server(flaky, lambda p: p.fp, budget_bytes=100, slots=1).run(reqs)
    assert "1 requests failed" in str(e.value) and "setup failed" in str(e.value)
    assert len(log) == 7 and active["mem"] == 0 and active["n"] == 0


def test_latency_stats():
    from paper_2403_11636_gb300.serve import Result
    rs = [Result(k, 0.0, 0.0, float(k + 1), 1, 0.0, 0.0, 0.0, 0) for k in range(100)]
    st = latency_stats(rs)
    assert st["p50_s"] in (50.0, 51.0) and st["p99_s"] >= 99.0 and abs(st["solves_per_s"] - 1.0) < 1e-12


def test_serving_stream_recipe():
    s1 = inputs.serving_stream(0, count=20)
    s2 = inputs.serving_stream(0, count=20)
    assert [t for t, _ in s1] == [t for t, _ in s2]
    gaps = np.diff([0.0] + [t for t, _ in inputs.serving_stream(1, count=400)])
    assert 0.015 < gaps.mean() < 0.025          # mean gap 1/50 s
    for _, p in s1:
        assert p.n[0] in (16, 32, 48, 64, 96) and 5 <= len(p.shapes) <= 200
        assert p.n[0] % 2 ** (p.nlevels - 1) == 0


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build
    build.build()
    probs = [inputs.porous_3d(k, n=16, nspheres=5 + 3 * k, nlevels=3) for k in range(4)]
    probs.append(inputs.porous_3d(9, n=32, nspheres=20, nlevels=4))
    alone = Server.gpu(budget_bytes=150e9, slots=1, keep_solutions=True).run(
        [Request(k, p, 0.0) for k, p in enumerate(probs)])
    mixed = Server.gpu(budget_bytes=150e9, slots=4, keep_solutions=True).run(
        [Request(k, p, 0.0) for k, p in enumerate(probs)])
    for a, m in zip(alone, mixed):
        assert a.iterations == m.iterations and m.relres <= 1e-8
        np.testing.assert_array_equal(a.solution, m.solution)


def make_batch_fakes(setup_dur=0.02, round_dur=0.05):
    """Fakes of setup / round / release that record memory in flight, the
    rounds and which requests each round held."""
    lock = threading.Lock()
    st = {"mem": 0, "max_mem": 0, "n": 0, "max_n": 0, "rounds": []}

    def setup(p, stream):
        with lock:
            st["mem"] += p.fp
            st["n"] += 1
            st["max_mem"] = max(st["max_mem"], st["mem"])
            st["max_n"] = max(st["max_n"], st["n"])
        if getattr(p, "fail", False):
            with lock:
                st["mem"] -= p.fp
                st["n"] -= 1
            raise RuntimeError("setup failed")
        time.sleep(p.dur if p.dur else setup_dur)
        return p

    def solve_round(handles, stream):
        with lock:
            st["rounds"].append([h.rid for h in handles])
        time.sleep(round_dur)
        return [(5, 1e-9, None) for _ in handles]

    def release(h):
        with lock:
            st["mem"] -= h.fp
            st["n"] -= 1

    return setup, solve_round, release, st


class FP:
    def __init__(self, rid, fp, dur=0.0, fail=False):
        self.rid, self.fp, self.dur, self.fail = rid, fp, dur, fail


def test_batch_server_rounds_budget_and_slots():
    setup, solve_round, release, st = make_batch_fakes()
    reqs = [Request(k, FP(k, 30 + 10 * (k % 3)), arrival=0.003 * k) for k in range(16)]
    res = BatchServer(setup, solve_round, release, lambda p: p.fp, budget_bytes=150, slots=4).run(reqs)
    assert [r.rid for r in res] == list(range(16))
    assert st["max_mem"] <= 150 and st["max_n"] <= 4
    assert max(len(r) for r in st["rounds"]) >= 2            # sweeps of several requests batched
    assert sorted(sum(st["rounds"], [])) == list(range(16))  # every request solved in exactly one round
    assert all(r.round_size == len(st["rounds"][r.round_id]) for r in res)
    assert all(r.arrival <= r.admitted + 1e-9 <= r.finished + 1e-9 for r in res)
    assert st["mem"] == 0 and st["n"] == 0


def test_batch_server_arrival_during_round_joins_a_later_round():
    setup, solve_round, release, st = make_batch_fakes(setup_dur=0.01, round_dur=0.2)
    reqs = [Request(0, FP(0, 10), 0.0), Request(1, FP(1, 10), 0.0), Request(2, FP(2, 10), 0.1)]
    res = BatchServer(setup, solve_round, release, lambda p: p.fp, budget_bytes=100, slots=8).run(reqs)
    r0 = {r.rid: r.round_id for r in res}
    assert r0[2] > r0[0]
    assert res[2].finished > res[0].finished


def test_batch_server_fifo_admission_by_memory():
    setup, solve_round, release, st = make_batch_fakes(setup_dur=0.01, round_dur=0.05)
    reqs = [Request(0, FP(0, 90), 0.0), Request(1, FP(1, 90), 0.001), Request(2, FP(2, 5), 0.002)]
    res = BatchServer(setup, solve_round, release, lambda p: p.fp, budget_bytes=100, slots=4).run(reqs)
    # request 2 fits beside request 0 but arrives after request 1, which does not
    assert res[2].admitted >= res[1].admitted
    assert res[1].admitted >= res[0].finished - 1e-3


def test_batch_server_failed_setup_reported_and_rest_served():
    setup, solve_round, release, st = make_batch_fakes()
    reqs = [Request(k, FP(k, 20, fail=(k == 3)), arrival=0.002 * k) for k in range(6)]
    with pytest.raises(RuntimeError) as e:
        BatchServer(setup, solve_round, release, lambda p: p.fp, budget_bytes=100, slots=2).run(reqs)
    assert "1 requests failed" in str(e.value)
    assert sorted(sum(st["rounds"], [])) == [0, 1, 2, 4, 5]
    assert st["mem"] == 0 and st["n"] == 0


@pytest.mark.gpu
def test_batched_results_same_alone_and_in_the_mix():
    """Rounds of in-flight requests share one fc_batch; with the fixed tile a
    request's solution is bit-identical when it is served alone (a round of
    one) and in the mix, and every request reaches the tolerance."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build
    build.build()
    probs = [inputs.porous_3d(k, n=16, nspheres=5 + 3 * k, nlevels=3) for k in range(4)]
    probs.append(inputs.porous_3d(9, n=32, nspheres=20, nlevels=4))
    for prec in ("fp32", "fp64"):
        alone = BatchServer.gpu(budget_bytes=150e9, slots=1, prec=prec, keep_solutions=True).run(
            [Request(k, p, 0.0) for k, p in enumerate(probs)])
        mixed = BatchServer.gpu(budget_bytes=150e9, slots=5, prec=prec, keep_solutions=True, gather_s=5.0).run(
            [Request(k, p, 0.0) for k, p in enumerate(probs)])
        assert all(a.round_size == 1 for a in alone)
        assert max(m.round_size for m in mixed) >= 2
        for a, m in zip(alone, mixed):
            assert a.iterations == m.iterations and m.relres <= 1e-8
            np.testing.assert_array_equal(a.solution, m.solution)


def test_batch_server_gather_window_fills_a_round():
    setup, solve_round, release, st = make_batch_fakes(setup_dur=0.0, round_dur=0.02)
    reqs = [Request(k, FP(k, 10, dur=0.01 * (k + 1)), 0.0) for k in range(4)]
    BatchServer(setup, solve_round, release, lambda p: p.fp, budget_bytes=100, slots=4, gather_s=1.0).run(reqs)
    assert st["rounds"] == [[0, 1, 2, 3]]


class LiveFP(FP):
    """A request of the live fakes that converges in its `cycles`-th restart
    cycle."""

    def __init__(self, rid, fp, cycles):
        super().__init__(rid, fp)
        self.cycles = cycles


def make_live_fakes(setup_dur=0.01, cycle_dur=0.03):
    """Fakes for the live driver: the state of a request counts the restart
    cycles it has run; a cycle reports 30 iterations, or 7 and convergence
    in the request's last cycle.  Records the members of every cycle."""
    setup, _, release, st = make_batch_fakes(setup_dur=setup_dur)
    st["cycles"] = []

    def cycle(items, stream):
        st["cycles"].append([h.rid for h, _ in items])
        time.sleep(cycle_dur)
        out = []
        for h, state in items:
            done = (state or 0) + 1
            conv = done >= h.cycles
            out.append((7 if conv else 30, 1e-9 if conv else 1e-3, done, conv))
        return out

    return setup, cycle, release, st


def test_live_batch_server_joins_and_leaves_between_cycles():
    setup, cycle, release, st = make_live_fakes(cycle_dur=0.05)
    reqs = [Request(0, LiveFP(0, 10, 6), 0.0), Request(1, LiveFP(1, 10, 2), 0.0), Request(2, LiveFP(2, 10, 2), 0.12)]
    res = BatchServer(setup, None, release, lambda p: p.fp, budget_bytes=100, slots=8, cycle_fn=cycle).run(reqs)
    assert [r.rid for r in res] == [0, 1, 2]
    cyc = st["cycles"]
    # request 2 arrives while request 0 is still cycling and joins a live batch with it
    assert any(0 in c and 2 in c for c in cyc)
    # each request runs exactly its cycles and leaves after the last one
    assert sum(0 in c for c in cyc) == 6 and sum(1 in c for c in cyc) == 2 and sum(2 in c for c in cyc) == 2
    # iterations add up over the cycles: 30 per unconverged cycle, 7 in the last
    assert res[0].iterations == 5 * 30 + 7 and res[1].iterations == 30 + 7
    assert res[2].finished < res[0].finished
    assert all(r.relres <= 1e-9 for r in res) and st["mem"] == 0 and st["n"] == 0


def test_live_batch_server_budget_slots_and_cap():
    setup, cycle, release, st = make_live_fakes(cycle_dur=0.01)
    reqs = [Request(k, LiveFP(k, 30 + 10 * (k % 3), 1 + k % 4), arrival=0.004 * k) for k in range(12)]
    res = BatchServer(setup, None, release, lambda p: p.fp, budget_bytes=150, slots=4, cycle_fn=cycle,
                      max_iters=60).run(reqs)
    assert [r.rid for r in res] == list(range(12))
    assert st["max_mem"] <= 150 and st["max_n"] <= 4
    assert max(len(c) for c in st["cycles"]) >= 2
    # the iteration cap ends a request after the cycle that reaches it
    for r in res:
        need = 1 + r.rid % 4
        assert r.iterations == (30 * (need - 1) + 7 if need <= 2 else 60)
    assert st["mem"] == 0 and st["n"] == 0


def test_live_batch_server_failed_cycle_reports_members():
    setup, _, release, st = make_live_fakes()

    def cycle(items, stream):
        raise RuntimeError("cycle failed")

    reqs = [Request(k, LiveFP(k, 10, 1), 0.0) for k in range(3)]
    with pytest.raises(RuntimeError) as e:
        BatchServer(setup, None, release, lambda p: p.fp, budget_bytes=100, slots=4, cycle_fn=cycle).run(reqs)
    assert "requests failed" in str(e.value)
    assert st["mem"] == 0 and st["n"] == 0


@pytest.mark.gpu
def test_live_batched_results_same_alone_and_in_the_mix():
    """Live batching: requests join and leave between FGMRES restart cycles;
    a request's solution is bit-identical served alone and in the mix, and
    every request reaches the tolerance."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build
    build.build()
    probs = [inputs.porous_3d(k, n=16, nspheres=5 + 3 * k, nlevels=3) for k in range(4)]
    probs.append(inputs.porous_3d(9, n=32, nspheres=20, nlevels=4))
    for prec in ("fp32", "fp64"):
        alone = BatchServer.gpu(budget_bytes=150e9, slots=1, prec=prec, keep_solutions=True, live=True).run(
            [Request(k, p, 0.0) for k, p in enumerate(probs)])
        mixed = BatchServer.gpu(budget_bytes=150e9, slots=5, prec=prec, keep_solutions=True, live=True).run(
            [Request(k, p, 0.02 * k) for k, p in enumerate(probs)])
        assert all(a.round_size == 1 for a in alone)
        assert max(m.round_size for m in mixed) >= 2
        for a, m in zip(alone, mixed):
            assert a.iterations == m.iterations and m.relres <= 1e-8
            np.testing.assert_array_equal(a.solution, m.solution)
