"""The benchmark's host logic on CPU: the multi-rank path (gloo, world size
2) and the update count behind the metric.

With N GPUs the benchmark runs N independent problems, one per rank, with no
collective on the data path: each rank solves its own seeded porous problem,
and only the final timings and counts cross ranks (maximum of the timings,
sum of the counts).  The reference arm runs on rank 0 alone.  These tests
drive that host logic through torch.distributed with the gloo backend; no
GPU is involved.
"""
import argparse
import contextlib
import io
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: timings (10 + r, 5 (r + 1)), counts (100 (r + 1), 7)
        times, counts = bench.reduce_over_ranks(dist, "cpu", [10.0 + rank, 5.0 * (rank + 1)],
                                                [100.0 * (rank + 1), 7])
        dist.barrier()
        out.put((rank, times, counts))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_2():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, times, counts = out.get(timeout=120)
        got[rank] = (times, counts)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        times, counts = got[rank]
        assert times == [11.0, 10.0]          # maximum over ranks
        assert counts == [300.0, 14.0]        # whole-job sums


def test_reduce_over_ranks_single_process_is_identity():
    assert bench.reduce_over_ranks(None, "cpu", [3.5, 2], [7, 8.0]) == ([3.5, 2.0], [7.0, 8.0])


def test_ranks_get_independent_problems_of_equal_size():
    """Weak scaling: every rank solves a problem of the same size and
    structure, with its own seeded obstacles."""
    p0, p1 = bench.workload(seed=0), bench.workload(seed=1)
    assert p0.dim == p1.dim and tuple(p0.n) == tuple(p1.n) and p0.nlevels == p1.nlevels
    assert len(p0.shapes) == len(p1.shapes)
    assert not np.array_equal(np.asarray(p0.shapes), np.asarray(p1.shapes))
    assert bench.updates_per_solve(p0, 25) == bench.updates_per_solve(p1, 25)


def test_reference_arm_runs_on_rank_0_only():
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args, 1, 2) == 0
    assert buf.getvalue() == ""


def test_update_count_matches_the_free_dofs_of_the_oracle():
    """The metric counts one update per free DoF per sweep on every smoothed
    level; bench.free_dofs counts them in closed form, the oracle's
    constraint mask counts them directly."""
    import dataclasses

    from oracle import oracle as O
    from paper_2403_11636_gb300 import inputs
    probs = [inputs.porous_3d(0, n=8, nspheres=3, nlevels=2),
             dataclasses.replace(inputs.porous_3d(1, n=8, nspheres=3, nlevels=2), preset=0),
             inputs.channel_2d(0, n=16, nlevels=3),
             dataclasses.replace(inputs.channel_2d(1, n=16, nlevels=3), preset=1)]
    for p in probs:
        total = 0
        for level in range(2, p.nlevels + 1):
            L = O.Level.from_problem(p, level)
            L.assemble()
            fixed = L.csr()[2]
            assert bench.free_dofs(p, level) == fixed.size - int(fixed.sum()), (p.name, level)
            total += fixed.size - int(fixed.sum())
        assert bench.updates_per_solve(p, 3) == 3 * (p.nu_pre + p.nu_post) * total
