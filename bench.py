#!/usr/bin/env python
"""Benchmark: FGMRES-GMG solves of the 3D porous-medium finite cell Stokes
problem (64^3 background grid, 40 seeded spheres, alpha = 1e-8, octree depth 3,
5 levels, V(2,2), rtol 1e-8) with the restricted additive smoother, by
default with FP64 patch rows and FP64 arithmetic throughout (the plain
method).  --prec df64 / fp32 / bf16 selects the reduced-precision rows.

A step is one complete solve from x0 = 0 on the resident hierarchy (operator,
patch caches and coarse inverse built once per problem by fc_setup, whose time
is reported separately as setup_ms).  The metric is smoother owned-DoF
updates per second: every sweep of every smoothed level updates each free DoF
once, so one solve performs  its * (nu_pre + nu_post) * sum_l free_dofs(l)
updates.  value = those updates over all ranks / max-over-ranks wall time of
the K timed solves (CUDA events on the solver's stream, nothing else
instrumented).  Per-kernel times for the roofline come from a separate pass
of profiled solves after the timed ones.  With FP64 rows the patch apply is
bound by the FP64 pipe (GB300 runs FP64 at 1/64 of the FP32 rate), so its
roofline is FP64 FLOP/s against the nominal pipe peak, with the live FMA
probe and the HBM fraction beside it.

--impl reference times the FP64 CPU oracle (the plain implementation the
tests compare against) on the host cores, on a bounded sample of the same
workload (a 16^3 grid of the same sphere geometry, 3 levels).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "smoother patch-DoF updates/s"
UNIT = "owned-DoF updates/s"


def free_dofs(prob, level):
    """Free (unconstrained) DoFs of a level: counting only."""
    n = prob.level_n(level)
    dim = prob.dim
    nodes = 1
    for k in n:
        nodes *= k + 1
    if prob.preset == 1:
        inner = (n[1] - 1) * ((n[2] - 1) if dim == 3 else 1) * (n[0] + 1)
        fixed_nodes = nodes - inner
    elif prob.preset == 0:
        inner = n[0] * (n[1] - 1) * ((n[2] - 1) if dim == 3 else 1)
        fixed_nodes = nodes - inner
    else:
        fixed_nodes = 0
    return nodes * (dim + 1) - fixed_nodes * dim


def updates_per_solve(prob, its):
    per_cycle = sum(free_dofs(prob, l) for l in range(2, prob.nlevels + 1)) * (prob.nu_pre + prob.nu_post)
    return its * per_cycle


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [t.strip() for t in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sms.append(float(f[1]))
                    maxes.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() in ("active", "1", "yes"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes), "samples": len(sms),
                "reasons": sorted(reasons)}


def workload(seed=0):
    from paper_2403_11636_gb300 import inputs
    return inputs.porous_3d(seed)


def sample_workload(seed=0):
    from paper_2403_11636_gb300 import inputs
    return inputs.porous_3d(seed, n=16, nlevels=3)


def oracle_solve_rate(prob, budget_s=15.0, steps=None):
    """Oracle FGMRES-GMG solves on the host cores; returns rates per solve."""
    from oracle import oracle as O
    mg = O.MG(prob)                     # assembly + cached inverse rows (setup, untimed)
    b = mg.rhs()
    times, its_all = [], []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        _, its, rr, _ = mg.fgmres(b, rtol=prob.rtol, restart=prob.restart)
        times.append(time.perf_counter() - t0)
        its_all.append(its)
        if steps is not None and len(times) >= steps:
            break
        if steps is None and time.perf_counter() - t_start >= budget_s:
            break
    ups = [updates_per_solve(prob, i) for i in its_all]
    return ups, times, O.num_threads(), its_all


def emit(d):
    print(json.dumps(d), flush=True)


def reduce_over_ranks(dist, device, times, counts):
    """Whole-job aggregates of independent per-rank runs: the maximum over
    ranks of each timing and the sum over ranks of each count (identity
    without a process group).  Returns (times, counts) as lists of floats."""
    if dist is None:
        return [float(v) for v in times], [float(v) for v in counts]
    import torch
    t = torch.tensor([float(v) for v in times], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    prob = sample_workload()
    from oracle import oracle as O
    O.build()
    mg_warm = None
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_solve_rate(prob, steps=1)
    ups, times, cores, its = oracle_solve_rate(prob, steps=args.steps)
    value = sum(ups) / sum(times)
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": "porous3d sample: 16^3 grid, the 40-sphere geometry of seed 0, 3 levels, "
                                 "V(2,2), FGMRES(30) to 1e-8", "iterations": its[0]},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": "oracle FGMRES-GMG solves on the 16^3 sample, setup excluded"},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    del mg_warm
    return 0


FP64_FMA_PER_CLK_PER_SM = 2      # GB300: FP64 at 1/64 of the FP32 rate (128 FMA/clk/SM)


def fp64_peak(torch):
    """Nominal FP64 FMA throughput from unit counts and the maximum SM clock:
    SMs x 2 FP64 FMA/clock x 2 FLOP x clock (GB300: 152 x 2 x 2 x 2.07 GHz =
    1.2586 TFLOP/s, the 1.25 TFLOP/s of the part's data).  Returns TFLOP/s and
    a note of the figures used."""
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    tf = nsm * FP64_FMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12
    return tf, f"derived: {nsm} SMs x {FP64_FMA_PER_CLK_PER_SM} FP64 FMA/clk x 2 FLOP x {mhz:.0f} MHz"


def pct(vals, q):
    """Nearest-rank percentile of a list (q in (0, 100])."""
    v = sorted(vals)
    return v[min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))]


def timed_solves(s, b, prob, steps, stream, torch):
    """`steps` solves from x0 = 0 bracketed by CUDA events on the solver's
    stream; returns (per-step ms, total ms, iterations, relres)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    its_list, rr_list = [], []
    for k in range(steps):
        _, its, rr = s.solve(b, rtol=prob.rtol)
        its_list.append(its)
        rr_list.append(rr)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return step_ms, ev[0].elapsed_time(ev[-1]), its_list, rr_list


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2403_11636_gb300 import build, fc

    build.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob = workload(seed=rank)
    stream = torch.cuda.Stream()
    # arithmetic peaks of this GPU, measured before the timed region
    fp64_probe, _ = fc.probe_fma_rate("fp64")
    fp32_probe, _ = fc.probe_fma_rate("fp32")
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        s = fc.Solver(prob, cache=args.cache, prec=args.prec, stream=stream, dedup=args.dedup)
        torch.cuda.synchronize()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        b = s.rhs()
        for _ in range(args.warmup):
            x, its, rr = s.solve(b, rtol=prob.rtol)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # ---- headline: the timed solves, nothing instrumented
        clocks = Clocks(local_rank)
        clocks.start()
        l0 = fc.launch_count()
        step_ms, total_ms, its_list, rr_list = timed_solves(s, b, prob, args.steps, stream, torch)
        launches = fc.launch_count() - l0
        cl = clocks.stop()
        if dist:
            dist.barrier()
        # ---- per-kernel times from a separate profiled pass (CUDA events on
        # the solver stream around every apply / residual / V-cycle)
        s.profile(True)
        timed_solves(s, b, prob, max(1, min(args.steps, args.profile_steps)), stream, torch)
        n_apply, ms_apply, _ = s.profile_read(0)
        n_fine, ms_fine, bytes_fine = s.profile_read(4)
        n_res, ms_res, _ = s.profile_read(1)
        n_vc, ms_vc, _ = s.profile_read(2)
        s.profile(False)
        flops_fine = s.info()["bytes"][6]
        # ---- end to end through the public API with host buffers
        n = s.ndof()
        bh = torch.empty(n, dtype=torch.float64, pin_memory=True)
        bh.copy_(b.cpu())
        xh = torch.zeros(n, dtype=torch.float64, pin_memory=True)
        s.solve_host(bh, xh, rtol=prob.rtol)
        e2e_t = []
        for _ in range(args.steps):
            xh.zero_()
            t1 = time.perf_counter()
            its_h, rr_h = s.solve_host(bh, xh, rtol=prob.rtol)
            e2e_t.append(time.perf_counter() - t1)
        x_ref = torch.from_numpy(xh.numpy().copy())
        # ---- variants on rank 0: the float-pair solve, and one finest-level
        # sweep per cache policy / precision
        variants = {}
        if rank == 0 and args.policies:
            variants = {"solves": {**pair_solve_variant(prob, stream, args, s, b, x_ref),
                                   **galerkin_solve_variant(prob, stream, args, b, x_ref)},
                        "sweeps": policy_sweeps(prob, stream, args)}
    my_updates = sum(updates_per_solve(prob, i) for i in its_list)
    my_e2e_updates = updates_per_solve(prob, its_h) * len(e2e_t)
    (total_ms, e2e_ms), (all_updates, all_e2e) = reduce_over_ranks(
        dist, "cuda", [total_ms, sum(e2e_t) * 1e3], [my_updates, my_e2e_updates])
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        s.close()
        return 0
    hbm, peak_kind = peaks()
    avg_fine_ms = ms_fine / max(n_fine, 1)
    gbs = bytes_fine / (avg_fine_ms * 1e-3) / 1e9 if ms_fine > 0 else 0.0
    tflops = flops_fine / (avg_fine_ms * 1e-3) / 1e12 if ms_fine > 0 else 0.0
    traffic = load_traffic(args.prec) if not args.dedup else None
    if args.prec == "fp64":
        peak_tf, peak_note = fp64_peak(torch)
        roof = {"bound": "alu", "achieved": tflops, "peak": peak_tf, "unit": "TFLOP/s", "frac": tflops / peak_tf,
                "traffic": traffic, "pipe": "FP64 (DFMA)",
                "peak_source": peak_note,
                "peak_probe_tflops": fp64_probe / 1e12, "frac_of_probe": tflops / (fp64_probe / 1e12),
                "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm, "peak_source": peak_kind}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": traffic,
                "peak_source": peak_kind}
    roof.update({"kernel": "patch apply (cache_inverse) on the finest level", "launches": n_fine,
                 "avg_launch_ms": avg_fine_ms, "algorithmic_bytes_per_launch": bytes_fine,
                 "algorithmic_flop_per_launch": flops_fine,
                 "timing": f"CUDA events on the solver stream around every finest-level apply of "
                           f"{max(1, min(args.steps, args.profile_steps))} profiled solves after the timed ones"})
    out = {
        "metric": METRIC, "value": all_updates / (total_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "df64": "f32x2", "fp32": "f32", "bf16": "bf16"}[args.prec],
        "data": "synthetic",
        "config": {"workload": "porous3d 64^3 background grid, 40 non-overlapping seeded spheres "
                               "r~U[0.04,0.12], alpha 1e-8, octree depth 3, 5 levels, V(2,2), "
                               "FGMRES(30) rtol 1e-8, Q1-Q1 (1,098,500 DoFs)",
                   "cache": args.cache, "patch_rows": args.prec, "shared_class_blocks": bool(args.dedup),
                   "l2": "inputs larger than L2 (cached rows 4.1 GB per V-cycle)",
                   "iterations": its_list[0], "relres": max(rr_list), "setup_ms": setup_ms,
                   "solves_per_s": world * args.steps / (total_ms * 1e-3),
                   "latency_ms": {"p50": pct(step_ms, 50), "p99": pct(step_ms, 99), "n": len(step_ms),
                                  "note": "p99 of fewer than 100 samples is their maximum"},
                   "smoother_profiled_pass": {"apply_launches": n_apply, "apply_ms": ms_apply,
                                              "residual_launches": n_res, "residual_ms": ms_res,
                                              "vcycles": n_vc, "vcycle_ms": ms_vc},
                   "arith_probe": {"fp64_tflops": fp64_probe / 1e12, "fp32_tflops": fp32_probe / 1e12},
                   "parallelism": f"{world} independent problems, one per GPU" if world > 1 else "1 GPU",
                   "variants": variants},
        "roofline": roof,
        "e2e": {"value": all_e2e / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 2 * n * 8,
                "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches,
        "clocks": cl,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    emit(out)
    if dist:
        dist.destroy_process_group()
    s.close()
    return 0


def pair_solve_variant(prob, stream, args, s64, b, x64):
    """The float-pair rows (df64: rows, residual and x as float32 pairs inside
    the FP64 FGMRES) on the same workload: updates/s of the same timed solves,
    and how far they land from the FP64 GPU path of this run (solution, and
    one finest-level sweep).  The oracle parity of both paths is tested."""
    import torch
    from paper_2403_11636_gb300 import fc, inputs
    try:
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            sd = fc.Solver(prob, cache="inverse", prec="df64", stream=stream, dedup=args.dedup)
            torch.cuda.synchronize()
            setup_ms = 1e3 * (time.perf_counter() - t0)
            for _ in range(max(1, args.warmup)):
                sd.solve(b, rtol=prob.rtol)
            step_ms, total_ms, its_l, rr_l = timed_solves(sd, b, prob, args.steps, stream, torch)
            x, _, _ = sd.solve(b, rtol=prob.rtol)
            dx = (x.cpu() - x64).norm().item() / max(x64.norm().item(), 1e-300)
            x0 = torch.as_tensor(inputs.random_vector(prob, 3)).cuda()
            bb = torch.as_tensor(inputs.random_vector(prob, 4)).cuda()
            s_d = sd.smooth(x0, bb) - x0
            s_f = s64.smooth(x0, bb) - x0
            dsw = (s_d - s_f).norm().item() / max(s_f.norm().item(), 1e-300)
            sd.profile(True)
            timed_solves(sd, b, prob, 1, stream, torch)
            n_fine, ms_fine, bytes_fine = sd.profile_read(4)
            sd.profile(False)
            sd.close()
        hbm, _ = peaks()
        gbs = bytes_fine / (ms_fine / max(n_fine, 1) * 1e-3) / 1e9 if ms_fine > 0 else None
        return {"df64/per-patch": {
            "dtype": "f32x2", "updates_per_s": sum(updates_per_solve(prob, i) for i in its_l) / (total_ms * 1e-3),
            "ms_per_solve": total_ms / len(step_ms), "iterations": its_l[0], "relres": max(rr_l),
            "setup_ms": setup_ms,
            "solution_rel_diff_vs_fp64_gpu": dx, "sweep_rel_diff_vs_fp64_gpu": dsw,
            "oracle_parity": "per sweep <= 1e-10 relative (tests: test_gpu_fullsize, test_gpu_midsize, "
                             "test_gpu_parity)",
            "finest_apply_ms": ms_fine / max(n_fine, 1),
            "finest_apply_hbm_frac": gbs / hbm if gbs else None}}
    except Exception as e:  # reported, not fatal for the headline
        return {"df64/per-patch": {"error": str(e)[:200]}}


def galerkin_solve_variant(prob, stream, args, b, x64):
    """FP64 rows with Galerkin coarse operators (R L P of the next finer
    operator, no quadrature on the coarser grids) on the same workload:
    setup time, iterations and updates/s of the same timed solves, and the
    distance of the solution from the rediscretised hierarchy's."""
    import torch
    from paper_2403_11636_gb300 import fc
    try:
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            sg = fc.Solver(prob, cache="inverse", prec="fp64", stream=stream, dedup=args.dedup, galerkin=True)
            torch.cuda.synchronize()
            setup_ms = 1e3 * (time.perf_counter() - t0)
            for _ in range(max(1, args.warmup)):
                sg.solve(b, rtol=prob.rtol)
            step_ms, total_ms, its_l, rr_l = timed_solves(sg, b, prob, args.steps, stream, torch)
            x, _, _ = sg.solve(b, rtol=prob.rtol)
            dx = (x.cpu() - x64).norm().item() / max(x64.norm().item(), 1e-300)
            sg.close()
        return {"fp64/galerkin": {
            "dtype": "f64", "updates_per_s": sum(updates_per_solve(prob, i) for i in its_l) / (total_ms * 1e-3),
            "ms_per_solve": total_ms / len(step_ms), "iterations": its_l[0], "relres": max(rr_l),
            "setup_ms": setup_ms, "solution_rel_diff_vs_rediscretised": dx,
            "oracle_parity": "tests/test_gpu_galerkin.py (coarse operators 1e-12, V-cycle 1e-10, FGMRES counts)"}}
    except Exception as e:  # reported, not fatal for the headline
        return {"fp64/galerkin": {"error": str(e)[:200]}}


def cpu_baseline(args):
    """The FP64 CPU oracle on the host cores, on a bounded sample of the
    workload: FGMRES-GMG solves of the same 40-sphere geometry on a 16^3 grid
    (3 levels; the metric's unit), and per-sweep times of the finest level of
    that sample with every host thread and with one."""
    from oracle import oracle as O
    prob = sample_workload()
    ups, times, cores, its = oracle_solve_rate(prob, budget_s=args.cpu_budget)
    out = {"value": sum(ups) / sum(times), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(times)} oracle FGMRES-GMG solves of a 16^3 grid of the same 40-sphere geometry "
                     f"(3 levels, {its[0]} iterations), setup (assembly, patch inverses) excluded"}
    try:
        sw = oracle_sweep_rate(args.cpu_sweep_n)
        out["per_sweep"] = sw
    except Exception as e:
        out["per_sweep"] = {"error": str(e)[:200]}
    return out


def oracle_sweep_rate(n):
    """Per-sweep time of the oracle (residual + cached-row patch apply over
    every patch) on the finest level of an n^3 grid of the benchmark
    geometry, with every host thread and with one; setup excluded."""
    from oracle import oracle as O
    from paper_2403_11636_gb300 import inputs
    prob = inputs.porous_3d(0, n=n, nlevels=max(2, int(math.log2(n // 4)) + 1))
    L = O.Level.from_problem(prob)
    L.assemble()
    L.build_inverse()
    x = inputs.random_vector(prob, 3)
    b = inputs.random_vector(prob, 4)
    res = {"grid": f"{n}^3", "free_dofs": free_dofs(prob, prob.nlevels)}
    nthr = O.num_threads()
    for label, thr in (("all_threads", nthr), ("one_thread", 1)):
        O.set_threads(thr)
        L.sweep(b, x)
        ts = []
        t_end = time.perf_counter() + 3.0
        while time.perf_counter() < t_end or len(ts) < 3:
            t0 = time.perf_counter()
            L.sweep(b, x)
            ts.append(time.perf_counter() - t0)
        ms = 1e3 * statistics.median(ts)
        res[label] = {"threads": thr, "sweep_ms": ms, "updates_per_s": res["free_dofs"] / (ms * 1e-3),
                      "samples": len(ts)}
    O.set_threads(nthr)
    return res


def run_sweeps(args):
    """Finest-level smoother sweeps only (for bounded-size profiler captures):
    setup of a porous problem with n^3 cells, then --warmup + --steps sweeps."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    if args.workload == "roofline2d":
        # 2D roofline case: n^2 cells, one circle r = 0.2, alpha 1e-10,
        # levels halved down to 16^2 cells
        prob = inputs.roofline_2d(n=args.n, nlevels=max(2, int(math.log2(args.n // 16)) + 1))
    else:
        nlev = max(2, int(math.log2(args.n // 4)) + 1)
        prob = inputs.porous_3d(0, n=args.n, nlevels=nlev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        s = fc.Solver(prob, cache=args.cache, prec=args.prec, stream=stream, dedup=args.dedup)
        torch.cuda.synchronize()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        x = torch.as_tensor(inputs.random_vector(prob, 3)).cuda()
        b = torch.as_tensor(inputs.random_vector(prob, 4)).cuda()
        s.smooth_(x, b, nsweeps=args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.profile(True)
        e0.record(stream)
        s.smooth_(x, b, nsweeps=args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        na, ma, ba = s.profile_read(0)
        nr, mr, _ = s.profile_read(1)
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
    upd = free_dofs(prob, prob.nlevels)
    hbm, _ = peaks()
    wl = f"roofline2d {args.n}^2 finest-level sweeps" if args.workload == "roofline2d" else \
        f"porous3d {args.n}^3 finest-level sweeps"
    emit({"mode": "sweep", "workload": wl, "cache": args.cache,
          "prec": args.prec, "dedup": args.dedup, "cache_bytes": s.info()["bytes"][1], "sweep_ms": ms, "updates_per_s": upd / (ms * 1e-3),
          "apply_ms": ma / max(na, 1), "apply_bytes": ba, "residual_ms": mr / max(nr, 1),
          "apply_gbs": ba / (ma / max(na, 1) * 1e-3) / 1e9 if ma > 0 else None,
          "apply_frac_of_measured_hbm": (ba / (ma / max(na, 1) * 1e-3) / 1e9) / hbm if ma > 0 else None,
          "setup_ms": setup_ms})
    s.close()
    return 0


def run_serve(args):
    """Serving stream: Poisson arrivals (mean 50/s) of 3D porous solves on
    grids {16,32,48,64,96}^3 with 5-200 spheres, admitted by HBM footprint
    into a budget, FGMRES to 1e-8.  Five arms with the same slots, budget
    and shared class blocks, so that batching and precision separate:
    batched rounds (BatchServer: the sweeps of the requests in flight share
    fc_batch launches) and per-slot streams (Server), each with float32
    rows (the mixed-precision form) and with FP64 rows (the plain method);
    and live batching with float32 rows (requests join and leave the batch
    between FGMRES restart cycles)."""
    from paper_2403_11636_gb300 import build, inputs
    from paper_2403_11636_gb300.serve import BatchServer, Request, Server, latency_stats
    build.build()
    stream = inputs.serving_stream(0, count=args.requests, rate=args.rate)
    reqs = [Request(k, p, t) for k, (t, p) in enumerate(stream)]
    budget = args.budget_gb * 1e9
    arms = {}
    clocks = Clocks(0)
    clocks.start()
    for name, make in (
            ("batched_fp32", lambda: BatchServer.gpu(budget_bytes=budget, slots=args.slots, prec="fp32", dedup=1,
                                                     tc=args.tc)),
            ("batched_fp64", lambda: BatchServer.gpu(budget_bytes=budget, slots=args.slots, prec="fp64", dedup=1)),
            ("live_fp32", lambda: BatchServer.gpu(budget_bytes=budget, slots=args.slots, prec="fp32", dedup=1,
                                                  tc=args.tc, live=True)),
            ("streams_fp32", lambda: Server.gpu(budget_bytes=budget, slots=args.slots, prec="fp32", dedup=1)),
            ("streams_fp64", lambda: Server.gpu(budget_bytes=budget, slots=args.slots, prec="fp64", dedup=1))):
        try:
            out = make().run(reqs)
            st = latency_stats(out)
            st["n"] = st.pop("requests")
            st["iterations_mean"] = statistics.mean(r.iterations for r in out)
            st["max_relres"] = max(r.relres for r in out)
            st["setup_s_mean"] = statistics.mean(r.setup_s for r in out)
            st["solve_s_mean"] = statistics.mean(r.solve_s for r in out)
            if hasattr(out[0], "round_size"):
                st["rounds"] = len({r.round_id for r in out})
                st["round_size_mean"] = statistics.mean(r.round_size for r in out)
            arms[name] = st
        except Exception as e:
            arms[name] = {"error": str(e)[:200]}
    cl = clocks.stop()

    def ratio(a, b):
        try:
            return arms[a]["solves_per_s"] / arms[b]["solves_per_s"]
        except Exception:
            return None

    head = arms.get("batched_fp32", {})
    emit({"mode": "serve", "metric": "GMG solves/s", "value": head.get("solves_per_s"), "unit": "solves/s",
          "higher_is_better": True, "data": "synthetic",
          "config": {"workload": f"{args.requests} requests, Poisson arrivals {args.rate}/s, porous3d "
                                 "n in {16,32,48,64,96}, 5-200 spheres, FGMRES rtol 1e-8",
                     "budget_gb": args.budget_gb, "slots": args.slots, "shared_class_blocks": True,
                     "tc": args.tc, "latency": "seconds from arrival to result; p99 of fewer than 100 "
                                               "requests is their maximum"},
          "arms": arms,
          "speedup_mixed_vs_plain_fp64_batched": ratio("batched_fp32", "batched_fp64"),
          "speedup_mixed_vs_plain_fp64_streams": ratio("streams_fp32", "streams_fp64"),
          "speedup_batched_vs_streams_fp32": ratio("batched_fp32", "streams_fp32"),
          "speedup_batched_vs_streams_fp64": ratio("batched_fp64", "streams_fp64"),
          "speedup_live_vs_rounds_fp32": ratio("live_fp32", "batched_fp32"),
          "clocks": cl})
    return 0


def run_mixed(args):
    """Mixed precision on the 128^3 porous medium with 300 spheres (the
    radius range scaled to a 30 % solid fraction), 5 levels, V(2,2): cached
    patch rows in float32 / bfloat16 applied on CUDA cores or, for the
    shared class blocks, on the tensor cores (TF32, two-term TF32, BF16),
    inside the FP64 FGMRES to 1e-8; the FP64 rows (the plain method) and the
    float-pair rows beside them.  Per variant: setup, the timed solves,
    iterations, the error of velocity and pressure against the FP64 GPU
    solution (whose oracle parity the tests establish), and the
    finest-level patch apply timed alone (CUDA events)."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    prob = inputs.porous_3d(0, n=args.mixed_n, nspheres=300, nlevels=args.mixed_levels)
    stream = torch.cuda.Stream()
    variants = [("fp64", "none", 1), ("df64", "none", 1), ("fp32", "none", 1), ("fp32", "tf32x3", 1),
                ("fp32", "tf32", 1), ("fp32", "bf16", 1), ("bf16", "none", 1), ("bf16", "bf16", 1)]
    res, x64 = {}, None
    nd = prob.dim + 1
    clocks = Clocks(0)
    clocks.start()
    for prec, tc, dd in variants:
        key = f"{prec}/{tc}"
        try:
            with torch.cuda.stream(stream):
                t0 = time.perf_counter()
                s = fc.Solver(prob, prec=prec, tc=tc, dedup=dd, stream=stream)
                torch.cuda.synchronize()
                setup_ms = 1e3 * (time.perf_counter() - t0)
                b = s.rhs()
                for _ in range(args.warmup):
                    s.solve(b, rtol=prob.rtol, maxit=300)
                step_ms, total_ms, its_l, rr_l = timed_solves(s, b, prob, args.steps, stream, torch)
                x, _, _ = s.solve(b, rtol=prob.rtol, maxit=300)
                xc = x.cpu()
                entry = {"setup_ms": setup_ms, "ms_per_solve": total_ms / args.steps,
                         "solves_per_s": args.steps / (total_ms * 1e-3), "iterations": its_l[0],
                         "relres": max(rr_l),
                         "updates_per_s": sum(updates_per_solve(prob, i) for i in its_l) / (total_ms * 1e-3),
                         "cache_bytes": s.info()["bytes"][1], "badcut_patches": s.info()["bytes"][7],
                         "dense_lu_patches": s.info()["bytes"][5]}
                if x64 is None:
                    x64 = xc
                else:
                    for name, comp in (("u", list(range(prob.dim))), ("p", [prob.dim])):
                        idx = torch.cat([torch.arange(c, xc.numel(), nd) for c in comp])
                        entry[f"rel_err_{name}_vs_fp64_gpu"] = ((xc[idx] - x64[idx]).norm() / x64[idx].norm()).item()
                # the finest-level patch apply alone
                if prec in ("fp32", "bf16"):
                    B = fc.Batch([s])
                    X = torch.zeros_like(b)
                    B.smooth_(X, b, nsweeps=2)
                    B.profile(True)
                    B.smooth_(X, b, nsweeps=10)
                    na, ma, ba = B.profile_read(0)
                    B.profile(False)
                    B.close()
                else:
                    X = torch.zeros_like(b)
                    s.smooth_(X, b, nsweeps=2)
                    s.profile(True)
                    s.smooth_(X, b, nsweeps=10)
                    na, ma, ba = s.profile_read(4)
                    s.profile(False)
                entry["finest_apply_ms"] = ma / max(na, 1)
                entry["finest_apply_gbs"] = ba / (ma / max(na, 1) * 1e-3) / 1e9 if ma > 0 else None
                s.close()
                del s
            torch.cuda.synchronize()
            res[key] = entry
        except Exception as e:
            res[key] = {"error": str(e)[:200]}
    cl = clocks.stop()
    hbm, peak_kind = peaks()
    for e in res.values():
        if e.get("finest_apply_gbs"):
            e["finest_apply_hbm_frac"] = e["finest_apply_gbs"] / hbm
    emit({"mode": "mixed", "metric": "GMG solves/s", "unit": "solves/s", "higher_is_better": True,
          "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
          "config": {"workload": f"porous3d {args.mixed_n}^3, 300 spheres r~0.720 U[0.04,0.12] (30% solid), "
                                 f"alpha 1e-8, octree depth 3, {args.mixed_levels} levels, V(2,2), FGMRES(30) "
                                 "rtol 1e-8 in FP64, shared class blocks (dedup 1)",
                     "ndof": prob.ndof(), "hbm_peak_gbs": hbm, "hbm_peak_source": peak_kind},
          "variants": res, "clocks": cl})
    return 0


# Table tab:grid (Sec. 4): DoFs and GMG iteration counts of the paper's
# adaptive channel grids Omega^1..Omega^7 (no count is printed for Omega^1)
PAPER_TABLE_GRID = [("Omega^1", 790275, None), ("Omega^2", 1583127, 14), ("Omega^3", 4477533, 14),
                    ("Omega^4", 15004455, 7), ("Omega^5", 53016765, 5), ("Omega^6", 188665497, 5),
                    ("Omega^7", 665367261, 5)]


def run_replay(args):
    """The paper's experiment setting (Sec. 4): standalone GMG, V(6,6)
    cycles with damping 0.8, stop at a 1e9 residual reduction, alpha 1e-10,
    eta 1e-3, on the channel stand-in (2.2 x 0.41 box, cylinder of diameter
    0.1 near the inflow) at the size of the paper's coarse grid Omega^1
    (1024 x 256 cells, 790,275 DoFs) and uniform refinements of it, FP64
    rows.  Cycle counts are printed beside Table tab:grid's counts of the
    paper's adaptive grids (context only: uniform grids and a seeded
    cylinder position, not the benchmark's)."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    rows = []
    amr = args.replay_amr
    for k in range(args.replay_sizes):
        if amr:
            # adaptive: the 1024 x 256 grid everywhere (uniform level 6 over the
            # 16 x 4 root) and k + 1 further levels at the cylinder
            nx, ny = 1024 << (k + 1), 256 << (k + 1)
            nlev = 8 + k
            p = dataclasses.replace(inputs.channel_replay_2d(0, nx=nx, ny=ny, nlevels=nlev), amr_uniform=6)
        else:
            nx, ny = 1024 << k, 256 << k
            nlev = 7 + k                     # coarsest grid 16 x 4 cells
            p = inputs.channel_replay_2d(0, nx=nx, ny=ny, nlevels=nlev)
        try:
            t0 = time.perf_counter()
            s = fc.Solver(p, prec="fp64", dedup=0 if amr else 1)
            torch.cuda.synchronize()
            setup_ms = 1e3 * (time.perf_counter() - t0)
            b = s.rhs()
            s.gmg_solve(b, reduction=1e-9, maxit=200)      # warm-up (graphs, caches)
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, its, red = s.gmg_solve(b, reduction=1e-9, maxit=200)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            apply = None
            if amr:
                ups = its * sum(s.ndof(lv) for lv in range(2, nlev + 1)) * (p.nu_pre + p.nu_post)
                dofs = s.ndof()
                # the finest-level apply alone: 10 sweeps under the per-launch profiler
                X = torch.zeros_like(b)
                s.smooth_(X, b, nsweeps=2)
                s.profile(True)
                s.smooth_(X, b, nsweeps=10)
                na, ma, ba = s.profile_read(4)
                s.profile(False)
                torch.cuda.synchronize()
                avg = ma / max(na, 1)
                flop = float(s.info()["bytes"][6])
                tf, _ = fp64_peak(torch)
                hbm, _ = peaks()
                apply = {"ms": avg, "flop_per_launch": flop, "bytes_per_launch": ba,
                         "frac_of_fp64_peak": flop / (avg * 1e-3) / 1e12 / tf if avg else None,
                         "hbm_frac": ba / (avg * 1e-3) / 1e9 / hbm if avg else None}
            else:
                ups, dofs = updates_per_solve(p, its), p.ndof()
            rows.append({"grid": f"{nx}x{ny}" + (" lattice, adaptive" if amr else ""), "levels": nlev,
                         "dofs": dofs, "cycles": its, "reduction": red,
                         "solve_ms": ms, "ms_per_cycle": ms / max(its, 1), "setup_ms": setup_ms,
                         "sweep_updates_per_s": ups / (ms * 1e-3)})
            if apply:
                rows[-1]["finest_apply"] = apply
            s.close()
        except Exception as e:
            rows.append({"grid": f"{nx}x{ny}", "error": str(e)[:200]})
        torch.cuda.synchronize()
    emit({"mode": "replay", "metric": "GMG cycles to a 1e9 reduction", "unit": "cycles", "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": "channel stand-in 2.2 x 0.41, cylinder diameter 0.1 at a seeded position near the "
                                 "inflow, parabolic inflow ubar 0.3, alpha 1e-10, eta 1e-3, quadtree depth 4, "
                                 "standalone V(6,6), damping 0.8, coarsest grid 16 x 4, FP64 rows" +
                                 ("; adaptive quadtree: 1024 x 256 everywhere, cut cells refined k + 1 further "
                                  "levels, 2:1 balanced, Algorithm 1 hierarchy" if amr else "; uniform grids"),
                     "paper_table_grid": [{"grid": g, "dofs": d, "gmg_iterations": it} for g, d, it in PAPER_TABLE_GRID],
                     "note": "the paper's counts are for its adaptive grids and benchmark geometry: context, "
                             "not a parity target"},
          "sizes": rows})
    return 0


def run_q2(args):
    """The Q2-Q1 (Taylor-Hood) variant with the lower-corner ownership rule.
    2D (--q2-dim 2): the 2D channel (unit square, one circle r = 0.2,
    parabolic inflow, alpha 1e-8, quadtree depth 4) on an n x n grid, levels
    down to 16 x 16 cells.  3D (--q2-dim 3): the porous medium of the default
    line (40 spheres, alpha 1e-8, octree depth 3) on an n^3 grid, levels down
    to 4^3 cells.  V(2,2), FP64 rows, FGMRES to 1e-8.  Reports solves/s and
    owned-DoF updates/s over the timed solves, and the finest-level patch
    apply timed alone with its algorithmic FLOP (slots x owned rows x 2 per
    patch, upper bound) and bytes."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    dim = args.q2_dim
    n = args.q2_n if dim == 2 else args.q2_n3
    if dim == 2:
        nlev = max(2, int(math.log2(n // 16)) + 1)
        prob = inputs.channel_2d(0, n=n, nlevels=nlev)
        workload = f"Q2-Q1 channel2d {n}^2, one circle r 0.2, alpha 1e-8, quadtree depth 4, {nlev} levels"
        nslot, nrow = 171, 9
    else:
        nlev = max(2, int(math.log2(n // 4)) + 1)
        prob = inputs.porous_3d(0, n=n, nspheres=40, nlevels=nlev)
        workload = f"Q2-Q1 porous3d {n}^3, 40 spheres, alpha 1e-8, octree depth 3, {nlev} levels"
        nslot, nrow = 2214, 25
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        s = fc.Solver(prob, element="q2", stream=stream)
        torch.cuda.synchronize()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        b = s.rhs()
        for _ in range(args.warmup):
            s.solve(b, rtol=1e-8)
        step_ms, total_ms, its_l, rr_l = timed_solves(s, b, prob, args.steps, stream, torch)
        X = torch.zeros_like(b)
        s.smooth_(X, b, nsweeps=2)
        s.profile(True)
        s.smooth_(X, b, nsweeps=10)
        na, ma, ba = s.profile_read(4)
        nr, mr, _ = s.profile_read(1)
        s.profile(False)
        ndof = s.ndof()
        s.close()

    def owned(m):                              # DoFs of a level with m cells per direction
        return (2 * m + 1) ** dim * dim + (m + 1) ** dim
    nv1 = (n + 1) ** dim
    upd = owned(n)                             # owned DoFs of the finest level (each written once per sweep)
    per_solve = sum(owned(n >> k) for k in range(nlev - 1)) * 4
    avg = ma / max(na, 1)
    flop = nv1 * nslot * nrow * 2.0
    tf, note = fp64_peak(torch)
    hbm, _ = peaks()
    emit({"mode": "q2", "metric": "smoother patch-DoF updates/s", "unit": "owned-DoF updates/s", "dtype": "f64",
          "data": "synthetic",
          "value": sum(its_l) * per_solve / (total_ms * 1e-3),
          "config": {"workload": workload + ", V(2,2), FGMRES(30) rtol 1e-8, FP64 rows", "dim": dim, "ndof": ndof,
                     "iterations": its_l[0], "relres": max(rr_l), "setup_ms": setup_ms,
                     "solves_per_s": args.steps / (total_ms * 1e-3), "ms_per_solve": total_ms / args.steps,
                     "finest_owned_dofs": upd},
          "finest_apply": {"ms": avg, "launches": na, "residual_ms": mr / max(nr, 1),
                           "flop_per_launch": flop, "tflops": flop / (avg * 1e-3) / 1e12 if avg else None,
                           "frac_of_fp64_peak": flop / (avg * 1e-3) / 1e12 / tf if avg else None,
                           "fp64_peak_tflops": tf, "fp64_peak_source": note,
                           "bytes_per_launch": ba, "hbm_frac": ba / (avg * 1e-3) / 1e9 / hbm if avg else None}})
    return 0


def run_amr(args):
    """Adaptive space-tree grids, FGMRES with the V(2,2) RA smoother on every
    level.  3D (--amr-dim 3): the duct on the unit cube with one sphere
    (r = 0.2, seeded centre, product-parabola inflow, alpha 1e-8, octree
    depth 3) on an --amr-n^3 lattice, root grid 8^3, every cell refined to
    the quarter lattice and the cut cells to the lattice; 2D (--amr-dim 2):
    the 2D channel with one circle on an --amr-n^2 lattice, root 16^2, every
    cell refined to the quarter lattice.  FP64 rows.  Reports solves/s, the
    finest-level patch apply timed alone (algorithmic FLOP: owned rows x
    patch DoFs x 2 summed over the patches) against the FP64 peak, and the
    residual time."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    dim, n = args.amr_dim, args.amr_n
    root = 8 if dim == 3 else 16
    nlev = int(round(math.log2(n // root))) + 1
    if dim == 3:
        prob = dataclasses.replace(inputs.channel_3d(0, n=n, nlevels=nlev), amr_uniform=nlev - 3)
        workload = (f"adaptive octree, duct on the unit cube with one sphere r 0.2, lattice {n}^3, root 8^3, "
                    f"uniform to {n // 4}^3, cut cells to {n}^3, 2:1 balanced, {nlev} levels (Algorithm 1), "
                    f"alpha 1e-8, octree depth 3")
    else:
        prob = dataclasses.replace(inputs.channel_2d(0, n=n, nlevels=nlev), amr_uniform=nlev - 3)
        workload = (f"adaptive quadtree, channel on the unit square with one circle r 0.2, lattice {n}^2, root "
                    f"16^2, uniform to {n // 4}^2, cut cells to {n}^2, 2:1 balanced, {nlev} levels (Algorithm 1), "
                    f"alpha 1e-8, quadtree depth 4")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        s = fc.Solver(prob, stream=stream, dedup=0)
        torch.cuda.synchronize()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        b = s.rhs()
        for _ in range(args.warmup):
            s.solve(b, rtol=1e-8)
        step_ms, total_ms, its_l, rr_l = timed_solves(s, b, prob, args.steps, stream, torch)
        X = torch.zeros_like(b)
        s.smooth_(X, b, nsweeps=2)
        s.profile(True)
        s.smooth_(X, b, nsweeps=10)
        na, ma, ba = s.profile_read(4)
        nr, mr, _ = s.profile_read(1)
        s.profile(False)
        ndof = [s.ndof(lv) for lv in range(1, nlev + 1)]
        flop = float(s.info()["bytes"][6])
        s.close()
    avg = ma / max(na, 1)
    per_solve = sum(ndof[1:]) * (prob.nu_pre + prob.nu_post)
    tf, note = fp64_peak(torch)
    hbm, _ = peaks()
    emit({"mode": "amr", "metric": "smoother patch-DoF updates/s", "unit": "owned-DoF updates/s", "dtype": "f64",
          "data": "synthetic",
          "value": sum(its_l) * per_solve / (total_ms * 1e-3),
          "config": {"workload": workload + ", V(2,2), FGMRES(30) rtol 1e-8, FP64 rows", "dim": dim,
                     "ndof_per_level": ndof, "iterations": its_l[0], "relres": max(rr_l), "setup_ms": setup_ms,
                     "solves_per_s": args.steps / (total_ms * 1e-3), "ms_per_solve": total_ms / args.steps},
          "finest_apply": {"ms": avg, "launches": na, "residual_ms": mr / max(nr, 1),
                           "flop_per_launch": flop, "tflops": flop / (avg * 1e-3) / 1e12 if avg else None,
                           "frac_of_fp64_peak": flop / (avg * 1e-3) / 1e12 / tf if avg else None,
                           "fp64_peak_tflops": tf, "fp64_peak_source": note,
                           "bytes_per_launch": ba, "hbm_frac": ba / (avg * 1e-3) / 1e9 / hbm if avg else None}})
    return 0


def run_batch(args):
    """Uneven batch: 256 independent 2D channel problems (grids 16..128^2,
    1-8 ellipses, alpha 1e-6..1e-10) solved together by fc_batch_solve
    (persistent launches over all problems, one CUDA graph per Arnoldi step,
    autotuned patch tile), reduced-precision rows inside the FP64 FGMRES to
    1e-8; against the plain FP64 GPU solver taking the same problems one at
    a time."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    probs = [inputs.batch_2d(s) for s in range(args.batch)]
    rtol, maxit = 1e-8, 400
    t0 = time.perf_counter()
    solvers = [fc.Solver(p, prec=args.batch_prec, dedup=1) for p in probs]
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    B = fc.Batch(solvers)
    create_ms = 1e3 * (time.perf_counter() - t0)
    stream = torch.cuda.current_stream()
    b = B.rhs()
    for _ in range(args.warmup):
        B.solve(b, rtol=rtol, maxit=maxit)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    l0 = fc.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    its_all, rr_all = [], []
    for k in range(args.steps):
        _, its, rr = B.solve(b, rtol=rtol, maxit=maxit)
        its_all.append(its)
        rr_all.append(max(rr))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    launches = fc.launch_count() - l0
    cl = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    updates = sum(updates_per_solve(p, i) for its in its_all for p, i in zip(probs, its))
    # the dominant kernel: the batched patch apply over every finest level
    X = torch.zeros_like(b)
    B.smooth_(X, b, nsweeps=3)
    B.profile(True)
    B.smooth_(X, b, nsweeps=20)
    na, ma, ba = B.profile_read(0)
    nr, mr, _ = B.profile_read(1)
    B.profile(False)
    hbm, peak_kind = peaks()
    achieved = ba / (ma / na * 1e-3) / 1e9
    # end to end from pinned host buffers
    bh = torch.empty(B.ndof, dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    xh = torch.zeros(B.ndof, dtype=torch.float64, pin_memory=True)
    B.solve_host(bh, xh, rtol=rtol, maxit=maxit)
    e2e_t, e2e_up = [], 0
    for _ in range(args.steps):
        xh.zero_()
        t1 = time.perf_counter()
        its_h, _ = B.solve_host(bh, xh, rtol=rtol, maxit=maxit)
        e2e_t.append(time.perf_counter() - t1)
        e2e_up += sum(updates_per_solve(p, i) for p, i in zip(probs, its_h))
    tile = B.tile()
    info = B.info()
    B.close()
    for s_ in solvers:
        s_.close()
    # the plain FP64 GPU solver, one problem at a time, same problems
    probs_plain = [] if args.no_plain else probs
    plain = [fc.Solver(p, prec="fp64", dedup=0) for p in probs_plain]
    rhs = [s_.rhs() for s_ in plain]
    for s_, r in zip(plain[:8], rhs[:8]):
        s_.solve(r, rtol=rtol, maxit=maxit)
    torch.cuda.synchronize()
    lat = []
    its_plain = []
    tp0 = time.perf_counter()
    for s_, r in zip(plain, rhs):
        t1 = time.perf_counter()
        _, i1, _ = s_.solve(r, rtol=rtol, maxit=maxit)
        lat.append(time.perf_counter() - t1)
        its_plain.append(i1)
    plain_s = max(time.perf_counter() - tp0, 1e-9)
    for s_ in plain:
        s_.close()
    lat = sorted(lat) or [float("nan")]
    its_plain = its_plain or [0]
    step_sorted = sorted(step_ms)
    solves_per_s = len(probs) * args.steps / (total_ms * 1e-3)
    out = {
        "mode": "batch", "metric": METRIC, "value": updates / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[args.batch_prec], "data": "synthetic",
        "config": {"workload": f"{len(probs)} independent 2D channel problems, grids drawn from "
                               "{16,32,64,128}^2, 1-8 seeded ellipses (semi-axes U[0.03,0.2]), alpha in "
                               "{1e-6,1e-8,1e-10}, levels down to 4^2 cells, V(2,2), FGMRES(30) rtol 1e-8 "
                               "per problem; a step solves all of them",
                   "problems": len(probs), "ndof_total": info["ndof"], "patches_finest": info["npatch_finest"],
                   "levels_max": info["levels_max"], "patch_rows": args.batch_prec,
                   "tile": {"lanes_per_patch": tile[0], "threads": tile[1], "ctas_per_sm": tile[2]},
                   "l2": "rows of all finest levels exceed L2 (about 1 GB in FP32)",
                   "iterations_min_max": [min(its_all[0]), max(its_all[0])], "relres_max": max(rr_all),
                   "setup_ms": setup_ms, "batch_create_ms": create_ms,
                   "solves_per_s": solves_per_s,
                   "latency_ms_p50": statistics.median(step_sorted),
                   "latency_ms_p99": step_sorted[min(len(step_sorted) - 1,
                                                     int(math.ceil(0.99 * len(step_sorted))) - 1)],
                   "plain_fp64_gpu": None if args.no_plain else {"solves_per_s": len(probs) / plain_s,
                                      "latency_ms_p50": 1e3 * statistics.median(lat),
                                      "latency_ms_p99": 1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                                      "iterations_min_max": [min(its_plain), max(its_plain)],
                                      "note": "same problems solved one after another, FP64 rows"},
                   "speedup_solves_per_s_vs_plain_fp64": None if args.no_plain else solves_per_s / (len(probs) / plain_s),
                   "smoother": {"apply_launches": na, "apply_ms": ma / na, "residual_ms": mr / max(nr, 1)}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "batched patch apply over all finest levels",
                     "launches": na, "avg_launch_ms": ma / na, "algorithmic_bytes_per_launch": ba,
                     "peak_source": peak_kind},
        "e2e": {"value": e2e_up / sum(e2e_t), "unit": UNIT, "h2d_bytes_per_step": 2 * B.ndof * 8,
                "d2h_bytes_per_step": B.ndof * 8},
        "gpu_launches": launches,
        "clocks": cl,
    }
    if not args.no_cpu_baseline:
        sample = [p for p in probs if p.n[0] <= 32][:4]
        tot_u, tot_t, cores = 0.0, 0.0, 1
        for p in sample:
            ups, times, cores, _ = oracle_solve_rate(p, budget_s=args.cpu_budget / max(len(sample), 1))
            tot_u += sum(ups)
            tot_t += sum(times)
        out["cpu_baseline"] = {"value": tot_u / tot_t, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"oracle FGMRES-GMG solves of {len(sample)} problems of the batch "
                                         "with grids <= 32^2, setup excluded"}
    emit(out)
    return 0


def run_batch_sweeps(args):
    """Finest-level smoother sweeps of the uneven 2D batch only (bounded
    profiler captures): --warmup + --steps batched sweeps, optionally with a
    fixed patch-apply tile (--tile lanes,threads,ctas_per_sm)."""
    import torch
    from paper_2403_11636_gb300 import build, fc, inputs
    build.build()
    if args.batch_workload == "porous3d":
        # one 3D porous problem of n^3 cells through the batched kernels
        probs = [inputs.porous_3d(0, n=args.n, nlevels=max(2, int(math.log2(args.n // 4)) + 1))]
    else:
        probs = [inputs.batch_2d(s) for s in range(args.batch)]
    solvers = [fc.Solver(p, prec=args.batch_prec, dedup=args.dedup, tc=args.tc) for p in probs]
    B = fc.Batch(solvers)
    if args.tile:
        B.set_tile(*[int(v) for v in args.tile.split(",")])
    b = B.rhs()
    X = torch.zeros_like(b)
    B.smooth_(X, b, nsweeps=args.warmup)
    B.profile(True)
    B.smooth_(X, b, nsweeps=args.steps)
    na, ma, ba = B.profile_read(0)
    nr, mr, _ = B.profile_read(1)
    hbm, _ = peaks()
    info = B.info()
    emit({"mode": "batch-sweep", "workload": args.batch_workload,
          "problems": len(probs), "patches_finest": info["npatch_finest"],
          "prec": args.batch_prec, "dedup": args.dedup, "tc": args.tc, "tile": B.tile(),
          "apply_ms": ma / max(na, 1), "apply_bytes": ba,
          "apply_gbs": ba / (ma / na * 1e-3) / 1e9 if na else None,
          "residual_ms": mr / max(nr, 1),
          "updates_per_s": info["npatch_finest"] * 3 / ((ma / max(na, 1) + mr / max(nr, 1)) * 1e-3)})
    B.close()
    return 0


def policy_sweeps(prob, stream, args):
    """One finest-level smoother sweep (residual + patch solve) per cache
    policy / precision, CUDA events on the solver stream."""
    import torch
    from paper_2403_11636_gb300 import fc, inputs
    res = {}
    combos = [("inverse", "fp64", 1), ("inverse", "df64", 1), ("inverse", "fp32", 1), ("inverse", "bf16", 1),
              ("inverse", "df64", 0), ("inverse", "fp64", 0), ("matrix", "fp64", 1), ("matrix", "fp64", 0),
              ("none", "fp64", 1)]
    x0 = torch.as_tensor(inputs.random_vector(prob, 3)).cuda()
    bb = torch.as_tensor(inputs.random_vector(prob, 4)).cuda()
    upd = free_dofs(prob, prob.nlevels)
    for cache, prec, dd in combos:
        try:
            t0 = time.perf_counter()
            s = fc.Solver(prob, cache=cache, prec=prec, stream=stream, dedup=dd)
            torch.cuda.synchronize()
            setup = time.perf_counter() - t0
            x = x0.clone()
            reps = 1 if cache == "none" else 5
            s.smooth_(x, bb, nsweeps=1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.profile(True)
            e0.record(stream)
            s.smooth_(x, bb, nsweeps=reps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            na, ma, ba = s.profile_read(0)
            s.profile(False)
            info = s.info()
            res[f"{cache}/{prec}/{'shared' if dd else 'per-patch'}"] = {"sweep_ms": ms, "updates_per_s": upd / (ms * 1e-3),
                                      "apply_ms": ma / max(na, 1),
                                      "apply_gbs": (ba / (ma / max(na, 1) * 1e-3) / 1e9) if ma > 0 and ba > 0 else None,
                                      "setup_ms": setup * 1e3,
                                      "cache_bytes": info["bytes"][1]}
            s.close()
            del s
        except Exception as e:  # a policy that does not fit reports why
            res[f"{cache}/{prec}/{'shared' if dd else 'per-patch'}"] = {"error": str(e)[:200]}
        torch.cuda.synchronize()
    return res


def load_traffic(prec):
    """DRAM bytes per finest-level launch of the patch apply, from the
    committed ncu summary of this precision (a line 'traffic_bytes_64: N')."""
    path = os.path.join(ROOT, "profiles", f"patch_apply_{prec}_porous48.md")
    # the summary is of the per-patch layout (one stored block per patch)
    try:
        for line in open(path):
            if line.strip().startswith("traffic_bytes_64:"):
                return float(line.split(":", 1)[1].strip().split()[0])
    except Exception:
        pass
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cache", default="inverse", choices=["inverse", "matrix", "none"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "df64", "fp32", "bf16"])
    ap.add_argument("--policies", type=int, default=1)
    ap.add_argument("--dedup", type=int, default=0,
                    help="1: patches with bit-identical blocks share one stored block (same results)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-sweep-n", type=int, default=16,
                    help="grid of the oracle per-sweep timing (16: the solve sample's finest level)")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="profiled solves after the timed ones (per-kernel CUDA events)")
    ap.add_argument("--mode", default="solve", choices=["solve", "sweep", "serve", "batch", "batch-sweep", "mixed", "replay", "q2", "amr"])
    ap.add_argument("--mixed-n", type=int, default=128, help="grid of --mode mixed")
    ap.add_argument("--q2-n", type=int, default=256, help="grid of --mode q2 in 2D")
    ap.add_argument("--replay-amr", action="store_true", help="--mode replay on adaptive quadtree grids")
    ap.add_argument("--q2-n3", type=int, default=16, help="grid of --mode q2 in 3D")
    ap.add_argument("--q2-dim", type=int, default=2, choices=[2, 3], help="dimension of --mode q2")
    ap.add_argument("--amr-dim", type=int, default=3, choices=[2, 3], help="dimension of --mode amr")
    ap.add_argument("--amr-n", type=int, default=64, help="lattice of --mode amr (cells per direction)")
    ap.add_argument("--replay-sizes", type=int, default=4,
                    help="--mode replay: 1024x256 and this many - 1 uniform refinements")
    ap.add_argument("--batch-workload", default="batch2d", choices=["batch2d", "porous3d"],
                    help="problems of --mode batch-sweep: the 2D batch, or one porous3d --n problem")
    ap.add_argument("--tc", default="none", choices=["none", "tf32", "tf32x3", "bf16"],
                    help="tensor-core apply of the class blocks (--mode batch-sweep)")
    ap.add_argument("--mixed-levels", type=int, default=5, help="levels of --mode mixed")
    ap.add_argument("--tile", default="", help="lanes,threads,ctas_per_sm of --mode batch-sweep")
    ap.add_argument("--batch", type=int, default=256, help="problems of --mode batch")
    ap.add_argument("--batch-prec", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--no-plain", action="store_true", help="--mode batch without the one-at-a-time FP64 runs")
    ap.add_argument("--requests", type=int, default=24, help="requests of --mode serve")
    ap.add_argument("--rate", type=float, default=50.0, help="arrivals per second of --mode serve")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--n", type=int, default=48, help="grid size of --mode sweep")
    ap.add_argument("--workload", default="porous3d", choices=["porous3d", "roofline2d"],
                    help="problem of --mode sweep")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "sweep":
        return run_sweeps(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "batch-sweep":
        return run_batch_sweeps(args)
    if args.mode == "mixed":
        return run_mixed(args)
    if args.mode == "replay":
        return run_replay(args)
    if args.mode == "q2":
        return run_q2(args)
    if args.mode == "amr":
        return run_amr(args)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
