"""Benchmark of the coupled D3Q19 BGK + multi-direct-forcing IBM step.

Workload: the 256^3 periodic box (tau 0.6) with a 4x4x4 array of 64 rotating
four-blade propellers (blades 24 x 6 at 0.7 spacing: 89,600 Lagrangian
points), 5 fixed-point iterations per step, FP32 storage.  One step = one pass
of the whole path (kinematics, binning, moments, 5 x (interpolation,
spreading), fused collide-stream, FP64 sums).  Metric: million lattice-cell
updates per second (MLUPS) of the whole step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank advances its own replica of the workload
(replicas only: the path is not sharded), value = all ranks' cell updates /
the slowest rank's time.  --impl reference times the FP64 CPU oracle (the
only reference there is) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LBM-IBM MLUPS"
UNIT = "MLUPS"
WINDOWS = 5  # timed windows of --steps steps; the reported value is their median


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler (every 5 ms) around the timed region; only samples
    that arrive between mark_start() and mark_end() count."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, interval_ms=5):
        self.dev = device_index
        self.interval = interval_ms
        self.p = None
        self.lines = []
        self.t_start = self.t_end = None

    def __enter__(self):
        """Starts the sampler and waits for its first sample, so that the
        tool's start-up (which can hold the driver for seconds on a fresh
        machine) falls before the timed region rather than inside it."""
        import threading
        first = threading.Event()
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", str(self.interval)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except Exception:
            self.p = None
            return self

        def reader():
            for l in self.p.stdout:
                if l.strip():
                    self.lines.append((time.perf_counter(), l))
                    first.set()
            first.set()

        self.t = threading.Thread(target=reader, daemon=True)
        self.t.start()
        first.wait(timeout=30)
        return self

    def mark_start(self):
        self.t_start = time.perf_counter()

    def mark_end(self):
        self.t_end = time.perf_counter()

    def __exit__(self, *a):
        if self.p is not None:
            # let the samples taken during the region reach the reader
            time.sleep(3 * self.interval / 1e3)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.t.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = self.t_start if self.t_start is not None else -1e30
        t1 = self.t_end if self.t_end is not None else 1e30
        for ts, l in self.lines:
            if not (t0 <= ts <= t1):
                continue
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"],
                    "interval_ms": self.interval}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.interval,
                "region_s": (t1 - t0) if self.t_end is not None else None}


def _captured_traffic(name):
    """DRAM bytes per launch from a committed ncu capture, or None when the
    kernel's sources changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", name)))
        for path, digest in rec["sources_sha256"].items():
            if hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest() != digest:
                return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


def combine_ranks(ms, cells, steps, ws, device="cpu"):
    """Replicas only: every rank advances its own copy of the workload.  The
    job's time is the slowest rank's; the value counts every rank's cells."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * cells * steps / (ms / 1e3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_run(w, steps, warmup=0):
    """Times the FP64 oracle on the full workload (host cores, OpenMP)."""
    import oracle
    sim = oracle.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=w.n_iter)
    if warmup:
        sim.step(warmup)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dt, cores


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1904_02108_gb300 import workload as W
    w = W.dense_array_256()
    dt, cores = cpu_oracle_run(w, args.steps, args.warmup)
    value = w.cells * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(w, "f32"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d full steps of the workload after %d warm-up steps"
                                   % (args.steps, args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(w, storage):
    return {"workload": w.name, "cells": w.cells, "shape": list(w.shape),
            "points": w.props.n_points, "bodies": w.props.n_bodies, "ibm_iters": w.n_iter,
            "tau": w.tau, "storage": storage, "delta": "cosine",
            "l2": "inputs larger than L2 (2 x %.2f GB of populations per step)"
                  % (19 * 4 * w.cells / 1e9)}


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1904_02108_gb300 import binding, workload as W
    try:
        binding.load()
    except RuntimeError:
        import __graft_entry__
        __graft_entry__.build()
        binding.load()

    w = W.dense_array_256()
    st = torch.cuda.current_stream()
    lat = binding.Lattice(w.shape, w.tau, storage=args.storage, stream=st)
    lat.set_propellers(w.props)
    if args.overlap:
        lat.set_overlap(True)
    # launch shapes from the project's autotuner (results do not depend on
    # them; the lattice is left where it was)
    shape = lat.autotune(w.n_iter, 6) if not args.no_autotune else lat.launch_shape()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- warm-up
    lat.step(args.warmup, w.n_iter)
    barrier()

    # ---- timed region (device time, CUDA events on the library's stream).
    # WINDOWS windows of exactly K steps each, every one bracketed by a
    # barrier and a synchronisation; the line reports the median window.
    # Then, inside the same clock-sampled region, one more window of K steps
    # with the collide-stream kernel bracketed by events inside the library,
    # for its launch time (an event recorded between two kernels ends their
    # programmatic dependent launch: ~10 us per step, so the value comes from
    # the windows without them).
    launches0 = lat.stats()["kernel_launches"]
    evs_t = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(WINDOWS + 1)]
    barrier()
    with Clocks(local) as clk:
        clk.mark_start()
        for i, (e0, e1) in enumerate(evs_t):
            if i == WINDOWS:
                lat.enable_timing(["collide_stream"])
            barrier()
            e0.record(st)
            lat.step(args.steps, w.n_iter)
            e1.record(st)
            barrier()
        clk.mark_end()
    window_ms = [e0.elapsed_time(e1) for e0, e1 in evs_t[:WINDOWS]]
    instrumented_ms = evs_t[WINDOWS][0].elapsed_time(evs_t[WINDOWS][1])
    ms = statistics.median(window_ms)
    stage = lat.timing()
    s = lat.stats()
    launches = (s["kernel_launches"] - launches0) // (WINDOWS + 1)
    ms, value = combine_ranks(ms, w.cells, args.steps, ws, device="cuda")
    lat.enable_timing(False)

    # ---- per-stage breakdown (separate pass, every stage bracketed)
    lat.enable_timing(True)
    nb_steps = max(2, args.steps // 2)
    lat.step(nb_steps, w.n_iter)
    breakdown = {k: v[0] / nb_steps for k, v in lat.timing().items()}
    lat.enable_timing(False)

    # ---- the same steps replayed from captured CUDA graphs (two steps each)
    lat.set_graph(True)
    lat.step(2, w.n_iter)  # capture
    barrier()
    graph_ms = _device_ms(lambda: lat.step(args.steps, w.n_iter), st) / args.steps
    lat.set_graph(False)

    # ---- end to end through the C ABI with host buffers: per step the point
    # positions are uploaded from pinned memory (ibm_update_points), the step
    # runs, and du and the FP64 sums are read back into pinned memory
    # (ibm_read_points_async, lbm_read_sums_async), with mapped host
    # transfers (lbm_set_host_io: the kinematics read the positions from the
    # pinned buffer, small kernels write the read-outs into theirs, so no copy
    # operation sits between the steps' kernels; also timed with the default
    # copies); the host waits for step s-1's results (an event) while step s
    # runs, and checks them (double-buffered: every step's results reach the
    # host)
    npnt = w.props.n_points
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).pin_memory().numpy()
    X = pin(w.props.xrest, np.float64)
    du_host = [torch.empty((npnt, 3), dtype=torch.float32).pin_memory().numpy()
               for _ in range(2)]
    sums_host = [torch.zeros(4, dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    L = binding.load()
    # a steady-state window: the first step's enqueue and the last step's
    # read-out are not hidden behind other steps, so the window is several
    # times the timed region's step count
    e2e_steps = max(10, 2 * args.steps)

    def consume(b):
        evs[b].synchronize()
        return int(not (np.isfinite(sums_host[b]).all() and np.isfinite(du_host[b][0]).all()))

    def e2e_loop(host_io):
        lat.set_host_io(host_io)
        bad = 0
        barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            b = k % 2
            binding._check(L.ibm_update_points(lat.h, npnt, binding._ptr(X), None), lat.h)
            lat.step(1, w.n_iter)
            lat.points_async(du=du_host[b])
            lat.sums_async(sums_host[b])
            evs[b].record(st)
            if k > 0:
                bad += consume(1 - b)
        bad += consume((e2e_steps - 1) % 2)
        barrier()
        dt = time.perf_counter() - t0
        lat.set_host_io("copy")
        assert bad == 0, "non-finite results in the end-to-end loop"
        return dt

    e2e_copy_s = e2e_loop("copy")
    e2e_s = e2e_loop("mapped")
    h2d = npnt * 24
    d2h = npnt * 12 + 32

    _, e2e = combine_ranks(e2e_s * 1e3, w.cells, e2e_steps, ws, device="cuda")
    _, e2e_copy = combine_ranks(e2e_copy_s * 1e3, w.cells, e2e_steps, ws, device="cuda")

    # ---- roofline of the dominant kernel (collide-stream, HBM-bound): 19
    # FP32 populations read and 19 written per cell, and the IBM force of the
    # active bricks' cells.  With --overlap it does only the cells outside
    # the active bricks (the others follow in a kernel of their own).
    coll_ms, coll_n = stage["collide_stream"]
    per_launch_s = coll_ms / 1e3 / max(1, coll_n)
    active = s["active_bricks"]
    pop_bytes = 4 if args.storage == "f32" else 2
    if args.overlap:
        alg_bytes = (w.cells - 64 * active) * 19 * pop_bytes * 2
    else:
        alg_bytes = w.cells * 19 * pop_bytes * 2 + active * 64 * 12
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = _captured_traffic("collide_stream_traffic.json") if args.storage == "f32" else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, args.storage),
        "windows": {"n": WINDOWS, "steps_each": args.steps,
                    "ms_per_step": [round(t / args.steps, 5) for t in window_ms],
                    "value": "median window",
                    "collide_timed_window_ms_per_step": round(instrumented_ms / args.steps, 5)},
        "point_updates_per_s": ws * npnt * w.n_iter * args.steps / (ms / 1e3),
        "gpu_launches": launches,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "transfers": "mapped pinned host memory (lbm_set_host_io)",
                "value_with_copies": e2e_copy},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "collide_stream",
                     "peak_source": "measured" if peaks else "fallback",
                     "alg_bytes_per_launch": alg_bytes,
                     "launch_ms": per_launch_s * 1e3},
        # device time of each stage (with --overlap each on its own stream,
        # the collide concurrent with the IBM stages)
        "stage_ms_per_step": {k: round(v, 5) for k, v in breakdown.items()},
        "overlap": bool(args.overlap),
        "launch_shape": shape,
        "graph_ms_per_step": graph_ms,
        "clocks": clk.summary(),
    }
    lat.close()
    if not args.no_extras and ws == 1:
        line["batched"] = bench_batched()
        line["precision"] = bench_precision()
        line["tolerance"] = bench_tolerance()
        line["paper_sweep"] = bench_paper_sweep()
        line["delta_kernels"] = bench_delta_kernels()
        line["point_order"] = bench_point_order()
        line["mlp"] = bench_mlp()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        wcpu = W.dense_array_256()
        dt, cores = cpu_oracle_run(wcpu, 2)
        line["cpu_baseline"] = {"value": wcpu.cells * 2 / dt / 1e6, "unit": UNIT,
                                "cores": cores, "kind": "oracle",
                                "sample": "2 full steps of the workload from rest, FP64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


WEIGHTS = os.path.join(ROOT, "paper_1904_02108_gb300", "data", "warm_start_256.npy")


def _device_ms(fn, st):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def bench_batched(steps=100, warmup=4):
    """48 uneven periodic cubes (side U{48,64,80,96}) with 1-8 propellers
    each, one launch per stage for all of them, replayed as a CUDA graph."""
    import torch
    from paper_1904_02108_gb300 import binding, workload as W
    doms, dropped = W.batched_domains()
    st = torch.cuda.current_stream()
    lats = []
    for w in doms:
        lat = binding.Lattice(w.shape, w.tau, stream=st)
        lat.set_propellers(w.props)
        lats.append(lat)
    batch = binding.Batch(lats)
    shape = batch.autotune(5, 2)
    batch.set_graph(True)
    batch.step(warmup, 5)
    l0 = lats[0].stats()["kernel_launches"]
    ms = _device_ms(lambda: batch.step(steps, 5), st)
    launches = lats[0].stats()["kernel_launches"] - l0
    cells = sum(w.cells for w in doms)
    out = {"workload": "batched_domains_48", "value": cells * steps / (ms / 1e3) / 1e6,
           "unit": "MLUPS", "domains": len(doms), "cells": cells,
           "points": sum(w.props.n_points for w in doms), "propellers_dropped": dropped,
           "steps": steps, "ms_per_step": ms / steps, "graph": True, "launch_shape": shape,
           "launches_per_step": launches / steps}
    batch.close()
    for lat in lats:
        lat.close()
    out["tolerance"] = bench_batched_tolerance(doms, shape)
    return out


def bench_batched_tolerance(doms, shape, steps=5, warmup=3, tol=1e-4, max_iter=2000):
    """The same 48 domains with every domain iterating the paper's loop to
    its own eps <= tol from the previous step's force (one batch launch per
    stage and iteration, the host reading all domains' stop flags between
    chunks): ms per step and the iterations the domains took."""
    import numpy as np
    import torch
    from paper_1904_02108_gb300 import binding
    st = torch.cuda.current_stream()
    lats = []
    for w in doms:
        lat = binding.Lattice(w.shape, w.tau, warm="previous", ibm_tol=tol, ibm_max_iter=max_iter,
                              stream=st)
        lat.set_propellers(w.props)
        lats.append(lat)
    batch = binding.Batch(lats)
    batch.set_launch_shape(**shape)
    batch.step(warmup, 0)
    t_ms, its, capped = 0.0, [], 0
    for _ in range(steps):
        t_ms += _device_ms(lambda: batch.step(1, 0), st)
        it = [lat.stats()["last_ibm_iters"] for lat in lats]
        its.append(it)
        capped += sum(int(lat.stats()["last_residual"] > tol) for lat in lats)
    its = np.array(its)
    out = {"tol": tol, "solver": "mdf", "start": "previous", "steps": steps,
           "ms_per_step": t_ms / steps, "iters_mean": float(its.mean()),
           "iters_max_per_step": float(its.max(axis=1).mean()), "capped_domain_steps": capped}
    batch.close()
    for lat in lats:
        lat.close()
    return out


def bench_tolerance(steps=8, warmup=3, tol=1e-4, max_iter=1000):
    """ms per step when every step iterates the fixed point to eps <= tol,
    on the 256^3 propeller array: zero start, previous-force start, the
    learned start, and the previous-force start on 16-bit storage, with the
    paper's loop ("mdf") and with conjugate gradients on the same fixed point
    ("cg")."""
    import numpy as np
    import torch
    from paper_1904_02108_gb300 import binding, workload as W
    w = W.dense_array_256()
    st = torch.cuda.current_stream()
    variants = [("zero_f32", "zero", "f32", "mdf"), ("previous_f32", "previous", "f32", "mdf")]
    P = None
    if os.path.exists(WEIGHTS):
        P = np.load(WEIGHTS)
        variants.append(("learned_f32", "mlp", "f32", "mdf"))
    variants += [("previous_bf16", "previous", "bf16", "mdf"),
                 ("previous_f16", "previous", "f16", "mdf"),
                 ("cg_zero_f32", "zero", "f32", "cg"), ("cg_previous_f32", "previous", "f32", "cg"),
                 ("cg_previous_bf16", "previous", "bf16", "cg"),
                 ("cg_previous_f16", "previous", "f16", "cg")]
    if P is not None:
        variants.append(("cg_learned_f32", "mlp", "f32", "cg"))
    out = {"tol": tol, "max_iter": max_iter, "workload": w.name, "steps": steps}
    for name, warm, storage, solver in variants:
        lat = binding.Lattice(w.shape, w.tau, storage=storage, warm=warm, ibm_tol=tol,
                              ibm_max_iter=max_iter, stream=st, solver=solver)
        lat.set_propellers(w.props)
        if warm == "mlp":
            lat.set_mlp_weights(P)
        lat.autotune(w.n_iter, 3)
        lat.step(warmup, 0)
        # steps one call each (iteration counts and residuals per step), then
        # as many steps in one call (each step's kinematics and pair lists
        # built while the step before it collides): the ms per step of a run
        iters, capped = 0, 0
        t_ms = 0.0
        for _ in range(steps):
            t_ms += _device_ms(lambda: lat.step(1, 0), st)
            s = lat.stats()
            iters += s["last_ibm_iters"]
            capped += int(s["last_residual"] > tol)
        call_ms = _device_ms(lambda: lat.step(steps, 0), st)
        out[name] = {"ms_per_step": call_ms / steps, "ms_per_step_one_call_each": t_ms / steps,
                     "iters_per_step": iters / steps, "capped_steps": capped, "solver": solver,
                     "iters_from": "the one-call-each steps"}
        if warm == "mlp":
            # device time of the learned start's kernels (features, MLP,
            # initial guess) per step, in a separate pass with that stage timed
            lat.enable_timing(["mlp"])
            lat.step(2, 0)
            mlp_ms, mlp_n = lat.timing()["mlp"]
            lat.enable_timing(False)
            out[name]["mlp_stage_ms_per_step"] = mlp_ms / 2
            out[name]["mlp_stage_launches_per_step"] = mlp_n / 2
        lat.close()
    return out


def bench_paper_sweep(steps=200, warmup=5):
    """The shape of the paper's own benchmark (Sec. 6, Figs. 5-6): MLUPS of
    the coupled step (5 iterations) on a 160 x 160 x 320 lattice with 1 to 6
    and 18 rotating propellers of 3872 points each (the paper's Blender
    propeller, not available, has 3930), FP32, for each way of pre-computing
    U0 before the fixed point: the active bricks (this library's default),
    the paper's box strategy and its kernel strategy (Sec. 5).  Beside the
    MLUPS, the device time per step of the stage that holds the U0
    pre-computation (with the first brick pass of the fixed point).  The
    paper's P100 figures quoted in its text are given for context."""
    import torch
    from paper_1904_02108_gb300 import binding, workload as W
    st = torch.cuda.current_stream()
    strategies = ("bricks", "box", "kernel")
    out = {"workload": "paper_sweep_160x160x320", "cells": 160 * 160 * 320, "n_iter": 5,
           "steps": steps, "points_per_propeller": W.paper_sweep(1).props.n_points,
           "paper_p100_mlups": {"1": 893.0, "6": 650.0, "18": 344.2},
           "mlups": {s: {} for s in strategies}, "u0_stage_ms": {s: {} for s in strategies}}
    for n in (1, 2, 3, 4, 5, 6, 18):
        w = W.paper_sweep(n)
        shape = None
        for strat in strategies:
            lat = binding.Lattice(w.shape, w.tau, stream=st)
            lat.set_u0_strategy(strat)
            lat.set_propellers(w.props)
            if shape is None:
                shape = lat.autotune(w.n_iter, 3)
            else:
                lat.set_launch_shape(**shape)
            lat.step(warmup, w.n_iter)
            ms = _device_ms(lambda: lat.step(steps, w.n_iter), st)
            out["mlups"][strat][str(n)] = w.cells * steps / (ms / 1e3) / 1e6
            lat.enable_timing(["brick_init"])
            lat.step(20, w.n_iter)
            out["u0_stage_ms"][strat][str(n)] = lat.timing()["brick_init"][0] / 20
            lat.enable_timing(False)
            lat.close()
    return out


def bench_delta_kernels(steps=100, warmup=5, tol_steps=6, tol=1e-4):
    """The paper's two weighting functions on the 256^3 array: the cosine
    kernel (the default) and Peskin's four-point kernel (Sec. 3).  Per kernel:
    MLUPS at 5 iterations, and the iterations and ms per step to the residual
    eps <= tol (conjugate gradients from the previous step's force)."""
    import torch
    from paper_1904_02108_gb300 import binding, workload as W
    w = W.dense_array_256()
    st = torch.cuda.current_stream()
    out = {"workload": w.name, "steps": steps, "tol": tol, "tol_steps": tol_steps}
    for delta in ("cosine", "peskin"):
        lat = binding.Lattice(w.shape, w.tau, delta=delta, stream=st)
        lat.set_propellers(w.props)
        lat.autotune(w.n_iter, 3)
        lat.step(warmup, w.n_iter)
        ms = _device_ms(lambda: lat.step(steps, w.n_iter), st)
        lat.close()
        lat = binding.Lattice(w.shape, w.tau, delta=delta, warm="previous", ibm_tol=tol,
                              ibm_max_iter=1000, stream=st, solver="cg")
        lat.set_propellers(w.props)
        lat.step(3, 0)
        t_ms, iters = 0.0, 0
        for _ in range(tol_steps):
            t_ms += _device_ms(lambda: lat.step(1, 0), st)
            iters += lat.stats()["last_ibm_iters"]
        lat.close()
        out[delta] = {"mlups": w.cells * steps / (ms / 1e3) / 1e6,
                      "tol_ms_per_step": t_ms / tol_steps, "tol_iters_per_step": iters / tol_steps}
    return out


def bench_point_order(steps=200, warmup=5):
    """Ablation of the points' order (the paper notes that per-point accesses
    to the neighbourhood are uncoalesced): the 256^3 array at 5 iterations
    with its points in the generated order (blade by blade, radius-major), in
    a seeded random permutation, and in Morton order of the 4^3 brick holding
    each rest position.  Results are the same up to the FP32 order of sums."""
    import numpy as np
    import torch
    from paper_1904_02108_gb300 import binding, workload as W
    w = W.dense_array_256()
    p = w.props
    st = torch.cuda.current_stream()
    b = np.floor(p.xrest / 4.0).astype(np.int64)

    def morton(v):
        out = np.zeros(len(v), np.int64)
        for bit in range(7):
            for c in range(3):
                out |= ((v[:, c] >> bit) & 1) << (3 * bit + c)
        return out

    orders = {"generated": np.arange(p.n_points),
              "random": np.random.default_rng(1241).permutation(p.n_points),
              "brick_morton": np.argsort(morton(b), kind="stable")}
    out = {"workload": w.name, "steps": steps, "mlups": {}}
    for name, perm in orders.items():
        q = W.Propellers(p.xrest[perm], p.area[perm], p.body[perm], p.centre, p.omega, p.phase,
                         p.blade_length, p.blade_width)
        lat = binding.Lattice(w.shape, w.tau, stream=st)
        lat.set_propellers(q)
        lat.autotune(w.n_iter, 3)
        lat.step(warmup, w.n_iter)
        ms = _device_ms(lambda: lat.step(steps, w.n_iter), st)
        out["mlups"][name] = w.cells * steps / (ms / 1e3) / 1e6
        lat.close()
    return out


def bench_mlp(reps=50):
    """The learned start's network on the tensor cores: one inference pass
    over the 89,600 points of the 256^3 array (mlp_forward_dev) and one
    loss-gradient pass over a training batch of 16,384 samples
    (mlp_loss_grad_dev), device time per call and the tensor FLOP rate
    (2 x (16 x 64 + 64 x 64 + 64 x 3) = 10,624 FLOP per sample forward; the
    backward adds the data gradient of layer 2 and the weight gradients of
    layers 1 and 2, 2 x (64 x 64 + 64 x 64 + 16 x 64) = 18,432)."""
    import numpy as np
    import torch
    from paper_1904_02108_gb300 import binding, learned, workload as W
    st = torch.cuda.current_stream()
    P = torch.tensor(learned.init_params(11), device="cuda")
    packed = torch.empty(binding.mlp_packed_bytes(), dtype=torch.uint8, device="cuda")
    binding.mlp_pack_dev(P, packed, st)
    n_inf, n_tr = 89600, 16384
    g = torch.Generator(device="cuda")
    g.manual_seed(12)
    X = torch.rand((n_inf, 16), device="cuda", generator=g) * 2 - 1
    Y = torch.empty((n_inf, 3), device="cuda")
    T = torch.rand((n_tr, 3), device="cuda", generator=g) - 0.5
    grad = torch.zeros_like(P)
    loss = torch.zeros(1, device="cuda")
    scratch = torch.empty(binding.mlp_grad_scratch_bytes(n_tr), dtype=torch.uint8, device="cuda")
    binding.mlp_forward_dev(X, packed, Y, st)
    binding.mlp_loss_grad_dev(X[:n_tr].contiguous(), T, P, packed, grad, loss, scratch, st)
    Xt = X[:n_tr].contiguous()
    f_ms = _device_ms(lambda: [binding.mlp_forward_dev(X, packed, Y, st) for _ in range(reps)],
                      st) / reps
    t_ms = _device_ms(lambda: [binding.mlp_loss_grad_dev(Xt, T, P, packed, grad, loss, scratch, st)
                               for _ in range(reps)], st) / reps
    fwd, bwd = 10624, 18432
    return {"inference": {"samples": n_inf, "ms": f_ms,
                          "tflops": n_inf * fwd / (f_ms / 1e3) / 1e12},
            "loss_grad": {"samples": n_tr, "ms": t_ms,
                          "tflops": n_tr * (fwd + bwd) / (t_ms / 1e3) / 1e12},
            "engine": "tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in tensor memory"}


def bench_precision(steps=100, warmup=5):
    """384^3 array of 216 propellers (5 iterations per step) with 16-bit
    deviation storage: MLUPS and the collide-stream kernel's HBM roofline."""
    import torch
    from paper_1904_02108_gb300 import binding, workload as W
    w = W.dense_array_384()
    st = torch.cuda.current_stream()
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    out = {"workload": w.name, "cells": w.cells, "points": w.props.n_points, "steps": steps}
    for storage in ("bf16", "f16"):
        lat = binding.Lattice(w.shape, w.tau, storage=storage, stream=st)
        lat.set_propellers(w.props)
        shape = lat.autotune(w.n_iter, 3)
        lat.step(warmup, w.n_iter)
        lat.enable_timing(["collide_stream"])
        ms = _device_ms(lambda: lat.step(steps, w.n_iter), st)
        cms, cn = lat.timing()["collide_stream"]
        s = lat.stats()
        alg = w.cells * 19 * 2 * 2 + s["active_bricks"] * 64 * 12
        ach = alg / (cms / 1e3 / cn) / 1e9
        out[storage] = {"value": w.cells * steps / (ms / 1e3) / 1e6, "unit": "MLUPS",
                        "ms_per_step": ms / steps, "launch_shape": shape,
                        "collide_roofline": {"achieved": ach, "peak": peak, "unit": "GB/s",
                                             "frac": ach / peak, "alg_bytes_per_launch": alg}}
        lat.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--overlap", action="store_true",
                    help="collide the cells outside the active bricks concurrently with the "
                         "IBM stages (off by default: slower on this workload)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="population storage of the timed workload (FP32 is the benchmark; "
                         "the 16-bit forms for profiling their collide kernels)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, 16-bit and tolerance-mode measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
