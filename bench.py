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


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


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
    lat = binding.Lattice(w.shape, w.tau, storage="f32", stream=st)
    lat.set_propellers(w.props)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- warm-up
    lat.step(args.warmup, w.n_iter)
    barrier()

    # ---- timed region (device time, CUDA events on the library's stream);
    # the collide-stream kernel is bracketed by events inside the library
    lat.enable_timing(["collide_stream"])
    launches0 = lat.stats()["kernel_launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        e0.record(st)
        lat.step(args.steps, w.n_iter)
        e1.record(st)
        barrier()
    ms = e0.elapsed_time(e1)
    stage = lat.timing()
    s = lat.stats()
    launches = s["kernel_launches"] - launches0
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    lat.enable_timing(False)

    # ---- per-stage breakdown (separate pass, every stage bracketed)
    lat.enable_timing(True)
    nb_steps = max(2, args.steps // 2)
    lat.step(nb_steps, w.n_iter)
    breakdown = {k: v[0] / nb_steps for k, v in lat.timing().items()}
    lat.enable_timing(False)

    # ---- end to end through the C ABI with host buffers: per step the point
    # set is uploaded from pinned memory and du + the FP64 sums read back
    npnt = w.props.n_points
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).pin_memory().numpy()
    X = pin(w.props.xrest, np.float64)
    A = pin(w.props.area, np.float32)
    B = pin(w.props.body, np.int32)
    du_host = torch.empty((npnt, 3), dtype=torch.float32).pin_memory().numpy()
    L = binding.load()
    e2e_steps = max(3, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        binding._check(L.ibm_set_points(lat.h, npnt, binding._ptr(X), None, binding._ptr(A),
                                        binding._ptr(B)), lat.h)
        lat.step(1, w.n_iter)
        binding._check(L.ibm_read_points(lat.h, None, None, binding._ptr(du_host)), lat.h)
        lat.stats()
    barrier()
    e2e_s = time.perf_counter() - t0
    h2d = npnt * (24 + 4 + 4 + 12)
    d2h = npnt * 12 + 32

    value = ws * w.cells * args.steps / (ms / 1e3) / 1e6
    e2e = ws * w.cells * e2e_steps / e2e_s / 1e6

    # ---- roofline of the dominant kernel (collide-stream, HBM-bound)
    coll_ms, coll_n = stage["collide_stream"]
    per_launch_s = coll_ms / 1e3 / max(1, coll_n)
    active = s["active_bricks"]
    alg_bytes = w.cells * 19 * 4 * 2 + active * 64 * 12
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = _captured_traffic("collide_stream_traffic.json")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, "f32"),
        "point_updates_per_s": ws * npnt * w.n_iter * args.steps / (ms / 1e3),
        "gpu_launches": launches,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "collide_stream",
                     "peak_source": "measured" if peaks else "fallback",
                     "alg_bytes_per_launch": alg_bytes,
                     "launch_ms": per_launch_s * 1e3},
        "stage_ms_per_step": {k: round(v, 5) for k, v in breakdown.items()},
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        wcpu = W.dense_array_256()
        dt, cores = cpu_oracle_run(wcpu, 2)
        line["cpu_baseline"] = {"value": wcpu.cells * 2 / dt / 1e6, "unit": UNIT,
                                "cores": cores, "kind": "oracle",
                                "sample": "2 full steps of the workload from rest, FP64"}
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
