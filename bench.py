#!/usr/bin/env python3
"""Benchmark of the SPH interaction sweep on one or more GB300 GPUs.

Workload (default): the 3D tank of 1 x 1 x 2 with fluid to z = 1 at dx = 0.01
(938,336 fluid particles) and 64 rigid spheres (61,664 rigid particles, radii uniform in
[0.04, 0.08], density ratios in [1.5, 3]) plus 280,908 wall particles; seeded synthetic
data.  One step = one full time step of the method (dt, kick/drift, rebin, density,
extrapolation, force/heat/contact sweep, body reduction and integration, final kick).

value  = ordered pair interactions evaluated by the force/heat sweep per second of the
         whole step (FP32 pair sums, FP64 bodies), summed over ranks / max time.
Every rank runs its own replica of the scene (weak scaling, no collective on the data
path).  ``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH pair-interactions/s & steps/s at 1M particles; p50/p99 job latency vs plain"
FLOP_PER_PAIR = 62      # FP32 pair arithmetic of the force/heat sweep, FMA = 2 (see the design notes)
BYTES_PER_TARGET = 72   # algorithmic HBM bytes per target particle of the force sweep (FP32)
FP32_LANES_PER_SM = 128
N_SM = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--key-order", type=int, default=0)
    ap.add_argument("--dx", type=float, default=0.01)
    ap.add_argument("--skin", type=float, default=0.3, help="Verlet skin in units of h")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(dx):
    from paper_2103_07925_gb300 import scenes
    if abs(dx - 0.01) < 1e-12:
        return scenes.tank3d_spheres()
    return scenes.tank3d_spheres(dx=dx)


def run_reference(args):
    """The FP64 CPU oracle on the host cores (rank 0 only), bounded samples per step."""
    from oracle.oracle import OracleScene
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # bounded sample: the full scene when the run is short, else a coarser copy of it
    total = args.steps + args.warmup
    dx = 0.01 if total <= 12 else (0.02 if total <= 200 else 0.03)
    sc = workload(dx)
    o = OracleScene(sc)
    o.step(args.warmup)
    p0 = o.diagnostics()[15]
    t0 = time.perf_counter()
    pairs = 0.0
    for _ in range(args.steps):
        o.step(1)
        pairs += o.diagnostics()[15]
    t = time.perf_counter() - t0
    val = pairs / t
    cores = os.cpu_count()
    n = len(sc["particles"]["mass"])
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pair-interactions/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "tank3d_64spheres", "dx": dx, "particles": n, "l2": "inputs larger than L2"},
           "cpu_baseline": {"value": val, "unit": "pair-interactions/s", "cores": cores, "kind": "oracle",
                            "sample": "%d oracle steps of the tank scene at dx=%g (%d particles)" % (args.steps, dx, n)},
           "e2e": {"value": val, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "first_step_pairs": p0}
    print(json.dumps(out))


def cpu_baseline():
    """Oracle timed on the host cores on a bounded sample (full scene, 2 steps)."""
    from oracle.oracle import OracleScene
    sc = workload(0.01)
    o = OracleScene(sc)
    t0 = time.perf_counter()
    pairs = 0.0
    for _ in range(2):
        o.step(1)
        pairs += o.diagnostics()[15]
    t = time.perf_counter() - t0
    return {"value": pairs / t, "unit": "pair-interactions/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "2 FP64 oracle steps of the full 1,280,908-particle tank scene (%.1f s)" % t}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def allmax(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def allsum(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    from paper_2103_07925_gb300.sph import Scene
    hbm, smmax, peak_src = peaks()
    sc = workload(args.dx)
    stream = torch.cuda.Stream()
    skin = args.skin * sc["params"]["h"]
    g = Scene(sc, precision=args.precision, stream=stream.cuda_stream, key_order=args.key_order, skin=skin)
    info = g.info()
    g.step(args.warmup)
    clocks = Clocks(local)
    p_before = g.info()["pairs_total"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        g.step(args.steps, sync=False)
        e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    p_after = g.info()["pairs_total"]
    pairs = p_after - p_before
    ms_max = allmax(ms)
    pairs_all = allsum(pairs)
    value = pairs_all / (ms_max / 1e3)
    steps_per_s = args.steps / (ms_max / 1e3)
    # per-kernel device times over the same number of steps, kernels launched one by one
    prof = g.profile(min(args.steps, 50))
    force_ms = prof["force"]
    pairs_per_step = pairs / args.steps
    achieved_tf = pairs_per_step * FLOP_PER_PAIR / (force_ms * 1e-3) / 1e12
    clock_mhz = smmax
    peak_tf = N_SM * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    n_targets = info["n_fluid"] + info["n_rigid"]
    hbm_ach = n_targets * BYTES_PER_TARGET / (force_ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": "pair-interactions/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
           "config": {"workload": "tank3d_64spheres (1x1x2 tank, fluid to z=1, dx=%g)" % args.dx,
                      "particles": info["n"], "fluid": info["n_fluid"], "rigid": info["n_rigid"],
                      "wall": info["n_wall"], "bodies": info["n_bodies"], "cells": info["n_cells"],
                      "precision": "FP32 pair sums, FP64 bodies" if args.precision == 32 else "FP64",
                      "key_order": "morton" if args.key_order == 0 else "row-major",
                      "skin_h": args.skin,
                      "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (info["bytes"] / 1e6),
                      "parallelism": "replica per GPU" if world > 1 else "1 GPU"},
           "steps_per_s": steps_per_s * world,
           "pairs_per_step": pairs_per_step,
           "list_rebuilds": g.info()["rebuilds"],
           "gpu_launches": args.steps * g.info()["kernels_per_step"],
           "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                        "frac": achieved_tf / peak_tf, "traffic": None, "kernel": "k_force",
                        "peak_source": "FP32 FMA lanes x SMs x 2 x max SM clock (%s clocks)" % peak_src,
                        "hbm": {"achieved_gbs": hbm_ach, "peak_gbs": hbm, "frac": hbm_ach / hbm,
                                "peak_source": peak_src}},
           "profile_ms": prof, "clocks": clk}
    # plain FP64 path on the same workload
    if not args.no_fp64 and args.precision == 32:
        s64 = torch.cuda.Stream()
        g64 = Scene(sc, precision=64, stream=s64.cuda_stream, key_order=args.key_order, skin=skin)
        g64.step(2)
        k64 = max(5, min(args.steps // 10, 30))
        q0 = g64.info()["pairs_total"]
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record(s64)
        g64.step(k64, sync=False)
        f1.record(s64)
        torch.cuda.synchronize()
        m64 = f0.elapsed_time(f1)
        q1 = g64.info()["pairs_total"]
        out["fp64"] = {"value": (q1 - q0) / (m64 / 1e3), "ms_per_step": m64 / k64, "steps": k64,
                       "steps_per_s": k64 / (m64 / 1e3)}
        g64.close()
    # end to end through the C ABI with host buffers: upload, step, read back
    if not args.no_e2e:
        n = info["n"]
        pos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        vel = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        tmp = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        outp = {"pos": torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy(),
                "vel": torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()}
        cur = g.read("pos", "vel", "temp")
        pos[:] = cur["pos"]
        vel[:] = cur["vel"]
        tmp[:] = cur["temp"]
        ke = max(3, min(args.steps // 10, 20))
        q0 = g.info()["pairs_total"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            g.write(pos=pos, vel=vel, temp=tmp)
            g.step(1)
            g.read("pos", "vel", out=outp)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        q1 = g.info()["pairs_total"]
        te = allmax(te)
        out["e2e"] = {"value": allsum(q1 - q0) / te, "unit": "pair-interactions/s",
                      "h2d_bytes_per_step": int(pos.nbytes + vel.nbytes + tmp.nbytes),
                      "d2h_bytes_per_step": int(outp["pos"].nbytes + outp["vel"].nbytes), "steps": ke,
                      "ms_per_step": 1e3 * te / ke}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    g.close()
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
