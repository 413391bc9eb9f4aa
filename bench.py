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
# density sweep: offset 6, squared distance 5, root 1, q 1, kernel polynomial 11,
# accumulation 1 FP32 operations per pair inside the support; 28 algorithmic bytes per
# fluid target (position, mass and material in, density out)
FLOP_PER_DENSITY_PAIR = 25
BYTES_PER_DENSITY_TARGET = 28
# DRAM bytes (read + write) of one launch on the default workload, from `ncu --set full`
# captures of this kernel version (a smaller tank, scaled by the targets), per kernel and
# cell layout (key order, skin in h) they were captured with; emptied whenever a kernel
# changes
TRAFFIC = {("k_force", 1, 0.5): 583.8e6, ("k_density", 1, 0.5): 1194.8e6,
           ("k_force", 1, 0.7): 582.3e6, ("k_density", 1, 0.7): 1301.8e6}
FP64_SKIN_H = 0.15  # Verlet skin of the FP64 leg, in h (see the FP64 leg in main())
FP32_LANES_PER_SM = 128  # nominal, for the context figure beside the measured peak


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
    ap.add_argument("--cells-per-group", type=int, default=0,
                    help="row-major keys: cells along x per search warp (0 automatic, -1 windows of 32 particles)")
    ap.add_argument("--dx", type=float, default=None, help="lattice spacing (default 0.01 tank, 0.005 powder)")
    ap.add_argument("--skin", type=float, default=0.3, help="Verlet skin in units of h")
    ap.add_argument("--workload", default="tank3d", choices=["tank3d", "powder", "batch", "serve"],
                    help="tank3d: the 1.28M-particle tank (default); powder: the 2.1M-particle powder "
                         "bed with melting grains; batch: 256 mixed scenes in one batch; serve: Poisson "
                         "job arrivals served by continuous batching")
    ap.add_argument("--p-background", type=float, default=0.0,
                    help="tank/powder: background pressure of the transport-velocity formulation, in "
                         "units of p0 = rho0 c^2 of the first fluid (the paper's examples use 1); 0: off")
    ap.add_argument("--preheat", default=None,
                    help="powder: 'A,wavelength': grains start at T_melt + A sin(2 pi x / wavelength) (gas at "
                         "T_melt), so metal melts and solidifies throughout the timed steps")
    ap.add_argument("--scenes", type=int, default=256, help="batch: number of scenes")
    ap.add_argument("--jobs", type=int, default=32, help="serve: number of jobs")
    ap.add_argument("--job-steps", type=int, default=1000, help="serve: steps per job")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (tank/powder: use --key-order and --skin; batch: default layout)")
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


DEFAULT_DX = {"tank3d": 0.01, "powder": 0.005}
WORKLOAD_NAME = {"tank3d": "tank3d_64spheres (1x1x2 tank, fluid to z=1, dx=%g)",
                 "powder": "powder_bed (1x0.5x0.5 box, gas, metal grains melting under a moving source, dx=%g)"}


def workload(dx, name="tank3d", preheat=None):
    from paper_2103_07925_gb300 import scenes
    if name == "powder":
        return scenes.powder_bed(dx=dx, preheat=preheat)
    if abs(dx - 0.01) < 1e-12:
        return scenes.tank3d_spheres()
    return scenes.tank3d_spheres(dx=dx)


REF_BUDGET_S = 150.0  # timed oracle steps of the reference arm stop within about this


def oracle_single_thread(dx, name, preheat=None):
    """Pair rate of the oracle on one host thread: one step of the same scene in a child
    process with OMP_NUM_THREADS=1 (the oracle's OpenMP loops then run serially)."""
    code = ("import sys, time, json; sys.path.insert(0, %r)\n"
            "import bench\n"
            "from oracle.oracle import OracleScene\n"
            "o = OracleScene(bench.workload(%r, %r, %r))\n"
            "t0 = time.perf_counter(); o.step(1); t = time.perf_counter() - t0\n"
            "print(json.dumps({'value': o.diagnostics()[15] / t, 'seconds': t}))\n") % (ROOT, dx, name, preheat)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": "pair-interactions/s", "cores": 1, "kind": "oracle",
            "sample": "1 FP64 oracle step of the same scene on one thread (%.1f s)" % d["seconds"]}


def run_reference(args):
    """The FP64 CPU oracle on the host cores (rank 0 only) on the same scene as our arm.
    It runs the requested warm-up and timed steps while they fit in about REF_BUDGET_S
    seconds (one oracle step of the 1.28M-particle tank takes about 1.5 s on 16 cores) and
    prints the numbers of steps it actually ran; the value is a rate.  A single-thread rate
    of the oracle is reported beside it."""
    from oracle.oracle import OracleScene
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload if args.workload in DEFAULT_DX else "tank3d"
    dx = args.dx or DEFAULT_DX[name]
    preheat = tuple(float(v) for v in args.preheat.split(",")) if args.preheat else None
    sc = workload(dx, name, preheat)
    o = OracleScene(sc)
    t0 = time.perf_counter()
    o.step(1)  # one untimed step sizes the sample
    t_one = time.perf_counter() - t0
    fit = max(1, int(REF_BUDGET_S / max(t_one, 1e-9)))
    k = max(1, min(args.steps, fit))
    w = max(0, min(args.warmup - 1, fit - k))
    o.step(w)
    w += 1
    t0 = time.perf_counter()
    pairs = 0.0
    for _ in range(k):
        o.step(1)
        pairs += o.diagnostics()[15]
    t = time.perf_counter() - t0
    val = pairs / t
    cores = os.cpu_count()
    n = len(sc["particles"]["mass"])
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pair-interactions/s",
           "n_gpus": args.gpus, "steps": k, "warmup": w,
           "ms_per_step": 1e3 * t / k, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME[name] % dx, "particles": n,
                      "l2": "inputs larger than L2",
                      "requested": {"steps": args.steps, "warmup": args.warmup}},
           "cpu_baseline": {"value": val, "unit": "pair-interactions/s", "cores": cores, "kind": "oracle",
                            "sample": "%d timed FP64 oracle steps (after %d warm-up) of the same %d-particle "
                                      "scene" % (k, w, n)},
           "cpu_baseline_1thread": oracle_single_thread(dx, name, preheat),
           "e2e": {"value": val, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cpu_baseline(sc):
    """Oracle timed on the host cores on a bounded sample (the same scene, 2 steps)."""
    from oracle.oracle import OracleScene
    o = OracleScene(sc)
    t0 = time.perf_counter()
    pairs = 0.0
    for _ in range(2):
        o.step(1)
        pairs += o.diagnostics()[15]
    t = time.perf_counter() - t0
    return {"value": pairs / t, "unit": "pair-interactions/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "2 FP64 oracle steps of the same %d-particle scene (%.1f s)" % (len(sc["particles"]["mass"]), t)}


def bench_batch(args, rank, world, allmax, allsum, barrier):
    """Many independent scenes of uneven size advanced together (one launch per stage over
    all scenes, one CUDA graph per step), against the plain per-scene FP64 path."""
    import numpy as np
    import torch
    from paper_2103_07925_gb300 import scenes as S
    from paper_2103_07925_gb300.sph import Batch, Scene
    from paper_2103_07925_gb300.tune import tune_batch
    mix = S.batch_mix(count=args.scenes, seed=2103 + rank)
    scs = [sc for sc, _ in mix]
    nparts = int(sum(m["n"] for _, m in mix))
    tuned = {}
    if not args.no_tune:
        tuned = tune_batch(None, scs, precision=32, steps=8, warmup=2)
    B = Batch(capacity=len(scs), precision=32)
    t0 = time.perf_counter()
    ids = []
    for sc in scs:
        ov = dict(tuned[sc["params"]["dim"]].params) if sc["params"]["dim"] in tuned else {}
        j = B.admit(sc, 0, **ov)
        if j is None:
            raise SystemExit("batch does not fit")
        ids.append(j)
    torch.cuda.synchronize()
    t_admit = time.perf_counter() - t0
    if tuned:  # layouts come from the tuner's cache; launch shapes are tuned on the batch itself
        tuned = tune_batch(B, scs, precision=32)
    B.step(args.warmup)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    q0 = B.info()["pairs_total"]
    ms = B.time_steps(args.steps)
    barrier()
    clk = clocks.stop()
    info = B.info()
    pairs = info["pairs_total"] - q0
    ms_max = allmax(ms)
    value = allsum(len(scs) * args.steps) / (ms_max / 1e3)
    # end to end: admission (host inputs to the device), the timed steps, read-back of positions
    t1 = time.perf_counter()
    outs = [B.read(j, "pos") for j in ids]
    t_read = time.perf_counter() - t1
    e2e_s = allmax(t_admit + ms / 1e3 + t_read)
    h2d = int(sum(sum(np.asarray(v).nbytes for v in sc["particles"].values()) for sc in scs))
    d2h = int(sum(o.nbytes for o in outs))
    B.close()
    # plain path: every scene alone, FP64 and FP32 (device time of a few steps each)
    plain = {}
    for prec in (64, 32):
        tot_ms = 0.0
        k = 2
        for sc in scs:
            g = Scene(sc, precision=prec)
            g.step(1)
            tot_ms += g.time_steps(k) / k
            g.close()
        plain[prec] = len(scs) / (allmax(tot_ms) / 1e3) * world
    # FP64 check of the batched FP32 form on 8 sampled scenes: one step in a batch of the
    # sample against each scene alone on the FP64 path
    from paper_2103_07925_gb300.errors import field_scales, rel_err
    pick = [int(q) for q in np.linspace(0, len(scs) - 1, 8)]
    Bc = Batch(capacity=8, precision=32)
    cids = [Bc.admit(scs[q], 1) for q in pick]
    Bc.step(1)
    Bc.poll()
    flds = ("pos", "vel", "rho", "pres", "temp")
    check = {f: 0.0 for f in flds}
    for q, cid in zip(pick, cids):
        r32 = Bc.read(cid, *flds)
        g64 = Scene(scs[q], precision=64)
        g64.step(1)
        r64 = g64.read(*flds)
        g64.close()
        sca = field_scales(scs[q])
        for f in flds:
            check[f] = max(check[f], rel_err(r32[f], r64[f], scale=sca.get(f, 0.0)))
    Bc.close()
    out = {"metric": "scene-steps/s, batched form (%d mixed 2D/3D scenes)" % len(scs), "value": value,
           "unit": "scene-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batched mix: %d scenes, log N ~ normal around sqrt(1e4 x 5e5), clipped to "
                                  "[1e4, 5e5], 2D/3D by a seeded coin, 0-50 bodies" % len(scs),
                      "particles": nparts, "scenes_2d": sum(m["dim"] == 2 for _, m in mix),
                      "bodies": int(sum(m["bodies"] for _, m in mix)),
                      "tuned": {d: dict(t.params, **t.launch) for d, t in tuned.items()},
                      "l2": "inputs larger than L2 (%.1f GB resident)" % (info["bytes"] / 1e9)},
           "pairs_per_s": allsum(pairs) / (ms_max / 1e3),
           "plain_fp64": {"value": plain[64], "unit": "scene-steps/s", "kind": "each scene alone, FP64"},
           "plain_fp32": {"value": plain[32], "unit": "scene-steps/s", "kind": "each scene alone, FP32"},
           "speedup_vs_plain_fp64": value / plain[64],
           "fp64_check": {"scenes": pick, "max_error_after_1_step": check, "tolerance": 1e-5},
           "gpu_launches": args.steps * info["kernels_per_step"],
           "e2e": {"value": allsum(len(scs) * args.steps) / e2e_s, "unit": "scene-steps/s",
                   "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
                   "note": "admission of all scenes + timed steps + read-back of positions"},
           "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def bench_serve(args, rank, world, allmax, allsum, barrier):
    """Poisson arrivals served by continuous batching, against one scene at a time."""
    from paper_2103_07925_gb300.serve import Server, percentiles, serve_plain, serving_jobs
    from paper_2103_07925_gb300.sph import Batch, Scene
    jobs = serving_jobs(args.jobs, rate=20.0, steps=args.job_steps, seed=2103 + rank)
    work = sum(j.steps for j in jobs)
    res = {}
    runs = (("sjf_cap150GB", 150 << 30, "sjf"), ("fifo_cap150GB", 150 << 30, "fifo"),
            ("sjf_cap2GB", 2 << 30, "sjf"), ("fifo_cap2GB", 2 << 30, "fifo"))
    for name, cap, policy in runs:
        B = Batch(capacity=256, hbm_cap_bytes=cap, precision=32)
        srv = Server(B, step_batch=10, fields=("pos",), policy=policy,
                     max_particles=2_000_000 if policy == "sjf" else None, max_wait=30.0)
        barrier()
        t0 = time.perf_counter()
        done = srv.run(jobs)
        t = allmax(time.perf_counter() - t0)
        B.close()
        res[name] = dict(percentiles(done), scene_steps_per_s=allsum(work) / t, seconds=t,
                         peak_jobs=srv.max_jobs, peak_bytes=srv.max_bytes, failed=sum(d.failed for d in done))
    for policy in ("fifo", "sjf"):
        barrier()
        t0 = time.perf_counter()
        done = serve_plain(jobs, lambda sc, **kw: Scene(sc, precision=32, **kw), fields=("pos",), policy=policy)
        t = allmax(time.perf_counter() - t0)
        res["plain_" + policy] = dict(percentiles(done), scene_steps_per_s=allsum(work) / t, seconds=t,
                                      failed=sum(d.failed for d in done))
    b = res["sjf_cap150GB"]
    out = {"metric": "p50/p99 job latency, serving (Poisson 20/s) vs plain", "value": b["p50"], "unit": "s",
           "n_gpus": world, "steps": args.job_steps, "warmup": 0, "ms_per_step": None,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "%d jobs, N log-uniform [5e3, 1e6], 0-100 bodies, %d steps each, Poisson "
                                  "arrivals 20/s" % (len(jobs), args.job_steps),
                      "policy": "shortest work first, 2M resident particles, 150 GB cap (all runs in 'serving')",
                      "particles": int(sum(len(j.scene["particles"]["mass"]) for j in jobs))},
           "p99": b["p99"], "serving": res,
           "e2e": {"value": b["p50"], "unit": "s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                   "note": "latency is end to end: host inputs in, positions out"}}
    if rank == 0:
        print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    from paper_2103_07925_gb300.replicas import from_env
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep, local = from_env("nccl")  # one replica per GPU; no collective on the data path
    world, rank, dist = rep.world, rep.rank, rep.dist
    barrier, allmax, allsum = rep.barrier, rep.max, rep.sum

    if args.workload == "batch":
        bench_batch(args, rank, world, allmax, allsum, barrier)
        return
    if args.workload == "serve":
        bench_serve(args, rank, world, allmax, allsum, barrier)
        return
    from paper_2103_07925_gb300.sph import Scene, fp32_peak
    hbm, smmax, peak_src = peaks()
    # FP32 FMA peak of this GPU, measured by the library's own microbenchmark (best of four
    # launches of about 40 ms), and the SM count it found
    peak_tf, n_sm, _ = fp32_peak()
    dx = args.dx or DEFAULT_DX[args.workload]
    preheat = tuple(float(v) for v in args.preheat.split(",")) if args.preheat else None
    sc = workload(dx, args.workload, preheat)
    if args.p_background > 0:
        fl = [m for m in sc["materials"] if m["kind"] == 0][0]
        sc["params"]["p_background"] = args.p_background * fl["rho0"] * fl["c"] ** 2
    stream = torch.cuda.Stream()
    # cell layout and launch shape: the autotuner's pick on this workload (steps 30-60 from
    # the initial state), or the command-line layout with --no-tune
    if args.no_tune:
        layout = dict(key_order=args.key_order, cells_per_group=args.cells_per_group, skin=args.skin * sc["params"]["h"])
        launch = dict(sweep_block=256, sweep_waves=0, search_waves=0)
        tuned = None
    else:
        from paper_2103_07925_gb300.tune import tune_scene
        t_tune = time.perf_counter()
        tn = tune_scene(sc, precision=args.precision, steps=30, warmup=30, use_cache=False)
        layout, launch = dict(tn.params), dict(tn.launch)
        tuned = dict(layout, **launch, ms_per_step=tn.ms_per_step, seconds=time.perf_counter() - t_tune,
                     trials=len(tn.table))
    relabel_step1 = None
    if args.workload == "powder" and any(m["transitions_to"] >= 0 for m in sc["materials"]):
        # the first step of a fresh scene, stage by stage (the preheated bed melts the hot
        # parts of its grains there): relabelled particles and the time of each stage
        g1 = Scene(sc, precision=args.precision, stream=stream.cuda_stream, **layout)
        g1.set_launch(**launch)
        prof1 = g1.profile(1)
        relabel_step1 = {"relabelled": g1.info()["relabelled"], "profile_ms": prof1}
        g1.close()
    g = Scene(sc, precision=args.precision, stream=stream.cuda_stream, **layout)
    g.set_launch(**launch)
    info = g.info()
    g.step(args.warmup)
    clocks = Clocks(local)
    p_before = g.info()["pairs_total"]
    rl_before = g.info()["relabelled"]
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
    pairs_per_step = pairs / args.steps
    # context: the nominal FP32 peak at the SM clock sampled during the timed region
    clock_mhz = clk["sm_mhz"] or smmax
    nominal_tf = n_sm * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    full_tank = args.workload == "tank3d" and dx == 0.01 and args.precision == 32 and args.p_background == 0
    skin_h = round(layout["skin"] / sc["params"]["h"], 3)

    def roofline(kernel, ms, flop, alg_bytes):
        ach = flop / (ms * 1e-3) / 1e12
        hb = alg_bytes / (ms * 1e-3) / 1e9
        return {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s", "frac": ach / peak_tf,
                "traffic": TRAFFIC.get((kernel, layout["key_order"], skin_h)) if full_tank else None,
                "kernel": kernel, "ms_per_launch": ms,
                "peak_source": "measured: FP32 FMA microbenchmark of the library (sph_fp32_peak) on this "
                               "GPU, %d SMs" % n_sm,
                "nominal_at_sampled_clock": {"value": nominal_tf, "sm_mhz": clock_mhz, "frac": ach / nominal_tf},
                "hbm": {"achieved_gbs": hb, "peak_gbs": hbm, "frac": hb / hbm, "peak_source": peak_src}}

    rl_force = roofline("k_force", prof["force"], pairs_per_step * FLOP_PER_PAIR,
                        (info["n_fluid"] + info["n_rigid"]) * BYTES_PER_TARGET)
    rl_density = roofline("k_density", prof["density"], pairs_per_step * FLOP_PER_DENSITY_PAIR,
                          info["n_fluid"] * BYTES_PER_DENSITY_TARGET)
    dominant, other = (rl_density, rl_force) if prof["density"] >= prof["force"] else (rl_force, rl_density)
    out = {"metric": METRIC, "value": value, "unit": "pair-interactions/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME[args.workload] % dx,
                      "particles": info["n"], "fluid": info["n_fluid"], "rigid": info["n_rigid"],
                      "wall": info["n_wall"], "bodies": info["n_bodies"], "cells": info["n_cells"],
                      "precision": "FP32 pair sums, FP64 bodies" if args.precision == 32 else "FP64",
                      "p_background_over_p0": args.p_background,
                      "preheat": preheat,
                      "grains": sc.get("info", {}).get("grains"),
                      "key_order": "morton" if layout["key_order"] == 0 else "row-major",
                      "cells_per_group": layout.get("cells_per_group", 0),
                      "skin_h": layout["skin"] / sc["params"]["h"],
                      "launch": launch, "tuned": tuned,
                      "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (info["bytes"] / 1e6),
                      "parallelism": "replica per GPU" if world > 1 else "1 GPU"},
           "steps_per_s": steps_per_s * world,
           "pairs_per_step": pairs_per_step,
           "list_rebuilds": g.info()["rebuilds"],
           "relabelled": g.info()["relabelled"],
           "relabelled_per_timed_step": (g.info()["relabelled"] - rl_before) / args.steps,
           "first_step_of_a_fresh_scene": relabel_step1,
           "gpu_launches": args.steps * g.info()["kernels_per_step"],
           "roofline": dominant,
           "roofline_" + other["kernel"]: other,
           "profile_ms": prof, "clocks": clk}
    # plain FP64 path on the same workload, with its own skin: its sweeps walk the full
    # lists with the distance test and its pair arithmetic is bound by the FP64 units, so
    # short lists pay more than rare rebuilds (200 steps of the tank: 25.5 ms/step at
    # 0.15 h, 29.7 at 0.3 h, 39.4 at 0.7 h)
    if not args.no_fp64 and args.precision == 32:
        s64 = torch.cuda.Stream()
        layout64 = dict(layout, skin=FP64_SKIN_H * sc["params"]["h"])
        g64 = Scene(sc, precision=64, stream=s64.cuda_stream, **layout64)
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
                       "steps_per_s": k64 / (m64 / 1e3), "skin_h": FP64_SKIN_H,
                       "window": "steps 3-%d of a fresh scene" % (2 + k64)}
        g64.close()
    # FP32 against the FP64 path on the same workload and layout: every output field after
    # one step from the same initial state, body trajectories after 100 steps
    if not args.no_fp64 and args.precision == 32:
        from paper_2103_07925_gb300.errors import PLAIN32, body_errors, edge_only_boundary, field_scales, rel_err
        a32 = Scene(sc, precision=32, **layout)
        a64 = Scene(sc, precision=64, **layout)
        a32.set_launch(**launch)
        a32.step(1)
        a64.step(1)
        flds = ("pos", "vel", "acc", "rho", "pres", "temp", "dtemp", "force", "vext")
        f32, f64 = a32.read(*flds), a64.read(*flds)
        sca = field_scales(sc)
        step1 = {f: rel_err(f32[f], f64[f], scale=sca.get(f, 0.0)) for f in flds}
        # wall / rigid particles whose fluid neighbours all sit at the support edge
        edge = edge_only_boundary(sc, f64["pos"], sc["particles"]["material"])
        step1_edge = {f: rel_err(f32[f], f64[f], mask=~edge, scale=sca.get(f, 0.0)) for f in ("pres", "vext")}
        # the same without term scales: relative to max(|x64|, RMS(x64)) of the field itself,
        # and the force on each body (the sum over its particles)
        plain1 = {f: rel_err(f32[f], f64[f], mask=~edge if f in ("pres", "vext") else None) for f in flds}
        bo32, bo64 = a32.bodies(), a64.bodies()
        plain1["body_force"] = float(np.max(np.abs(bo32["force"] - bo64["force"])) / np.max(np.abs(bo64["force"])))
        a32.step(99)
        a64.step(99)
        b100 = body_errors(a32.bodies(), a64.bodies(), sc, a64.read("body"))
        out["fp32_vs_fp64"] = {"step1_fields": step1,
                               "step1_fields_plain": plain1,
                               "tolerance_plain": PLAIN32,
                               "step1_without_edge_only_boundary": dict(step1_edge, particles_excluded=int(edge.sum())),
                               "bodies_after_100_steps": b100,
                               "tolerance": {"fields_per_step": 1e-5, "bodies_100_steps": 1e-3},
                               "metric": "max |x32 - x64| / max(|x64|, RMS(x64), term scale of the field); "
                                         "plain: max |x32 - x64| / max(|x64|, RMS(x64)), pres and vext without "
                                         "the edge-only boundary particles"}
        a32.close()
        a64.close()
    # end to end through the C ABI with host buffers: the host holds the fluid state; every
    # step writes it from pinned memory, advances one step and reads the new state back
    # into the same pinned arrays (so the scene evolves as in the device-timed run)
    if not args.no_e2e:
        n = info["n"]
        st = {"pos": torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy(),
              "vel": torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy(),
              "temp": torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()}
        g.read("pos", "vel", "temp", out=st)
        ke = max(3, min(args.steps // 10, 20))
        q0 = g.info()["pairs_total"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            g.write(pos=st["pos"], vel=st["vel"], temp=st["temp"])
            g.step(1)
            g.read("pos", "vel", "temp", out=st)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        q1 = g.info()["pairs_total"]
        te = allmax(te)
        nbytes = int(sum(a.nbytes for a in st.values()))
        # the host link alone: plain copies of the same bytes between page-locked host memory
        # and the device, one way and then the other (the floor of the added time per step)
        hb = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        db = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        for _ in range(2):
            db.copy_(hb, non_blocking=True)
            hb.copy_(db, non_blocking=True)
        c0.record()
        for _ in range(ke):
            db.copy_(hb, non_blocking=True)
        c1.record()
        for _ in range(ke):
            hb.copy_(db, non_blocking=True)
        c2.record()
        torch.cuda.synchronize()
        h2d_ms, d2h_ms = c0.elapsed_time(c1) / ke, c1.elapsed_time(c2) / ke
        del hb, db
        out["e2e"] = {"value": allsum(q1 - q0) / te, "unit": "pair-interactions/s",
                      "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": ke,
                      "ms_per_step": 1e3 * te / ke,
                      "host_link": {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms, "h2d_gbs": nbytes / h2d_ms / 1e6,
                                    "d2h_gbs": nbytes / d2h_ms / 1e6}}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(sc)
    g.close()
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
