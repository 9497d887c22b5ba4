"""Benchmark of the NBGS granular time step on GB300.

A step is one nbgs_step(): contact detection, colouring, NBGS sweeps
(100 or residual 1e-6) and integration.  The default workload is the settled
1M-sphere pour: 1,000,000 polydisperse spheres (r ~ U(0.4, 0.6), density 1)
poured from a loose lattice at volume fraction 0.3 into a walled
100 x 100 x 200 box and settled under gravity (untimed, on the GPU: 3,000
steps of 2e-3 with 30 sweeps), then measured at mu = 0.5, dt = 5e-4, 100
sweeps or residual 1e-6, previous-step warm start, FP32 sweeps, FP64
positions.  Its working set (~0.8 GB) is larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  value = contact updates per second of whole-step
device time (CUDA events on the scene stream), summed over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contact updates/s in NBGS sweeps"
UNIT = "contact updates/s"
SWEEPS, TOL = 100, 1e-6
# algorithmic bytes per contact update of the sweep kernel (read + write of
# what must move once): sphere-sphere and sphere-wall, FP32 / FP64
BYTES = {"fp32": (168, 112), "fp64": (328, 216)}
# composites: record 80 / 160 B, impulse read + write, per body 4 records
# read (v, w, inverse inertia) and 2 written
BYTES_COMP = {"fp32": (80 + 32 + 2 * 96, 80 + 32 + 96), "fp64": (160 + 64 + 2 * 192, 160 + 64 + 192)}


def workload(name: str):
    from paper_1501_05810_gb300 import scenes
    if name == "pour1m":
        sc = scenes.loose_pour(seed=0, n=1_000_000, precision="fp32", warm_start="prev")
        dt_s, sw_s, n_s = PRE_SETTLE["pour1m"]
        desc = ("settled pour of 1,000,000 spheres r~U(0.4,0.6) (loose lattice at phi=0.3 in a walled 100x100x200 "
                f"box, settled under gravity for {n_s} untimed steps of dt={dt_s:g} with {sw_s} sweeps), mu=0.5, "
                "dt=5e-4, 100 sweeps or residual 1e-6, previous-step warm start, FP32 sweeps, FP64 positions")
        return sc, desc
    if name == "dense1m":
        sc = scenes.dense_packing(1_000_000, seed=0, precision="fp32", warm_start="prev")
        desc = ("dense packing of 1,000,000 spheres (HCP 100x100x100, r=0.5, periodic x,y, walls z), "
                "gravity -9.81 z, mu=0.5, dt=5e-4, 100 sweeps or residual 1e-6, previous-step warm start, "
                "FP32 sweeps, FP64 positions")
        return sc, desc
    if name == "config1":
        sc = scenes.config1(0)
        return sc, "1,000 spheres in a 10.5^3 walled box, FP64, mu=0.5, dt=1e-3, 50 sweeps"
    if name == "config1_1e6":
        sc = scenes.config1(0)
        return sc, ("1,000 spheres in a 10.5^3 walled box, FP64, mu=0.5, dt=1e-3, time steps to residual 1e-6 "
                    "(at most 1,000 sweeps), cold start")
    if name == "gas":
        sc = scenes.granular_gas(cells=196, seed=0, precision="fp32", contacts_per_body=2)
        return sc, (f"dense granular gas, {len(sc['radius']):,} spheres r~U(0.45,0.55), FCC start at phi=0.5, "
                    "triply periodic, v~N(0,1), mu=0.3, dt=1e-4, 50 sweeps, FP32 sweeps, FP64 positions")
    if name == "ramp":
        sc = scenes.hcp_packing(100, 100, 100, dt=1e-5, tau=0.005, mu=0.85, tilt_deg=30.0, v0=0.1, omega=0.75,
                                precision="fp32", warm_start="prev")
        return sc, ("HCP ramp (Sect. 7.2.2 shape): 1,000,000 spheres r=0.5, periodic x,y, walls z, gravity tilted "
                    "30 deg, mu=0.85, v0=0.1 downhill, omega=0.75, dt=1e-5, 100 sweeps, previous-step warm start, "
                    "FP32 sweeps")
    if name == "batch":
        bs = scenes.batch_scenes(4096, seed=0, precision="fp32", contacts_per_body=4, warm_start="prev")
        return bs, (f"4,096 walled-box scenes, {sum(len(b['radius']) for b in bs):,} spheres in total, sizes "
                    "log-uniform in [200, 20000], r~U(0.4,0.6), mu~U(0.2,0.8), settling under gravity from a loose "
                    "lattice, dt=5e-4, residual 1e-6 per scene (max 1,000 sweeps), previous-step warm start, one "
                    "persistent sweep launch for all scenes per step, steps replayed from captured CUDA graphs")
    if name == "hopper":
        sc = scenes.hopper(2_000_000, seed=0, precision="fp32", warm_start="prev")
        return sc, ("conical hopper discharge: 2,000,000 spheres r~U(0.4,0.6), 30 deg half-angle, orifice 8 r_mean, "
                    "mu=0.5, dt=5e-4, previous-step warm start, measured after 2,000 settling steps (30 sweeps), "
                    "100 sweeps or residual 1e-6, FP32 sweeps, FP64 positions")
    if name == "compgas":
        sc = scenes.composite_gas(160, 160, 160, seed=0, precision="fp32", contacts_per_body=2)
        return sc, (f"granular gas of composite particles (Sect. 7.2.1 as run): {len(sc['pos']):,} bodies of 2-4 "
                    f"spheres ({len(sc['members']['body']):,} members, diameters U(0.6, 0.8) inside a bounding "
                    "sphere of diameter 1), Cartesian grid of spacing 1.1, velocities U(-0.2, 0.2) per component, "
                    "walls, no gravity, mu=0.1, omega=0.75, dt=1e-4, 10 sweeps, FP32 sweeps, FP64 positions")
    if name == "comppile":
        sc = scenes.composite_gas(100, 100, 100, seed=0, spacing=1.02, v_max=0.5, dt=2e-2, mu=0.4, omega=1.0,
                                  gravity=(0.0, 0.0, -9.81), precision="fp32", contacts_per_body=8,
                                  warm_start="prev")
        sc["vel"][:, 2] -= 3.0
        return sc, (f"pile of composite particles: {len(sc['pos']):,} bodies of 2-4 spheres "
                    f"({len(sc['members']['body']):,} members) on a grid of spacing 1.02 thrown down at 3 m/s into a "
                    "walled box under gravity, mu=0.4, dt=2e-2, 50 sweeps, previous-step warm start, FP32 sweeps, "
                    "FP64 positions")
    raise SystemExit(f"unknown workload {name}")


# sweeps and tolerance per workload: (max_sweeps, tol)
SOLVE = {"pour1m": (100, 1e-6), "dense1m": (100, 1e-6), "config1": (50, 0.0), "gas": (50, 0.0), "ramp": (100, 0.0),
         "batch": (1000, 1e-6),
         "hopper": (100, 1e-6), "compgas": (10, 0.0), "comppile": (50, 0.0), "config1_1e6": (1000, 1e-6)}
# untimed steps (sweeps, count) that bring a workload into its regime first
SETTLE = {"hopper": (30, 2000), "config1_1e6": (50, 150)}
# timed steps per workload when --steps is not given (the batch: the 500
# steps of its configuration)
DEFAULT_STEPS = {"batch": 500}
# workloads timed as replayed CUDA graphs by default
GRAPH_DEFAULT = ("batch",)
# settled first in a scene of its own with a larger time step: (dt, sweeps,
# steps); the measured scene starts from the settled state
PRE_SETTLE = {"pour1m": (2e-3, 30, 3000)}   # the schedule of workloads.POUR_SETTLE


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms by a
    reader thread; only samples taken inside [mark_start, mark_end] count."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        t = time.perf_counter()
        while not self.lines and time.perf_counter() - t < 5.0:   # wait for the first sample
            time.sleep(0.02)

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in list(self.lines):
            if self.t0 is not None and not (self.t0 <= ts <= (self.t1 or ts) + 0.2):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_traffic(prec, contacts, sweeps, variant="", kernel="k_solve_persistent", workload="pour1m"):
    """DRAM bytes per launch of the sweep kernel from the committed ncu
    capture of the same workload (profiles/traffic.json, key: kernel, then
    the workload and variant), scaled by the contact updates of one launch;
    None when there is no such capture or the kernel's sources (the entry's
    "sources", else solve.cu and nbgs_internal.cuh) changed since it."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    key = f"{kernel}<{'float' if prec == 'fp32' else 'double'}> {workload}" + variant
    d = json.load(open(p)).get(key)
    if not d:
        return None
    src = b"".join(open(os.path.join(ROOT, "paper_1501_05810_gb300", "csrc", f), "rb").read()
                   for f in d.get("sources", ("solve.cu", "nbgs_internal.cuh")))
    if hashlib.sha256(src).hexdigest()[:16] != d["source_sha256_16"]:
        return None
    return d["dram_bytes_per_update"] * contacts * sweeps


def count_contact_kinds(g, n):
    c = g.get_contacts()
    walls = int(np.count_nonzero(c["j2"] >= getattr(g, "n_members", n)))   # walls follow the members
    sizes = np.bincount(c["colour"][c["colour"] >= 0]).tolist() if len(c["colour"]) else []
    return len(c["j2"]) - walls, walls, sizes


def count_instances(g, n):
    """Subdomains: (bodies with more than one velocity instance, extra
    instances) of the last colouring -- every distinct (body, subdomain)
    pair among the contact ends beyond the first per body."""
    c = g.get_contacts()
    sub = g.get_subdomains().astype(np.int64)
    ends = np.concatenate([c["j1"].astype(np.int64), c["j2"].astype(np.int64)])
    subs = np.concatenate([sub, sub])
    keep = ends < n
    pairs = np.unique(ends[keep] * (int(sub.max()) + 1 if len(sub) else 1) + subs[keep])
    bodies = pairs // (int(sub.max()) + 1 if len(sub) else 1)
    per = np.bincount(bodies, minlength=n)
    return int(np.count_nonzero(per > 1)), int(np.maximum(per - 1, 0).sum())


# the oracle's sample of the pour: a 2,000-sphere pour of the same recipe
# (its box scaled with n^(1/3)), settled by the oracle itself (untimed)
CPU_POUR_N, CPU_POUR_SETTLE = 2000, (2e-3, 30, 1500)


def cpu_sample(name: str):
    """(oracle scene, description) of the bounded CPU sample of a workload."""
    import oracle
    from paper_1501_05810_gb300 import scenes
    if name == "pour1m":
        sc = scenes.loose_pour(seed=1, n=CPU_POUR_N, warm_start="prev")
        dt_s, sw_s, n_s = CPU_POUR_SETTLE
        o = oracle.OracleScene(dict(sc, params=dict(sc["params"], dt=dt_s)))
        for _ in range(n_s):
            o.step(sw_s)
        b = o.get_bodies()
        o.close()
        sc = dict(sc, pos=b["pos"], vel=b["vel"], angvel=b["angvel"])
        return oracle.OracleScene(sc), (f"a {CPU_POUR_N:,}-sphere pour of the same recipe settled by the oracle "
                                        f"({n_s} untimed steps of dt={dt_s:g}, {sw_s} sweeps)")
    sc = scenes.hcp_packing(24, 24, 10, radius=0.5, dt=5e-4, mu=0.5, tau=0.005)
    return oracle.OracleScene(sc), "a 5,760-sphere 24x24x10 cut of the dense packing"


def cpu_baseline(name: str = "pour1m", steps_budget_s: float = 15.0):
    """The oracle, as it stands, on a bounded sample of the same workload
    (cpu_sample), whole steps (O(N^2) detection + 100 sweeps or residual
    1e-6) for about steps_budget_s seconds."""
    o, what = cpu_sample(name)
    t0 = time.perf_counter()
    updates, steps = 0, 0
    while True:
        st = o.step(SWEEPS, TOL)
        updates += st["n_contacts"] * st["sweeps_done"]
        steps += 1
        if time.perf_counter() - t0 > steps_budget_s and steps >= 2:
            break
    dt = time.perf_counter() - t0
    return {"value": updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} whole oracle steps (brute-force detection + {SWEEPS} sweeps / tol {TOL}) of {what}, "
                      f"{updates:,} contact updates in {dt:.1f} s, 1 thread, host nproc={os.cpu_count()}"}, what


def steps_to_residual(nbgs, torch, local, steps=30):
    """The metric's second part, time steps per second to residual 1e-6, on
    the 1,000-sphere FP64 box (the large packings do not reach 1e-6 in a
    bounded run): settled for 150 steps of 50 sweeps, 3 warm-up steps, then
    `steps` whole steps timed with CUDA events, each solved to R_k <= 1e-6
    (at most 1,000 sweeps) from a cold start."""
    from paper_1501_05810_gb300 import scenes
    stream = torch.cuda.Stream(device=local)
    with torch.cuda.stream(stream):
        g = nbgs.Scene(scenes.config1(0), device=f"cuda:{local}", stream=stream)
        for _ in range(150):
            g.step(50, 0.0, stats=False)
        for _ in range(3):
            g.step(1000, 1e-6)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = [g.step(1000, 1e-6) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        g.close()
    return {"value": steps / (ms / 1e3), "unit": "time steps/s", "steps": steps,
            "workload": "1,000 spheres in a 10.5^3 walled box, FP64, mu=0.5, dt=1e-3, cold start, each step to "
                        "residual 1e-6 (at most 1,000 sweeps), after 150 settling steps",
            "sweeps_per_step_mean": statistics.mean(x["sweeps_done"] for x in st),
            "residual_max": max(float(x["residual"]) for x in st), "contacts": st[-1]["n_contacts"]}


def compare_one_by_one(nbgs, torch, g, scene_list, sweeps, tol, stream, local, sample=64, steps=5):
    """The batched form against the same scenes solved one by one by plain
    cold-start NBGS on the same GPU, from the batch's current state: the
    batch's next `steps` steps as replayed graphs (previous-step warm start),
    and for a sample of the scenes (evenly spaced in order of size) `steps`
    ordinary steps each in a scene of its own with no warm start, after one
    untimed step that sizes its buffers.  The sample's time is scaled by the
    scene count."""
    b = g.get_bodies()
    off = g.offsets
    S = len(scene_list)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.get_updates()
    e0.record(stream)
    g.graph_step(sweeps, tol, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1)
    u_batch = g.get_updates()
    sizes = np.diff(off)
    pick = np.argsort(sizes, kind="stable")[np.linspace(0, S - 1, min(sample, S)).astype(int)]
    t_one, u_one = 0.0, 0
    for i in pick:
        sl = slice(int(off[i]), int(off[i + 1]))
        d = dict(scene_list[i], pos=b["pos"][sl], vel=b["vel"][sl], angvel=b["angvel"][sl])
        d["params"] = dict(d["params"], warm_start="none")
        one = nbgs.Scene(d, device=f"cuda:{local}", stream=stream)
        one.step(sweeps, tol, stats=False)
        one.set_bodies(b["pos"][sl], b["quat"][sl], b["vel"][sl], b["angvel"][sl])
        one.get_updates()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            one.step(sweeps, tol, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t_one += e0.elapsed_time(e1)
        u_one += one.get_updates()
        one.close()
    est = t_one * S / len(pick)
    return {"scenes": S, "sample_scenes": int(len(pick)), "steps": steps, "sweeps_max": sweeps, "tol": tol,
            "batched_ms_per_step": t_batch / steps, "batched_contact_updates": int(u_batch),
            "one_by_one_ms_per_step_est": est / steps, "one_by_one_sample_contact_updates": int(u_one),
            "speedup_batched_over_one_by_one": est / t_batch if t_batch > 0 else None,
            "one_by_one": "each sampled scene alone, nbgs_step with no warm start (plain cold-start NBGS), "
                          "time scaled by scenes / sample"}


def steps_to_residual_batch(nbgs, torch, local, steps=200):
    """The metric's second part, time steps per second to residual 1e-6
    (at most 1,000 sweeps), on the largest workload that reaches it: the
    4,096-scene batch (17.6M spheres settling in their boxes), every scene
    solved to 1e-6 in every step, 3 ordinary warm-up steps then `steps`
    replayed graph steps timed with CUDA events."""
    from paper_1501_05810_gb300 import scenes
    stream = torch.cuda.Stream(device=local)
    with torch.cuda.stream(stream):
        bs = scenes.batch_scenes(4096, seed=0, precision="fp32", contacts_per_body=4, warm_start="prev")
        g = nbgs.BatchScene(bs, device=f"cuda:{local}", stream=stream)
        for _ in range(3):
            g.step(1000, 1e-6)
        g.graph_step(1000, 1e-6, 1)
        g.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.graph_step(1000, 1e-6, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ks, rs = g.scene_stats()
        nc = len(g.get_contacts()["j1"])
        g.close()
    return {"value": steps / (ms / 1e3), "unit": "time steps/s", "steps": steps,
            "workload": "4,096 walled-box scenes (17.6M spheres, sizes log-uniform in [200, 20000]) settling under "
                        "gravity, every scene to residual 1e-6 (at most 1,000 sweeps) in every step, FP32 sweeps, "
                        "previous-step warm start, replayed CUDA graphs",
            "scenes_at_tol_last_step": int(np.count_nonzero(rs <= 1e-6)), "sweeps_last_step_max": int(ks.max()),
            "contacts_last_step": nc}


def reduce_over_ranks(dist, ms_total, updates, device):
    """Replicas: the job's time is the slowest rank's, its work the sum of
    all ranks' (no data-path collective; this reduction runs once, after the
    timed region)."""
    if dist is None:
        return float(ms_total), float(updates)
    import torch
    t = torch.tensor([float(ms_total)], device=device, dtype=torch.float64)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    name = args.workload if args.workload in ("pour1m", "dense1m") else "pour1m"
    cb, what = cpu_baseline(name, min(20.0, 5.0 + 2.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"oracle on {what} (the full size needs O(N^2) detection)",
                       "l2": "inputs smaller than L2 (CPU run)"},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: 500 for batch, else 30)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="pour1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--sweep-flags", type=int, default=None, help="nbgs_params.sweep_flags override")
    ap.add_argument("--warm", default=None, choices=["none", "prev"], help="warm start of the solves")
    ap.add_argument("--subdomains", default=None,
                    help="subdomains of Alg. 1: 'jacobi' (one per contact) or a grid 'g0,g1,g2'")
    ap.add_argument("--omega", type=float, default=None, help="relaxation parameter of Alg. 1")
    ap.add_argument("--graph", default="auto", choices=["auto", "on", "off"],
                    help="time replayed CUDA graphs of the step (auto: for the batch)")
    ap.add_argument("--autotune", action="store_true",
                    help="after the warm-up, let nbgs_autotune pick the sweep schedule and blocks per SM (untimed)")
    args = ap.parse_args()

    steps = args.steps if args.steps is not None else DEFAULT_STEPS.get(args.workload, 30)
    args.steps = steps
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1501_05810_gb300 import nbgs
    sc, desc = workload(args.workload)
    batch = isinstance(sc, list)
    first = sc[0] if batch else sc
    if args.sweep_flags is not None:
        for x in (sc if batch else [sc]):
            x["params"]["sweep_flags"] = args.sweep_flags
    if args.warm is not None:
        for x in (sc if batch else [sc]):
            x["params"]["warm_start"] = args.warm
        desc += f", warm start {args.warm}"
    if args.subdomains is not None:
        sub = "jacobi" if args.subdomains == "jacobi" else tuple(int(v) for v in args.subdomains.split(","))
        for x in (sc if batch else [sc]):
            x["params"]["subdomains"] = sub
        desc += (", non-linear block Jacobi (one subdomain per contact)" if sub == "jacobi"
                 else f", subdomain NBGS on a {sub[0]}x{sub[1]}x{sub[2]} grid")
    if args.omega is not None:
        for x in (sc if batch else [sc]):
            x["params"]["omega"] = args.omega
        desc += f", omega={args.omega}"
    prec = first["params"].get("precision", "fp64")
    stream = torch.cuda.Stream(device=local)
    with torch.cuda.stream(stream):
        if args.workload in PRE_SETTLE:
            from paper_1501_05810_gb300 import workloads
            dt_s, sw_s, n_s = PRE_SETTLE[args.workload]
            sc = workloads.settle(sc, dt_s, sw_s, n_s, device=f"cuda:{local}", stream=stream)
        if batch:
            g = nbgs.BatchScene(sc, device=f"cuda:{local}", stream=stream)
        else:
            g = nbgs.Scene(sc, device=f"cuda:{local}", stream=stream)
        n = g.n
        sweeps, tol = SOLVE[args.workload]
        if args.workload in SETTLE:
            s_sweeps, s_steps = SETTLE[args.workload]
            for _ in range(s_steps):
                g.step(s_sweeps, 0.0, stats=False)
        for _ in range(max(args.warmup, 0)):
            g.step(sweeps, tol)
        tuned = None
        if args.autotune:
            g.detect_contacts()   # the tuner times solves on the current contacts
            f_, b_ = nbgs.autotune(g, sweeps, tol)
            tuned = {"sweep_flags": int(f_), "blocks_per_sm": int(b_)}
            desc += f", autotuned schedule (sweep flags {f_}, {b_} blocks per SM)"
        use_graph = args.graph == "on" or (args.graph == "auto" and args.workload in GRAPH_DEFAULT)
        if use_graph:
            g.graph_step(sweeps, tol, 1)   # captures the step (untimed), then replays it once
            g.sync()
        n_ss, n_sw, colour_sizes = count_contact_kinds(g, n)
        n_shared, n_extra = count_instances(g, n) if args.subdomains is not None else (0, 0)
        clocks = ClockSampler(local)
        clocks.start()
        g.get_updates()   # counted on the device; read (and reset) after the timed region
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.mark_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")   # a profiler can be limited to this range (ncu --nvtx-include timed/)
        e0.record(stream)
        stats = []
        if use_graph:
            g.graph_step(sweeps, tol, steps)   # no host synchronisation inside
        else:
            for _ in range(steps):
                g.step(sweeps, tol, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clocks.mark_end()
        if dist:
            dist.barrier()
        ck = clocks.stop()
        ms_total = e0.elapsed_time(e1)
        updates = g.get_updates()
        batch_stats = None
        if batch:
            ks, rs = g.scene_stats()
            batch_stats = {"scenes": int(len(ks)), "scenes_at_tol_last_step": int(np.count_nonzero(rs <= tol)),
                           "sweeps_last_step": {"median": float(np.median(ks)), "max": int(ks.max()),
                                                "min": int(ks.min())},
                           "residual_last_step_max": float(rs.max())}
        # phase breakdown and the sweep kernel's launch time: a few ordinary
        # steps with the library's CUDA-event timing, right after the timed ones
        g.enable_timing(True)
        n_phase = min(5, steps)
        for _ in range(n_phase):
            stats.append(g.step(sweeps, tol))
        phase_ms, launches = g.get_timings()
        g.enable_timing(False)
        phase_updates = g.get_updates()
        one_by_one = compare_one_by_one(nbgs, torch, g, sc, sweeps, tol, stream, local) if batch else None
        # end to end through the public API with host buffers: upload the
        # state from pinned memory, step, read the state back
        host = {k: torch.empty((n, d), dtype=torch.float64, pin_memory=True)
                for k, d in (("pos", 3), ("quat", 4), ("vel", 3), ("angvel", 3))}
        b = g.get_bodies()
        for k in host:
            host[k].copy_(torch.from_numpy(b[k]))
        torch.cuda.synchronize()
        g.get_updates()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            g.update_bodies(host["pos"], host["quat"], host["vel"], host["angvel"])
            g.step(sweeps, tol, stats=False)
            nbgs._call(g.h, "nbgs_get_bodies", *[host[k].data_ptr() for k in ("pos", "quat", "vel", "angvel")])
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_updates = g.get_updates()

    t_max, updates_all = reduce_over_ranks(dist, ms_total, updates, f"cuda:{local}")
    value = updates_all / (t_max / 1e3)
    sweeps_done = [s["sweeps_done"] for s in stats]
    residuals = [float(s["residual"]) for s in stats]
    contacts = [s["n_contacts"] for s in stats]
    comp = "members" in first
    b_ss, b_sw = (BYTES_COMP if comp else BYTES)[prec]
    # dominant kernel: the persistent sweep kernel, one launch per solve; its
    # contact updates per launch from the device count of the timing steps
    n_launch = max(1, launches["sweep_kernel"])
    upd_launch = phase_updates / n_launch
    per_update = (n_ss * b_ss + n_sw * b_sw) / max(1, n_ss + n_sw)
    sweeps_launch = upd_launch / max(1, n_ss + n_sw)
    alg_bytes_per_launch = upd_launch * per_update
    # subdomains: per sweep, each shared body's accumulator and own record
    # read and written, each extra instance read and written; once, the
    # instances and accumulators set from the bodies
    rec = 32 if prec == "fp32" else 64
    alg_bytes_per_launch += ((4 * rec * n_shared + 2 * rec * n_extra) * sweeps_launch
                             + 2 * rec * n_shared + rec * n_extra)
    per_launch_ms = phase_ms["sweep_kernel"] / n_launch
    sweep_rate = phase_updates / (phase_ms["sweep_kernel"] / 1e3) if phase_ms["sweep_kernel"] > 0 else None
    peak, peak_src = read_peaks()
    # with subdomains the traffic depends on the grid: a capture of the same
    # workload and grid only
    traffic = measured_traffic(prec, n_ss + n_sw, sweeps_launch,
                               "" if args.subdomains is None else f" subdomains {args.subdomains}",
                               "k_solve_comp" if comp else "k_solve_persistent", args.workload)
    achieved = alg_bytes_per_launch / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": t_max / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": desc, **({"bodies": n, "members": int(g.n_members)} if comp else {"spheres": n}),
                   "contacts": contacts[-1], "colours": stats[-1]["n_colours"], "colour_sizes": colour_sizes,
                   "sweeps_per_step": sweeps,
                   "tol": tol, "l2": "inputs larger than L2 (no flush)",
                   "timed_steps": "replayed CUDA graphs (nbgs_graph_step), no host synchronisation"
                                  if use_graph else "nbgs_step calls",
                   **({"autotuned": tuned} if tuned else {}),
                   **({"subdomains": args.subdomains, "shared_bodies": n_shared, "extra_instances": n_extra}
                      if args.subdomains is not None else {}),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "steps_per_s": steps / (t_max / 1e3),
        "contact_updates": updates,
        "sweep_updates_per_s": sweep_rate,
        "sweeps_done": sweeps_done, "residual_reached_max": max(residuals) if residuals else None,
        "phase_ms_per_step": {k: v / n_phase for k, v in phase_ms.items()},
        "phase_timing": f"{n_phase} nbgs_step calls with CUDA-event timing after the timed steps",
        "gpu_launches": int(round(sum(v for k, v in launches.items() if k != "sweep_kernel") * steps / n_phase)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": f"{'k_solve_comp' if comp else 'k_solve_persistent'}<{'float' if prec == 'fp32' else 'double'}>",
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "alg_bytes_per_launch": alg_bytes_per_launch, "launch_ms": per_launch_ms},
        "clocks": ck,
        "e2e": {"value": e2e_updates / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(13 * 8 * n), "d2h_bytes_per_step": int(13 * 8 * n),
                "steps": args.e2e_steps},
    }
    if batch_stats:
        line["batch"] = batch_stats
    if one_by_one:
        line["one_by_one"] = one_by_one
    if args.workload == "pour1m":
        line["steps_to_residual"] = steps_to_residual_batch(nbgs, torch, local)
    if args.workload == "dense1m":
        line["steps_to_residual"] = steps_to_residual(nbgs, torch, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in ("pour1m", "dense1m"):
        line["cpu_baseline"] = cpu_baseline(args.workload)[0]
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
