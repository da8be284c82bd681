"""Benchmark of the DEM contact pipeline on GB300: sphere-steps/s.

Workload (default): the polydisperse settling column, 4,000,000 spheres with R ~ U[0.8,
1.2] mm on a jittered 2.45 mm lattice in a 0.3 x 0.3 x 1.2 m walled box, E = 1e7 Pa,
nu = 0.3, e = 0.5, mu = 0.4, dt = 2e-6 s, synthetic seeded data.  A step is one pass of
the whole hot path (detection as scheduled, contact forces, per-owner reduction,
integration, audit).  The headline is the chosen form (voxel index + FP32 offset, FP32
forces, delayed detection audited every step); the plain FP64 every-step form is timed
on the same workload beside it.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]

Under torchrun (N > 1) every rank runs its own copy of the workload on its own GPU (no
collective in the data path: independent scenes shard trivially) and rank 0 prints one
JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sphere-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4_000_000, help="spheres (default: the 4M settling column)")
    ap.add_argument("--plain-steps", type=int, default=40, help="timed steps of the plain FP64 every-step form")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=4000)
    ap.add_argument("--cpu-sample-seconds", type=float, default=12.0)
    ap.add_argument("--tune-steps", type=int, default=60, help="steps per autotuner trial (0: no tuning)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- algorithmic bytes

def kernel_bytes(precision, n, n_with_entries, pairs, clumps=False):
    """Algorithmic DRAM bytes per launch of the two per-step kernels, each distinct array
    element counted once (state, constants, list rows, history, per-owner force/torque).

    k_integrate (per owner): state read and written, constants, the owner's list-row
    length, the per-owner accumulators, and the contact force/torque of owners with
    listed partners.  k_contact: the row length and active flag of every sphere; for a
    sphere with listed partners its state and constants and the force/torque it writes;
    per listed pair both row entries, one mirror byte, history read and written."""
    if precision == "voxel_fp32":
        integ = n * (1 + 1 + 24 + 16 + 16 + 16 + 4 + 16 + 2 + 1 + 8      # reads
                     + 24 + 16 + 16 + 16 + 1 + 8) + 32 * n_with_entries   # writes, force/torque read
        contact = 2 * n + n_with_entries * (24 + 16 + 16 + 4 + 4 + 2 + 2 + 32) + 33 * pairs
    else:
        integ = n * (1 + 1 + 32 + 32 + 32 + 32 + 8 + 32 + 2 + 1 + 8
                     + 32 + 32 + 32 + 32 + 1 + 8) + 64 * n_with_entries
        contact = 2 * n + n_with_entries * (32 + 32 + 32 + 8 + 2 + 2 + 64) + 57 * pairs
    if clumps:
        contact += n * (16 if precision == "voxel_fp32" else 32)
    return {"integrate": integ, "contact": contact}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- runs

def make_scene(n):
    from paper_2311_04648_gb300 import workloads as W
    return W.settling_column(n=n)


def profile_delta(p0, p1):
    nf = p1["n_force"] - p0["n_force"]
    ni = p1["n_integrate"] - p0["n_integrate"]
    nd = p1["n_detect"] - p0["n_detect"]
    return dict(contact_ms=(p1["ms_force"] - p0["ms_force"]) / max(nf, 1), n_contact=nf,
                integrate_ms=(p1["ms_integrate"] - p0["ms_integrate"]) / max(ni, 1), n_integrate=ni,
                detect_ms=(p1["ms_detect"] - p0["ms_detect"]) / max(nd, 1), n_detect=nd,
                hash_ms=(p1["ms_hash"] - p0["ms_hash"]) / max(nd, 1),
                link_ms=(p1["ms_link"] - p0["ms_link"]) / max(nd, 1),
                listed_pairs=p1["listed_pairs"], active_contacts=p1["active_contacts"],
                with_entries=p1["spheres_with_entries"], list_capacity=p1["list_capacity"])


def roofline(precision, n, prof, peak, peak_kind):
    kb = kernel_bytes(precision, n, prof["with_entries"], prof["listed_pairs"])
    per = {}
    for k in ("contact", "integrate"):
        ms = prof[f"{k}_ms"]
        per[k] = {"ms": ms, "bytes": kb[k], "gbs": kb[k] / (ms / 1000.0) / 1e9 if ms > 0 else None}
    dom = max(per, key=lambda k: per[k]["ms"])
    a = per[dom]["gbs"]
    return {"bound": "hbm", "kernel": {"contact": "k_contact (pair forces + per-owner sums)",
                                       "integrate": "k_integrate (owner update + audit)"}[dom],
            "achieved": a, "peak": peak, "unit": "GB/s", "frac": (a / peak) if a else None, "traffic": None,
            "peak_kind": peak_kind, "bytes_per_launch": per[dom]["bytes"], "avg_launch_ms": per[dom]["ms"],
            "kernels": per, "listed_pairs": prof["listed_pairs"], "spheres_with_entries": prof["with_entries"]}


def run_ours(args, device):
    import torch
    from paper_2311_04648_gb300 import dem

    torch.cuda.set_device(device)
    scene = make_scene(args.n)
    out = {}

    def timed(world, steps):
        stream = torch.cuda.ExternalStream(world.stream(), device=device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        world.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # chosen form: voxel + FP32, delayed detection on the second stream, audited
    w = dem.World.from_scene(scene, precision="voxel_fp32", schedule="velocity_bound", device=device)
    out["tuning"] = w.autotune(steps=args.tune_steps) if args.tune_steps > 0 else w.tuning()
    w.step(args.warmup)
    s0 = w.stats()
    with ClockSampler(device) as clk:
        ms = timed(w, args.steps)
    s1 = w.stats()
    steps = s1["steps"] - s0["steps"]
    rebuilds = s1["rebuilds"] - s0["rebuilds"]
    out["chosen"] = dict(ms=ms, steps=steps, rebuilds=rebuilds, clocks=clk.summary(), stats=s1)
    # profiled pass for per-kernel durations (events on each kernel's own stream)
    w.set_profiling(True)
    p0 = w.stats()
    w.step(max(20, args.steps // 4))
    p1 = w.stats()
    w.set_profiling(False)
    out["profile"] = profile_delta(p0, p1)
    # e2e through the C ABI with host buffers: state in from pinned memory, one step,
    # state out to pinned memory, every step
    n_own = scene.n_owner
    pin = {k: torch.empty(shape, dtype=torch.float64).pin_memory() for k, shape in
           (("x", (n_own, 3)), ("q", (n_own, 4)), ("v", (n_own, 3)), ("w", (n_own, 3)))}
    arrs = {k: t.numpy() for k, t in pin.items()}
    x, q, v, wb = w.owner_state()
    arrs["x"][:] = x; arrs["q"][:] = q; arrs["v"][:] = v; arrs["w"][:] = wb
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        w.set_owner_state(0, xyz=arrs["x"], quat=arrs["q"], vel=arrs["v"], omega=arrs["w"])
        w.step(1)
        L = w.L
        import ctypes as C
        st = L.dem_get_owner_state(w.h, 0, n_own, arrs["x"].ctypes.data_as(C.c_void_p),
                                   arrs["q"].ctypes.data_as(C.c_void_p), arrs["v"].ctypes.data_as(C.c_void_p),
                                   arrs["w"].ctypes.data_as(C.c_void_p))
        assert st == 0
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    out["e2e"] = dict(seconds=e2e_s, steps=args.e2e_steps, bytes_in=13 * 8 * n_own, bytes_out=13 * 8 * n_own)
    out["n_spheres"] = scene.n_sphere
    out["clumps"] = False
    w.close()
    del w
    torch.cuda.synchronize()

    # plain form: FP64, detection every step, same workload
    if args.plain_steps > 0:
        wp = dem.World.from_scene(scene, precision="fp64", schedule="every_step", device=device)
        wp.step(3)
        p0 = wp.stats()
        msp = timed(wp, args.plain_steps)
        p1 = wp.stats()
        wp.set_profiling(True)
        q0 = wp.stats()
        wp.step(5)
        q1 = wp.stats()
        out["plain"] = dict(ms=msp, steps=p1["steps"] - p0["steps"], profile=profile_delta(q0, q1))
        wp.close()
    return out


def cpu_baseline(args):
    """The oracle as it stands (single thread, O(N^2) detection) on a bounded sample of
    the same workload: the central column of the same generator with ~args.cpu_sample_n
    spheres, stepped until ~args.cpu_sample_seconds of CPU time."""
    import math
    import oracle
    from paper_2311_04648_gb300 import workloads as W

    n = args.cpu_sample_n
    # a square column holding ~n spheres over the first few hundred lattice layers
    per_layer = max(1, int(round((n / 28) ** 0.5)) ** 2)
    side = int(round(per_layer ** 0.5))
    width = side * 2.45e-3 + 2 * 1.2e-3 + 1e-6
    s = W.settling_column(n=n, column_width=width)
    ow = oracle.OracleWorld(s)
    ow.step(1)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < args.cpu_sample_seconds:
        ow.step(5)
        steps += 5
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{n}-sphere central column of the settling-column generator ({width * 1e3:.1f} mm wide), "
                      f"{steps} steps in {dt:.1f} s, single thread, brute-force O(N^2) contacts"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        w = args.warmup
        args.cpu_sample_seconds = max(3.0, args.cpu_sample_seconds)
        cb = cpu_baseline(args)
        line = {"metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": w, "ms_per_step": 1000.0 * args.cpu_sample_n / cb["value"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": "settling_column (bounded sample)", "sample": cb["sample"]},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = local
    res = run_ours(args, device)
    ms = res["chosen"]["ms"]
    steps = res["chosen"]["steps"]
    n_sph = res["n_spheres"]
    my_tput_time = ms
    if world > 1:
        import torch.distributed as tdist
        t = torch.tensor([ms], device=f"cuda:{device}", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
        tdist.barrier()
    value = world * n_sph * steps / (ms / 1000.0)
    if rank != 0:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()
        return 0
    prof = res["profile"]
    peak, peak_kind = peaks()
    e2e = res["e2e"]
    e2e_val = n_sph * e2e["steps"] / e2e["seconds"] * world
    plain = res.get("plain")
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms / max(steps, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "settling_column", "n_spheres": n_sph, "radius_mm": [0.8, 1.2],
                   "box_m": [0.3, 0.3, 1.2], "dt_s": 2e-6, "precision": "voxel index + FP32 offset, FP32 forces",
                   "schedule": "delayed detection on a second stream, velocity-bound cycle, audited every step",
                   "margin_m": res["chosen"]["stats"]["margin"],
                   "rebuilds_in_timed_region": res["chosen"]["rebuilds"],
                   "tuning": res["tuning"],
                   "l2": "inputs larger than L2 (owner state + contact lists > 0.5 GB)",
                   "parallelism": f"replica x{world}"},
        "roofline": roofline("voxel_fp32", n_sph, prof, peak, peak_kind),
        "kernels_ms": {"contact": prof["contact_ms"], "integrate": prof["integrate_ms"],
                       "detect": prof["detect_ms"], "hash": prof["hash_ms"], "link": prof["link_ms"]},
        "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": e2e["bytes_in"],
                "d2h_bytes_per_step": e2e["bytes_out"],
                "how": "dem_set_owner_state from pinned host buffers + dem_step(1) + dem_get_owner_state "
                       "to pinned host buffers, every step"},
        "gpu_launches": int(3 * steps + 20 * res["chosen"]["rebuilds"]),
        "clocks": res["chosen"]["clocks"],
    }
    if plain:
        pv = n_sph * plain["steps"] / (plain["ms"] / 1000.0) * world
        pp = plain["profile"]
        line["plain"] = {"value": pv, "unit": METRIC, "ms_per_step": plain["ms"] / max(plain["steps"], 1),
                         "dtype": "f64", "schedule": "every step",
                         "kernels_ms": {"contact": pp["contact_ms"], "integrate": pp["integrate_ms"],
                                        "detect": pp["detect_ms"]},
                         "roofline": roofline("fp64", n_sph, pp, peak, peak_kind),
                         "chosen_over_plain": value / pv}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
