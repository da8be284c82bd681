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
    ap.add_argument("--steps", type=int, default=5000, help="timed steps (the configuration runs 5,000)")
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4_000_000, help="spheres (default: the 4M settling column)")
    ap.add_argument("--plain-steps", type=int, default=40, help="timed steps of the plain FP64 every-step form")
    ap.add_argument("--e2e-steps", type=int, default=32, help="timed end-to-end steps (after 3 untimed)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=20000, help="spheres of the oracle's sub-box sample")
    ap.add_argument("--cpu-sample-seconds", type=float, default=10.0)
    ap.add_argument("--tune-steps", type=int, default=60, help="steps per autotuner trial (0: no tuning)")
    ap.add_argument("--tune-at", type=int, default=2500,
                    help="the autotuner times its candidates from the state after this many steps")
    ap.add_argument("--config-steps", type=int, default=5000, help="steps of the configuration (5,000)")
    ap.add_argument("--window-start", type=int, default=-1,
                    help="step at which the warm-up starts (-1: the tuning step when the warm-up and "
                         "timed steps fit in the configuration's steps after it, else as late as they fit)")
    ap.add_argument("--mixer-start", default="bed", choices=["bed", "above"],
                    help="mixer: elements start as a bed around the blades (mixing from the first step) or "
                         "above them (the paper's release)")
    ap.add_argument("--workload", default="column", choices=["column", "drum", "hopper", "batch", "mixer"],
                    help="column: the headline settling column; the others run one configuration at full size")
    ap.add_argument("--clump", default="sphere", choices=["sphere", "rod3", "six"],
                    help="mixer elements: single spheres, three-sphere or six-sphere clumps")
    ap.add_argument("--set-tuning", default="",
                    help="tuning fields applied after the autotuner, e.g. integrate_staged=1,contact_block=64")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (JSON lines): a later run with the same key reuses its result")
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

def algorithmic_bytes(precision, n, pairs, clumps=False, n_with_entries=0.0, contact_integrates=False):
    """Algorithmic bytes per launch of the two per-step kernels, from the per-unit figures
    of the method's force+integrate step: the owner state read and written once (voxel
    form: voxel 8 + offset 12 + v 12 + w 12 = 44 B each way, 88 B; FP64 form: 3 x 24 B each
    way, 144 B), clumps adding the quaternion (16 B each way), and per listed pair the two
    ids (8 B) with the tangential history read and written (voxel form 12 + 12 B; FP64
    24 + 24 B).  With contact_integrates the contact kernel also updates the owners with
    listed partners (n_with_entries of them) and the integration kernel the others."""
    per_owner = (88 if precision == "voxel_fp32" else 144) + (32 if clumps else 0)
    per_pair = 32 if precision == "voxel_fp32" else 56
    integ = per_owner * n
    contact = per_pair * pairs
    step = integ + contact
    if contact_integrates:
        contact += per_owner * n_with_entries
        integ = per_owner * (n - n_with_entries)
    # the fused step kernel does both: the whole force+integrate figure per launch
    return {"integrate": integ, "contact": contact, "step": step}


def detection_bytes(precision, n, pairs):
    """Algorithmic bytes of one list rebuild (per-unit figures of the method's detection):
    per sphere its position read (voxel form: voxel index 8 + offset 12 = 20 B; FP64 form
    24 B), the cell key and id written and read back (12 B each way), two sort passes over
    them (2 x 24 B) and its share of the cell table (4 B); per listed pair its two ids
    written (8 B) and the history remap, which reads the old ids and history and writes
    the new (2 x (8 + 12) B; FP64 form 2 x (8 + 24) B)."""
    if precision == "voxel_fp32":
        return 96 * n + 48 * pairs
    return 100 * n + 72 * pairs


def layout_bytes(precision, n, n_with_entries, pairs, clumps=False, contact_integrates=False, derived=False):
    """Bytes the kernels actually move in this implementation's layout, each distinct
    array element counted once per launch (context for the algorithmic figure).

    k_integrate (per owner): state read and written (voxel form: a 32-byte position record
    with mass and radius, a 32-byte velocity pair with the two audit accumulators in the
    fourth lanes; quaternion), constants, row length, flags, and the force/torque of
    owners with listed partners.  k_contact: per sphere with listed partners its compacted
    work entry (slot, row length, first partner), active flag, state and the force/torque
    it writes; per listed pair both row entries and both sides' history vectors read and
    written.  k_step_fused: both, without the force/torque array.  With contact_integrates
    (single spheres) the contact kernel also reads the quaternion and constants of its
    owners and writes their state instead of the force/torque, and the integration kernel
    reads every owner's flag and row length but the state of the others only, without
    constants or forces.  With derived constants (voxel form, single spheres of one
    inertia coefficient) no kernel reads 1/m or 1/I (20 B per owner)."""
    if precision == "voxel_fp32":
        # 32-byte position record (offset, mass, voxel index, radius pair) and 32-byte
        # velocity pair (v, w with the audit accumulators) per owner
        integ = n * (1 + 1 + 32 + 32 + 16 + 4 + 16 + 2 + 1              # reads
                     + 32 + 32 + 16 + 1) + 32 * n_with_entries            # writes, force/torque read
        contact = n_with_entries * (16 + 1 + 32 + 32 + 32) + pairs * (8 + 4 * 16)
        # fused step, per owner: permutation, row length, first entry, flag, position
        # record, velocity pair, quaternion, inverse mass and inertia read; record,
        # velocity pair, quaternion and flag written
        step = n * (1 + 1 + 4 + 1 + 32 + 32 + 16 + 4 + 16
                    + 32 + 32 + 16 + 1) + pairs * (8 + 4 * 16)
    else:
        integ = n * (1 + 1 + 32 + 32 + 32 + 32 + 8 + 32 + 2 + 1
                     + 32 + 32 + 32 + 32 + 1) + 64 * n_with_entries
        contact = n_with_entries * (16 + 1 + 32 + 32 + 32 + 16 + 64) + pairs * (8 + 4 * 32)
        step = n * (1 + 1 + 4 + 1 + 32 + 32 + 32 + 16 + 32 + 8 + 32
                    + 32 + 32 + 32 + 32 + 1) + pairs * (8 + 4 * 32)
    if clumps:
        contact += n * (16 if precision == "voxel_fp32" else 32)
    if derived and precision == "voxel_fp32" and not clumps and not contact_integrates:
        integ -= n * (4 + 16)
        step -= n * (4 + 16)
    if contact_integrates and not clumps:
        free = n - n_with_entries
        if precision == "voxel_fp32":
            # reads: quaternion, inverse mass and inertia; writes: record, velocity pair,
            # quaternion and flag, instead of the force/torque
            contact += n_with_entries * (16 + 4 + 16 + 32 + 32 + 16 + 1 - 32)
            integ = n * (1 + 1) + free * (32 + 32 + 16 + 4 + 32 + 32 + 16 + 1)
            if derived:
                contact -= n_with_entries * (4 + 16)
                integ -= free * 4
        else:
            contact += n_with_entries * (32 + 8 + 32 + 32 + 32 + 32 + 32 + 1 - 64)
            integ = n * (1 + 1) + free * (32 + 32 + 32 + 8 + 32 + 32 + 32 + 32 + 1)
    return {"integrate": integ, "contact": contact, "step": step}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one-pass
# ncu captures of the 4M-sphere bench workload mid-run (profiles/dram_traffic_settling_
# column_4M.md), valid while the kernels' source text (the kernel, the functions it
# inlines, the voxel form's storage) hashes to the recorded values.  The contact kernel's
# figure also needs the detection margin of the capture, since the margin sets how many
# pairs are listed.  The integration streams every owner whatever the margin; only its
# read of the force array (32 B per owner with listed partners, under 5% of its bytes
# here) depends on the margin, so its figure carries no margin.
_INTEGRATE_SOURCE = [("pipeline.cuh", "integrate_owner(const Dev<F> &d", "81371d9d1a4c53fd"),
                     ("pipeline.cuh", "integrate_core(const Dev<F> &d", "ceab88a14f25d2a5"),
                     ("pipeline.cuh", "audit_slots(unsigned int *audit", "bbac98b73df81d9c"),
                     ("common.cuh", "struct FormF32 {", "02359980dafed2e7")]
MEASURED_TRAFFIC = {
    "integrate": [
        {"n": 4_000_000, "margin": None, "bytes": 670.0e6, "tuning": {"integrate_staged": 0},
         "source": [("pipeline.cuh", "k_integrate(Dev<F> d)", "2a86d66be349aff5")] + _INTEGRATE_SOURCE},
        {"n": 4_000_000, "margin": None, "bytes": 665.4e6, "tuning": {"integrate_staged": 1},
         "source": [("pipeline.cuh", "k_integrate_staged(Dev<FormF32> d)", "a2d764678f9b801a"),
                    ("pipeline.cuh", "struct StageLayout {", "a4f1f17d327f7a13")] + _INTEGRATE_SOURCE},
    ],
    "contact": [
        {"n": 4_000_000, "margin": 2.1e-5, "bytes": 331.4e6, "tuning": {"contact_lean": 0, "contact_screen": 0},
         "source": [("pipeline.cuh", "k_contact(Dev<F> d, double *eval_F, double *eval_T)", "36e10c0e4e38a6ea"),
                    ("pipeline.cuh", "contact_slot(const Dev<F> &d", "363d4cb673f86026"),
                    ("pipeline.cuh", "pair_sums(const Dev<F> &d", "de27f25f313b3b49"),
                    ("pipeline.cuh", "wall_contact(const Dev<F> &d", "54458541bf779dd2"),
                    ("pipeline.cuh", "sphere_gap(const Dev<F> &d", "64de1a81d6ab41e3"),
                    ("pipeline.cuh", "sphere_finish(const Dev<F> &d", "3fde901e334f3796"),
                    ("pipeline.cuh", "load_sphere_pos(const Dev<F> &d", "f767f41ecac8ae6a"),
                    ("pipeline.cuh", "load_sphere(const Dev<F> &d", "e464faf6f6eeda0b"),
                    ("common.cuh", "struct FormF32 {", "02359980dafed2e7")]},
        # the two-pass contact step: both kernels of one step (the contact phase's time
        # covers both)
        {"n": 4_000_000, "margin": 3.0e-5, "bytes": 422.9e6, "tuning": {"contact_screen": 1},
         "source": [("pipeline.cuh", "k_contact_screen(Dev<F> d)", "eee7a70e82cd02b0"),
                    ("pipeline.cuh", "k_contact_eval(Dev<F> d)", "7cb6d5353d4b1f84"),
                    ("pipeline.cuh", "pair_sums(const Dev<F> &d", "c91a142e9d5d3105"),
                    ("pipeline.cuh", "wall_contact(const Dev<F> &d", "54458541bf779dd2"),
                    ("pipeline.cuh", "sphere_gap(const Dev<F> &d", "64de1a81d6ab41e3"),
                    ("pipeline.cuh", "sphere_finish(const Dev<F> &d", "3fde901e334f3796"),
                    ("pipeline.cuh", "load_sphere_pos(const Dev<F> &d", "f767f41ecac8ae6a"),
                    ("pipeline.cuh", "load_sphere(const Dev<F> &d", "e464faf6f6eeda0b"),
                    ("common.cuh", "struct FormF32 {", "02359980dafed2e7")]},
    ],
}


def kernel_source_hash(signature, fname="pipeline.cuh"):
    """Hash of the definition of the function whose text starts with signature (forward
    declarations, which end at a semicolon before any brace, are skipped)."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2311_04648_gb300", "csrc", fname)) as f:
        src = f.read()
    i = src.find(signature)
    while i >= 0:
        semi, brace = src.find(";", i), src.find("{", i)
        if brace >= 0 and (semi < 0 or brace < semi):
            j = src.index("\n}", i)
            return hashlib.sha1(src[i:j].encode()).hexdigest()[:16]
        i = src.find(signature, i + 1)
    return None


def measured_traffic(kernel, n, margin=None, tuning=None):
    """The recorded DRAM bytes per launch of `kernel` for a run of n owners at `margin` with
    `tuning`, from the record whose capture matches: the same size, the same kernel build
    (tuning fields such as staged integration or the lean contact kernel), for the contact
    kernel the same margin, and kernel source that still hashes to the captured one;
    None if no record matches."""
    for t in MEASURED_TRAFFIC.get(kernel, []):
        if t["n"] != n:
            continue
        if any((tuning or {}).get(k, v) != v for k, v in t.get("tuning", {}).items()):
            continue
        if t["margin"] is not None and (margin is None or abs(margin - t["margin"]) > 1e-6 * t["margin"]):
            continue
        if any(kernel_source_hash(sig, fn) != hv for fn, sig, hv in t["source"]):
            continue
        return t["bytes"]
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def device_copy_gbs(device, nbytes=2 << 30, reps=5):
    """This GPU's own device-to-device copy bandwidth (read + write bytes per second) with
    a torch copy, for reading the run against the machine's measured peak: GPUs of a pool
    differ."""
    import torch
    a = torch.empty(nbytes // 4, dtype=torch.float32, device=f"cuda:{device}")
    b = torch.empty_like(a)
    b.copy_(a)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record()
        b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * nbytes / (e0.elapsed_time(e1) / 1000.0) / 1e9)
    del a, b
    torch.cuda.empty_cache()
    return best


# ----------------------------------------------------------------------------- runs

def make_scene(n):
    from paper_2311_04648_gb300 import workloads as W
    return W.settling_column(n=n)


def profile_delta(p0, p1):
    nf = p1["n_force"] - p0["n_force"]
    ni = p1["n_integrate"] - p0["n_integrate"]
    nd = p1["n_detect"] - p0["n_detect"]
    ne = p1.get("n_contact_eval", 0) - p0.get("n_contact_eval", 0)
    return dict(contact_ms=(p1["ms_force"] - p0["ms_force"]) / max(nf, 1), n_contact=nf,
                # the two-pass contact step: its evaluation pass, within contact_ms
                eval_ms=(p1.get("ms_contact_eval", 0.0) - p0.get("ms_contact_eval", 0.0)) / max(ne, 1), n_eval=ne,
                integrate_ms=(p1["ms_integrate"] - p0["ms_integrate"]) / max(ni, 1), n_integrate=ni,
                detect_ms=(p1["ms_detect"] - p0["ms_detect"]) / max(nd, 1), n_detect=nd,
                hash_ms=(p1["ms_hash"] - p0["ms_hash"]) / max(nd, 1),
                link_ms=(p1["ms_link"] - p0["ms_link"]) / max(nd, 1),
                # per-step averages over the profiled steps (the contact count grows as the
                # column settles)
                listed_pairs=(p1["pair_steps"] - p0["pair_steps"]) / max(p1["steps"] - p0["steps"], 1),
                with_entries=(p1["busy_steps"] - p0["busy_steps"]) / max(p1["steps"] - p0["steps"], 1),
                listed_pairs_end=p1["listed_pairs"], with_entries_end=p1["spheres_with_entries"],
                active_contacts=p1["active_contacts"], list_capacity=p1["list_capacity"])


KERNEL_NAMES = {"contact": "k_contact (pair forces + per-owner sums)",
                "integrate": "k_integrate (owner update + audit)",
                "step": "k_step_fused (pair forces summed in registers + owner update + audit)",
                "detect": "detection phase (k_hash, radix sort, k_cellstart, k_narrow, k_link)"}


def fused_step(prof):
    """True when the profiled steps ran the fused kernel (no separate integration)."""
    return prof["n_integrate"] == 0 and prof["n_contact"] > 0


def roofline(precision, n, prof, peak, peak_kind, margin=None, rebuilds_per_step=0.0, contact_integrates=False,
             derived=False, tuning=None):
    """Roofline of the dominant kernel of a step (largest share of the step's time) and of
    each per-step kernel and the detection phase on its own: algorithmic bytes per
    launch over the average launch duration (CUDA events on the kernel's own stream)."""
    ci = bool(contact_integrates) and not fused_step(prof)
    ab = algorithmic_bytes(precision, n, prof["listed_pairs"], n_with_entries=prof["with_entries"],
                           contact_integrates=ci)
    lb = layout_bytes(precision, n, prof["with_entries"], prof["listed_pairs"], contact_integrates=ci,
                      derived=derived)
    per = {}
    for k in (("step",) if fused_step(prof) else ("contact", "integrate")):
        ms = prof["contact_ms" if k == "step" else f"{k}_ms"]
        sec = ms / 1000.0
        per[k] = {"ms": ms, "ms_per_step": ms, "bytes": ab[k], "gbs": ab[k] / sec / 1e9 if ms > 0 else None,
                  "moved_bytes": lb[k], "moved_gbs": lb[k] / sec / 1e9 if ms > 0 else None}
    if prof["n_detect"] > 0 and prof["detect_ms"] > 0:
        db = detection_bytes(precision, n, prof["listed_pairs"])
        dms = prof["detect_ms"]
        per["detect"] = {"ms": dms, "ms_per_step": dms * rebuilds_per_step, "bytes": db,
                         "gbs": db / (dms / 1000.0) / 1e9, "moved_bytes": None, "moved_gbs": None,
                         "what": "one list rebuild: hash, sort passes, cell table, narrow phase, history link"}
    for k, v in per.items():
        v["frac"] = (v["gbs"] / peak) if v["gbs"] else None
        v["traffic"] = (measured_traffic(k, n, margin, tuning) if precision == "voxel_fp32" and k in MEASURED_TRAFFIC
                        and not ci else None)
    # the dominant kernel: the single kernel with the largest share of the step (the
    # detection phase is several kernels on the second stream, reported beside them).  The
    # contact phase of the two-pass step is two kernels: its longer pass is what competes
    single = {k: per[k]["ms_per_step"] for k in per if k != "detect"}
    if prof.get("n_eval", 0) > 0 and "contact" in per:
        ev = prof["eval_ms"]
        sc = max(per["contact"]["ms"] - ev, 0.0)
        per["contact"]["passes"] = {"k_contact_screen_ms": sc, "k_contact_eval_ms": ev}
        single["contact"] = max(sc, ev)
    dom = max(single, key=single.get)
    a = per[dom]["gbs"]
    name = KERNEL_NAMES[dom]
    if ci:
        name = {"contact": "k_contact (pair forces + per-owner sums + update of the owners with partners)",
                "integrate": "k_integrate (update of the owners without partners + audit)"}.get(dom, name)
    screen = bool((tuning or {}).get("contact_screen", 0)) and not ci and not fused_step(prof)
    if screen:
        name = {"contact": "k_contact_screen + k_contact_eval (overlap screening of every listed entry, then "
                           "pair forces + per-owner sums of the spheres with touching entries)"}.get(dom, name)
    return {"bound": "hbm", "kernel": name, "contact_integrates": ci, "contact_screen": screen,
            "achieved": a, "peak": peak, "unit": "GB/s", "frac": (a / peak) if a else None,
            "traffic": per[dom]["traffic"],
            "peak_kind": peak_kind, "bytes_per_launch": per[dom]["bytes"], "avg_launch_ms": per[dom]["ms"],
            "moved_frac": (per[dom]["moved_gbs"] / peak) if per[dom]["moved_gbs"] else None,
            "kernels": per, "listed_pairs": prof["listed_pairs"], "spheres_with_entries": prof["with_entries"]}


def parse_tuning(text):
    """'name=value,...' of --set-tuning as keyword arguments of World.set_tuning."""
    kw = {}
    for item in text.split(","):
        k, v = item.split("=")
        kw[k.strip()] = float(v) if k.strip() in ("cell_factor", "margin") else int(v)
    return kw


def run_ours(args, device):
    import torch
    from paper_2311_04648_gb300 import dem

    torch.cuda.set_device(device)
    scene = make_scene(args.n)
    out = {}

    def timed(world, steps, label):
        stream = torch.cuda.ExternalStream(world.stream(), device=device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        # the NVTX range lets a profiler keep only the timed launches
        torch.cuda.nvtx.range_push(label)
        e0.record(stream)
        world.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return e0.elapsed_time(e1)

    # chosen form: voxel + FP32, delayed detection on the second stream, audited.  The
    # timed window lies inside the configuration's steps: it starts where the autotuner
    # tunes (mid-run, after the column has closed many lattice gaps) when the warm-up and
    # the timed steps fit after it, else as late as they fit, so that a short run times a
    # state in contact, not the contact-free initial lattice
    w = dem.World.from_scene(scene, precision="voxel_fp32", schedule="velocity_bound", device=device)
    start_at = args.window_start
    if start_at < 0:
        start_at = min(args.tune_at, max(0, args.config_steps - args.steps - args.warmup))
    out["window_start"] = start_at
    if args.tune_steps > 0:
        if start_at == args.tune_at:
            w.step(args.tune_at)
            out["tuning"] = w.autotune(steps=args.tune_steps, cache_path=args.tune_cache)
        else:
            start = w.save_state()
            w.step(args.tune_at)
            out["tuning"] = w.autotune(steps=args.tune_steps, cache_path=args.tune_cache)
            w.load_state(start)
            del start
            w.step(start_at)
    else:
        w.step(start_at)
        out["tuning"] = w.tuning()
    if args.set_tuning:
        w.set_tuning(**parse_tuning(args.set_tuning))
        out["tuning"] = w.tuning()
    # the state at the start of the warm-up, for the plain form's run from the same state
    window_state = w.owner_state()
    window_contacts = w.contacts()
    # the clock sampler covers the warm-up, the timed steps and the profiled pass over
    # the same steps (nvidia-smi samples every 50 ms: a short timed region alone may fall
    # between two samples)
    with ClockSampler(device) as clk:
        time.sleep(0.2)
        w.step(args.warmup)
        after_warmup = w.save_state()
        s0 = w.stats()
        ms = timed(w, args.steps, "timed_chosen")
        s1 = w.stats()
        steps = s1["steps"] - s0["steps"]
        rebuilds = s1["rebuilds"] - s0["rebuilds"]
        # profiled pass over the same steps (restored from the checkpoint) for per-kernel
        # durations: events on each kernel's own stream
        end_state = w.save_state()
        w.load_state(after_warmup)
        w.set_profiling(True)
        p0 = w.stats()
        w.step(args.steps)
        p1 = w.stats()
        w.set_profiling(False)
        time.sleep(0.2)
    out["chosen"] = dict(ms=ms, steps=steps, rebuilds=rebuilds, clocks=clk.summary(), stats=s1,
                         fallbacks=s1["audit_fallbacks"] - s0["audit_fallbacks"],
                         first_step=s0["steps"], contacts=(s0["active_contacts"], s1["active_contacts"]))
    out["profile"] = profile_delta(p0, p1)
    w.load_state(end_state)
    del after_warmup, end_state
    out["copy_gbs"] = device_copy_gbs(device)
    # e2e through the C ABI with host buffers: state in from pinned memory, one step,
    # state out to pinned memory, every step
    n_own = scene.n_owner
    pin = {k: torch.empty(shape, dtype=torch.float64).pin_memory() for k, shape in
           (("x", (n_own, 3)), ("q", (n_own, 4)), ("v", (n_own, 3)), ("w", (n_own, 3)))}
    arrs = {k: t.numpy() for k, t in pin.items()}
    x, q, v, wb = w.owner_state()
    arrs["x"][:] = x; arrs["q"][:] = q; arrs["v"][:] = v; arrs["w"][:] = wb
    import ctypes as C
    L = w.L

    def e2e_step():
        w.set_owner_state(0, xyz=arrs["x"], quat=arrs["q"], vel=arrs["v"], omega=arrs["w"])
        w.step(1)
        st = L.dem_get_owner_state(w.h, 0, n_own, arrs["x"].ctypes.data_as(C.c_void_p),
                                   arrs["q"].ctypes.data_as(C.c_void_p), arrs["v"].ctypes.data_as(C.c_void_p),
                                   arrs["w"].ctypes.data_as(C.c_void_p))
        assert st == 0

    # untimed warm-up: the checkpoint restore above makes the first step rebuild the list,
    # and the first upload sizes its scratch
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
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
        # the same state as the chosen form's window (positions, orientations, velocities
        # and the tangential history of its contacts)
        x, q, v, wb = window_state
        wp.set_owner_state(0, xyz=x, quat=q, vel=v, omega=wb)
        wp.step(0)
        wp.set_history(window_contacts["i"], window_contacts["j"], window_contacts["history"])
        del window_state, window_contacts
        wp.step(3)
        p0 = wp.stats()
        msp = timed(wp, args.plain_steps, "timed_plain")
        p1 = wp.stats()
        wp.set_profiling(True)
        q0 = wp.stats()
        wp.step(5)
        q1 = wp.stats()
        out["plain"] = dict(ms=msp, steps=p1["steps"] - p0["steps"], profile=profile_delta(q0, q1))
        wp.close()
    return out


def run_scale(args, device, rank=0, world=1):
    """The other configurations at full size, one JSON line each (not the headline):
    drum   -- 20M rods and tetrahedra (~70M spheres) in a drum spinning at 1 rad/s;
    hopper -- 10M spheres in a 30-degree conical hopper with a sink: the learned schedule
              (network trained on trajectories of the 2k-sphere box and a 1M-sphere
              section of the settling column) against the velocity-bound and every-step
              schedules, all audited;
    batch  -- 512 column collapses of 1k-50k spheres in one engine, autotuned on the state
              after half the timed steps (then restored to the start); with N
              ranks the scenes are split by greedy bin packing on spheres x steps and
              each rank steps its share as one batch (no exchange until the end)."""
    import torch
    from paper_2311_04648_gb300 import dem
    from paper_2311_04648_gb300 import workloads as W

    torch.cuda.set_device(device)

    def timed(step_fn, stream_ptr, steps, label):
        stream = torch.cuda.ExternalStream(stream_ptr, device=device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(label)
        e0.record(stream)
        step_fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return e0.elapsed_time(e1)

    steps = args.steps
    out = {"workload": args.workload}
    t0 = time.perf_counter()
    if args.workload == "drum":
        scene = W.clump_drum(n_clumps=args.n if args.n != 4_000_000 else 20_000_000)
        w = dem.World.from_scene(scene, precision="voxel_fp32", schedule="velocity_bound", device=device)
        out["setup_s"] = time.perf_counter() - t0
        out["tuning"] = w.autotune(steps=args.tune_steps, cache_path=args.tune_cache) if args.tune_steps > 0 else w.tuning()
        if args.set_tuning:
            w.set_tuning(**parse_tuning(args.set_tuning))
            out["tuning"] = w.tuning()
        w.step(args.warmup)
        s0 = w.stats()
        with ClockSampler(device) as clk:
            ms = timed(w.step, w.stream(), steps, "timed_drum")
        s1 = w.stats()
        n_sph = scene.n_sphere
        out.update(n_spheres=n_sph, n_clumps=scene.n_owner, ms=ms, steps=steps, clocks=clk.summary(),
                   rebuilds=s1["rebuilds"] - s0["rebuilds"], fallbacks=s1["audit_fallbacks"] - s0["audit_fallbacks"],
                   listed_pairs=s1["listed_pairs"], contacts=s1["active_contacts"],
                   value=n_sph * steps / (ms / 1000.0), drum_length_m=scene.meta.get("length"))
        w.close()
    elif args.workload == "hopper":
        # train on the method's own trajectories of the first two configurations
        teach = [W.settle_box(n=2000, vel_sigma=0.3, seed=2), W.settling_column(n=1_000_000)]
        blob = None
        tw = None
        for k, sc in enumerate(teach):
            tw = dem.World.from_scene(sc, precision="voxel_fp32", schedule="velocity_bound", device=device)
            if blob is not None:
                tw.load_schedule_model(blob)
            tw.schedule_collect(True)
            tw.step(2048 if k == 0 else 1536)
            tw.schedule_collect(False)
            out[f"train_samples_{k}"] = tw.stats()["schedule_samples"]
            out[f"train_loss_{k}"] = tw.schedule_train(epochs=60, lr=3e-3, seed=1)
            blob = tw.schedule_export()
            tw.close()
        scene = W.cone_hopper(n=args.n if args.n != 4_000_000 else 10_000_000)
        n_sph = scene.n_sphere
        out["setup_s"] = time.perf_counter() - t0
        res = {}
        for sched in ("learned", "velocity_bound", "every_step"):
            w = dem.World.from_scene(scene, precision="voxel_fp32", schedule=sched, device=device,
                                     margin=None if sched == "every_step" else 6e-5, margin_max=6e-5)
            if sched == "learned":
                w.load_schedule_model(blob)
            if args.set_tuning:
                w.set_tuning(**parse_tuning(args.set_tuning))
            out[f"tuning_{sched}"] = w.tuning()
            w.step(args.warmup)
            s0 = w.stats()
            k = steps if sched != "every_step" else max(1, min(steps, args.plain_steps))
            ms = timed(w.step, w.stream(), k, f"timed_hopper_{sched}")
            s1 = w.stats()
            res[sched] = dict(value=n_sph * k / (ms / 1000.0), steps=k, ms=ms,
                              rebuilds=s1["rebuilds"] - s0["rebuilds"],
                              fallbacks=s1["audit_fallbacks"] - s0["audit_fallbacks"])
            w.close()
        out.update(n_spheres=n_sph, steps=steps, schedules=res, value=res["learned"]["value"],
                   ms=res["learned"]["ms"])
    elif args.workload == "mixer":
        # Sec. 5's bladed mixer: 2,892 facets turning at 2 pi rad/s, elements released from
        # rest above it, dt = 5e-7 s
        scene = W.mixer(n=args.n if args.n != 4_000_000 else 2_000_000, clump=args.clump, start=args.mixer_start)
        w = dem.World.from_scene(scene, precision="voxel_fp32", schedule="velocity_bound", device=device)
        out["setup_s"] = time.perf_counter() - t0
        out["tuning"] = w.autotune(steps=args.tune_steps, cache_path=args.tune_cache) if args.tune_steps > 0 else w.tuning()
        if args.set_tuning:
            w.set_tuning(**parse_tuning(args.set_tuning))
            out["tuning"] = w.tuning()
        w.step(args.warmup)
        s0 = w.stats()
        with ClockSampler(device) as clk:
            ms = timed(w.step, w.stream(), steps, "timed_mixer")
        s1 = w.stats()
        n_sph = scene.n_sphere
        out.update(n_spheres=n_sph, n_elements=scene.n_owner, clump=args.clump, start=args.mixer_start, facets=2892,
                   ms=ms, steps=steps,
                   clocks=clk.summary(), rebuilds=s1["rebuilds"] - s0["rebuilds"],
                   fallbacks=s1["audit_fallbacks"] - s0["audit_fallbacks"], listed_pairs=s1["listed_pairs"],
                   wall_pairs=s1["wall_pairs"], contacts=s1["active_contacts"],
                   value=n_sph * steps / (ms / 1000.0), element_radius_m=scene.meta["element_radius"])
        w.close()
    elif args.workload == "batch":
        from paper_2311_04648_gb300 import shard
        all_scenes = W.batch_scenes(512)
        parts = shard.assign([sc.n_sphere for sc in all_scenes], world)
        scenes = [all_scenes[k] for k in parts[rank]]
        out["n_spheres_total"] = int(sum(sc.n_sphere for sc in all_scenes))
        b = dem.Batch(scenes, precision="voxel_fp32", schedule="velocity_bound", device=device)
        b.initialize()
        out["setup_s"] = time.perf_counter() - t0
        w0 = b.worlds[0]
        # tuned on a state in contact (the collapses under way at the tuning step), then
        # restored to the start: trials from the initial state favour shapes that lose
        # once contacts develop
        if args.tune_steps > 0:
            start = w0.save_state()
            b.step(min(args.tune_at, max(0, steps // 2)))
            out["tuning"] = w0.autotune(steps=args.tune_steps, cache_path=args.tune_cache)
            w0.load_state(start)
            del start
        else:
            out["tuning"] = w0.tuning()
        if args.set_tuning:
            w0.set_tuning(**parse_tuning(args.set_tuning))
            out["tuning"] = w0.tuning()
        b.step(args.warmup)
        s0 = w0.stats()
        with ClockSampler(device) as clk:
            ms = timed(b.step, w0.stream(), steps, "timed_batch")
        s1 = w0.stats()
        n_sph = int(sum(sc.n_sphere for sc in scenes))
        out.update(n_spheres=n_sph, n_scenes=len(scenes), ms=ms, steps=steps, clocks=clk.summary(),
                   rebuilds=s1["rebuilds"] - s0["rebuilds"], value=n_sph * steps / (ms / 1000.0))
        b.close()
    return out


def cpu_baseline(args, max_steps=None):
    """The oracle as it stands on the host cores, on bounded samples of the workload:

    value  -- the oracle's own O(N^2) contact search (the default mode), OpenMP over
              spheres on every host core, on the 20,000-sphere sub-box of the settling
              column (the same generator restricted to a 0.03 m central column), stepped
              from the lattice until ~args.cpu_sample_seconds have passed;
    cell_list      -- the same sub-box with the oracle's grid candidate enumeration (the
                      faster variant: the same contacts in the same order), all cores,
                      up to 500 steps;
    single_thread  -- the grid variant on one thread;
    c1_full        -- the 2,000-sphere box (seed 1, from rest) for its full 2,000 steps,
                      O(N^2) search on all cores.
    The oracle's threads find contacts in parallel and reduce them serially in the
    serial order, so every variant computes the same trajectory bits."""
    import oracle
    from paper_2311_04648_gb300 import workloads as W

    threads = max(1, os.cpu_count() or 1)
    sub = W.settling_column(n=args.cpu_sample_n, column_width=0.03)

    def rate(scene, cell_list, th, steps_cap, seconds):
        ow = oracle.OracleWorld(scene, cell_list=cell_list, threads=th)
        assert ow.step(1) == 0
        t0 = time.perf_counter()
        k = 0
        while k < steps_cap and (k == 0 or time.perf_counter() - t0 < seconds):
            assert ow.step(1) == 0
            k += 1
        dt = time.perf_counter() - t0
        return {"value": scene.n_sphere * k / dt, "steps": k, "seconds": dt, "threads": th}

    cap = 10 ** 9 if max_steps is None else max_steps
    brute = rate(sub, False, threads, cap, args.cpu_sample_seconds)
    out = {"value": brute["value"], "unit": METRIC, "cores": threads, "kind": "oracle",
           "sample": f"{sub.n_sphere}-sphere sub-box of the settling column (0.03 m central column), "
                     f"{brute['steps']} steps in {brute['seconds']:.1f} s from the lattice, O(N^2) contacts, "
                     f"{threads} OpenMP threads"}
    if max_steps is None:
        grid = rate(sub, True, threads, 500, 30.0)
        one = rate(sub, True, 1, 500, 4.0)
        c1 = W.settle_box(n=2000, seed=1)
        ow = oracle.OracleWorld(c1, threads=threads)
        t0 = time.perf_counter()
        assert ow.step(2000) == 0
        dt = time.perf_counter() - t0
        out.update(cell_list=grid, single_thread=one,
                   c1_full={"value": 2000 * 2000 / dt, "steps": 2000, "seconds": dt, "threads": threads,
                            "what": "2,000 spheres from rest in the 40x40x80 mm box, dt = 1e-6 s, FP64, "
                                    "O(N^2) contacts every step"},
                   max_threads_openmp=oracle.max_threads())
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        # the oracle on the host cores, one oracle step per step of the sub-box sample;
        # the warm-up and the timed steps are capped so that the run ends within minutes
        import oracle
        from paper_2311_04648_gb300 import workloads as W
        threads = max(1, os.cpu_count() or 1)
        sub = W.settling_column(n=args.cpu_sample_n, column_width=0.03)
        ow = oracle.OracleWorld(sub, threads=threads)
        for _ in range(min(args.warmup, 3)):
            assert ow.step(1) == 0
        t0 = time.perf_counter()
        k = 0
        while k < args.steps and (k == 0 or time.perf_counter() - t0 < 90.0):
            assert ow.step(1) == 0
            k += 1
        dt = time.perf_counter() - t0
        value = sub.n_sphere * k / dt
        sample = (f"{sub.n_sphere}-sphere sub-box of the settling column (0.03 m central column), {k} of "
                  f"{args.steps} steps timed in {dt:.1f} s, O(N^2) contacts, {threads} OpenMP threads")
        cb = {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample}
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * dt / max(k, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": "settling_column", "n_spheres": args.n, "radius_mm": [0.8, 1.2],
                           "box_m": [0.3, 0.3, 1.2], "dt_s": 2e-6, "precision": "FP64 (the oracle)",
                           "sample": sample},
                "cpu_baseline": cb,
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if args.workload != "column":
        if args.workload != "batch" or world == 1:
            if rank != 0:
                return 0
            r = run_scale(args, local)
            line = {"metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": 1, "steps": r["steps"],
                    "warmup": args.warmup, "ms_per_step": r["ms"] / max(r["steps"], 1), "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                    "config": {"workload": args.workload}, "details": r}
            print(json.dumps(line))
            return 0
        # batch over N ranks: each steps its share of the 512 scenes; the slowest sets the time
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        r = run_scale(args, local, rank, world)
        t = torch.tensor([r["ms"]], device=f"cuda:{local}", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tdist.barrier()
        ms = float(t.item())
        if rank == 0:
            value = r["n_spheres_total"] * r["steps"] / (ms / 1000.0)
            line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": r["steps"],
                    "warmup": args.warmup, "ms_per_step": ms / max(r["steps"], 1), "higher_is_better": True,
                    "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                    "config": {"workload": "batch", "parallelism": f"scenes split over {world} ranks"},
                    "details": r}
            print(json.dumps(line))
        tdist.destroy_process_group()
        return 0
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
                   "timed_window": f"steps {res['chosen']['first_step']}-{res['chosen']['first_step'] + steps} "
                                   f"of the configuration's {args.config_steps} (warm-up from step "
                                   f"{res['window_start']})",
                   "listed_pairs_per_sphere": prof["listed_pairs"] / n_sph,
                   "spheres_with_partners_per_sphere": prof["with_entries"] / n_sph,
                   "contacts_per_sphere": [c / n_sph for c in res["chosen"]["contacts"]],
                   "rebuilds_in_timed_region": res["chosen"]["rebuilds"],
                   "audit_fallbacks_in_timed_region": res["chosen"]["fallbacks"],
                   "device_copy_gbs_this_gpu": res["copy_gbs"],
                   "tuning": res["tuning"],
                   "binning": "counting sort" if res["chosen"]["stats"].get("counting_sort") else "radix sort",
                   "owner_constants": ("1/m and 1/I derived from mass and radius"
                                       if res["chosen"]["stats"].get("derived_constants") else "read per owner"),
                   "l2": "inputs larger than L2 (owner state + contact lists > 0.5 GB)",
                   "parallelism": f"replica x{world}"},
        "roofline": roofline("voxel_fp32", n_sph, prof, peak, peak_kind, margin=res["chosen"]["stats"]["margin"],
                             rebuilds_per_step=res["chosen"]["rebuilds"] / max(steps, 1),
                             contact_integrates=res["tuning"].get("contact_integrates", 0),
                             derived=bool(res["chosen"]["stats"].get("derived_constants", 0)), tuning=res["tuning"]),
        "kernels_ms": dict(({"step": prof["contact_ms"]} if fused_step(prof) else
                            {"contact": prof["contact_ms"], "integrate": prof["integrate_ms"]}),
                           detect_per_rebuild=prof["detect_ms"], hash=prof["hash_ms"], link=prof["link_ms"]),
        "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": e2e["bytes_in"],
                "d2h_bytes_per_step": e2e["bytes_out"],
                "how": "dem_set_owner_state from pinned host buffers + dem_step(1) + dem_get_owner_state "
                       "to pinned host buffers, every step"},
        "gpu_launches": int((2 if fused_step(prof) else 3) * steps + 20 * res["chosen"]["rebuilds"]),
        "clocks": res["chosen"]["clocks"],
    }
    if plain:
        pv = n_sph * plain["steps"] / (plain["ms"] / 1000.0) * world
        pp = plain["profile"]
        line["plain"] = {"value": pv, "unit": METRIC, "ms_per_step": plain["ms"] / max(plain["steps"], 1),
                         "dtype": "f64", "schedule": "every step",
                         "kernels_ms": dict(({"step": pp["contact_ms"]} if fused_step(pp) else
                                             {"contact": pp["contact_ms"], "integrate": pp["integrate_ms"]}),
                                            detect=pp["detect_ms"]),
                         "roofline": roofline("fp64", n_sph, pp, peak, peak_kind, rebuilds_per_step=1.0),
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
