"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU oracle.

Bars: contact sets bit-exact (same predicate, same positions); FP64 plain form within
1e-9 relative on forces and states (relative to the scale of the summed terms); the
voxel + FP32 form within 1e-4 on per-contact forces (error normalised by
max(|F64|, 1e-3 median |F64|)); schedules and batching bit-identical to the plain run.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_2311_04648_gb300 import dem, workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def dense_scene(n=1200, seed=3, vel=0.2, e=0.5, mu=0.4, h=1e-6):
    return W.dense_lattice(n=n, seed=seed, vel_sigma=vel, e=e, mu=mu, h=h)


def rel_err(a, b, scale):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / scale))


def owner_scale(ow, cs, F):
    """Per-owner scale: sum of |contact force| plus |m g| (the terms the sums add)."""
    sc = np.abs(ow.mass)[:, None] * 9.81 * np.ones((1, 3))
    for c in cs:
        oi = ow.owner[c["i"]]
        sc[oi] += np.abs(c["force"])
        if c["j"] >= 0:
            sc[ow.owner[c["j"]]] += np.abs(c["force"])
    return sc + 1e-300


def torque_scale(ow, cs):
    sc = np.zeros((ow.n_owner, 3)) + 1e-300
    for c in cs:
        for side, sgn in ((c["i"], 1.0), (c["j"], -1.0)):
            if side < 0:
                continue
            o = ow.owner[side]
            arm = np.abs(np.array(c["point"]) - ow.x[o])
            sc[o] += np.linalg.norm(arm) * np.abs(c["force"]).max() * np.ones(3)
    return sc


# ----------------------------------------------------------------------------- radix sort

@pytest.mark.parametrize("n,bits", [(0, 8), (1, 8), (1000, 13), (4096 * 3 + 17, 23), (300_000, 32), (65_537, 9)])
def test_radix_sort_is_a_stable_sort(n, bits):
    rng = np.random.default_rng(n + bits)
    hi = 1 << bits if bits < 32 else 1 << 32
    keys = rng.integers(0, min(hi, 1 << 32), size=n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 3] = keys[0]                   # many equal keys
    vals = np.arange(n, dtype=np.uint32)
    ko, vo = dem.radix_sort_u32(keys, vals, bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(ko, keys[order])
    assert np.array_equal(vo, vals[order])


# ----------------------------------------------------------------------------- contact sets

@pytest.mark.parametrize("precision", ["fp64", "voxel_fp32"])
def test_listed_sets_bit_exact(precision):
    s = dense_scene(n=1500, seed=4)
    beta = 4e-5
    w = dem.World.from_scene(s, precision=precision, margin=beta)
    ow = oracle.OracleWorld(s)
    gi, gj = w.listed_pairs()
    assert len(gi) > 1000
    if precision == "fp64":
        p, r = w.sphere_positions()
        oi, oj = oracle.listed_pairs_f64(p, r, ow.owner, beta)
        ow.rad[:] = r
    else:
        cell, off, L = w.sphere_voxels()
        _, r = w.sphere_positions()
        oi, oj = oracle.listed_pairs_voxel_f32(cell, off, np.float32(L), r.astype(np.float32), ow.owner,
                                               np.float32(beta))
        lo = np.asarray(s.box_lo)
        p = (lo + cell.astype(np.float64) * L) + off.astype(np.float64)
        ow.rad[:] = r.astype(np.float32).astype(np.float64)
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    si, wi = w.listed_wall_pairs()
    osi, owi = ow.listed_wall_pairs(p, beta)
    assert len(si) > 10
    assert np.array_equal(si, osi) and np.array_equal(wi, owi)


def test_listed_sets_bit_exact_for_clumps():
    s = W.packed_clumps(n=150, seed=5)
    beta = 5e-5
    w = dem.World.from_scene(s, precision="fp64", margin=beta)
    ow = oracle.OracleWorld(s)
    p, r = w.sphere_positions()
    po = ow.sphere_positions()
    assert np.max(np.abs(p - po)) == 0.0       # same exactly rounded formula on both sides
    gi, gj = w.listed_pairs()
    oi, oj = oracle.listed_pairs_f64(p, r, ow.owner, beta)
    assert len(gi) > 50
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)


# ----------------------------------------------------------------------------- forces

def compare_contacts(w, ow, tol):
    gc = w.contacts()
    F, T, oc = ow.eval()
    assert np.array_equal(gc["i"], oc["i"]) and np.array_equal(gc["j"], oc["j"])
    fs = np.abs(oc["force"]).max(axis=1, keepdims=True) + 1e-300
    assert rel_err(gc["force"], oc["force"], fs) < tol
    assert rel_err(gc["overlap"], oc["overlap"], oc["overlap"]) < tol * 1e3   # small differences of O(R)
    assert rel_err(gc["point"], oc["point"], 1e-3) < tol
    hs = np.abs(oc["ut"]).max(axis=1, keepdims=True) + 1e-20
    assert rel_err(gc["history"], oc["ut"], hs) < tol * 1e3
    return gc, oc


def test_fp64_forces_match_oracle_at_initial_and_later_states():
    s = dense_scene(n=800, seed=6)
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s)
    for rnd in range(3):
        gc, oc = compare_contacts(w, ow, TOL64)
        assert len(oc) > 200
        Fg, Tg = w.owner_forces()
        Fo, To, _ = ow.eval()
        assert rel_err(Fg, Fo, owner_scale(ow, oc, Fo)) < TOL64
        assert rel_err(Tg, To, torque_scale(ow, oc)) < TOL64
        w.step(25)
        ow.step(25)


def state_close(w, ow, tol):
    x, q, v, wb = w.owner_state()
    ext = float(np.max(np.abs(ow.x))) + 1e-300
    vs = float(np.max(np.abs(ow.v))) + 1e-300
    ws = float(np.max(np.abs(ow.wb))) + 1e-300
    errs = dict(x=rel_err(x, ow.x, ext), v=rel_err(v, ow.v, vs), w=rel_err(wb, ow.wb, ws),
                q=rel_err(q * np.sign(q[:, :1] + 1e-300), ow.q * np.sign(ow.q[:, :1] + 1e-300), 1.0))
    return errs, max(errs.values()) < tol


def oracle_threads():
    return max(1, os.cpu_count() or 1)


def sync_oracle_to_gpu(w, ow, stored):
    """Put the oracle at the GPU's current state: the owner state, and as the stored
    tangential history the updated history the GPU reported one step earlier
    (``stored``: ``dem.World.contacts`` of the previous state, None at the start).
    Owners the sink removed stay removed on both sides (the oracle's own flags; the GPU
    reports zero velocities for them)."""
    x, q, v, wb = w.owner_state()
    gone = ow.active == 0
    assert np.all(v[gone] == 0.0) and np.all(wb[gone] == 0.0)
    ow.x[:] = x
    ow.q[:] = q
    ow.v[:] = v
    ow.wb[:] = wb
    if stored is None:
        ow.set_history(np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3)))
    else:
        ow.set_history(stored["i"], stored["j"], stored["history"], age=stored.get("age"))


def one_step_parity(w, ow, stored, tol=TOL64, rolling=False):
    """From the GPU's own state: every contact's force, overlap, point and updated
    history, the per-owner force and torque sums, and the state after one step, against
    the oracle at 1e-9 (forces per contact relative to its largest component; overlaps
    relative to the largest radius; histories relative to the largest history; sums
    relative to the summed magnitudes).  Returns the largest errors and the contacts."""
    sync_oracle_to_gpu(w, ow, stored)
    gc = w.contacts()
    Fo, To, oc = ow.eval()
    assert np.array_equal(gc["i"], oc["i"]) and np.array_equal(gc["j"], oc["j"])
    fs = np.abs(oc["force"]).max(axis=1, keepdims=True) + 1e-300
    hs = max(float(np.max(np.abs(oc["ut"]))) if len(oc) else 0.0, 1e-300)
    Fg, Tg = w.owner_forces()
    if rolling:
        age, trf = w.contact_rolling()
        # the contact's age after this step's update: the same FP64 additions on both sides
        assert np.array_equal(age, oc["age"])
        assert rel_err(trf, oc["torque_force"], fs) < tol if len(oc) else True
        one_step_parity.rolling_on = int(np.sum(np.any(oc["torque_force"] != 0, axis=1))) if len(oc) else 0
    errs = dict(force=rel_err(gc["force"], oc["force"], fs) if len(oc) else 0.0,
                overlap=rel_err(gc["overlap"], oc["overlap"], float(np.max(ow.rad))) if len(oc) else 0.0,
                point=rel_err(gc["point"], oc["point"], 1e-3) if len(oc) else 0.0,
                history=rel_err(gc["history"], oc["ut"], hs) if len(oc) else 0.0,
                F=rel_err(Fg, Fo, owner_scale(ow, oc, Fo)), T=rel_err(Tg, To, torque_scale(ow, oc)))
    assert max(errs.values()) < tol, errs
    w.step(1)
    assert ow.step(1) == 0
    st, ok = state_close(w, ow, tol)
    assert ok, st
    errs.update(st)
    return errs, len(oc)


ONE_STEP_SCENES = {
    # name: (scene, free-running steps between the one-step checks)
    "dense_polydisperse": (lambda: dense_scene(n=600, seed=8, vel=0.5), (50, 100, 200)),
    "clumps_walls_gravity": (lambda: W.packed_clumps(n=150, seed=10), (100, 200)),
    "spinning_drum": (lambda: W.drum_bed(n=120, seed=1), (300, 700)),
    "cone_hopper_sink": (lambda: W.cone_bed(n=300, seed=13), (300, 600)),
}


@pytest.mark.parametrize("name", sorted(ONE_STEP_SCENES))
def test_fp64_one_step_parity_from_gpu_states(name):
    """One-step parity (contact forces, sums, state, history) at 1e-9 from the GPU's own
    state at several steps of a run, so that every step is checked against the oracle
    from identical inputs, whatever the separation of the free-running trajectories."""
    make, chunks = ONE_STEP_SCENES[name]
    s = make()
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    report = []
    errs, n = one_step_parity(w, ow, None)
    report.append((0, n, errs))
    for k in chunks:
        w.step(k - 1)
        assert ow.step(k - 1) == 0
        stored = w.contacts()          # the history the next step stores
        w.step(1)
        assert ow.step(1) == 0
        errs, n = one_step_parity(w, ow, stored)
        report.append((w.stats()["steps"] - 1, n, errs))
    print(name, [(d, n, {k: f"{v:.2g}" for k, v in e.items()}) for d, n, e in report])
    assert sum(n for _, n, _ in report) > 20


@pytest.mark.parametrize("seed,vel", [(1, 0.0), (2, 0.3)], ids=["C1_from_rest", "C1b_random_velocities"])
def test_fp64_full_c1_run_matches_oracle(seed, vel):
    """The 2,000-sphere box (R = 1 mm, 40 x 40 x 80 mm, dt = 1e-6 s, FP64, detection every
    step) for its full 2,000 steps, free-running, compared every 500 steps at 1e-9."""
    s = W.settle_box(n=2000, seed=seed, vel_sigma=vel)
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    worst = {}
    for _ in range(4):
        w.step(500)
        assert ow.step(500) == 0
        errs, ok = state_close(w, ow, TOL64)
        assert ok, errs
        worst = {k: max(worst.get(k, 0.0), v) for k, v in errs.items()}
    st = w.stats()
    assert st["steps"] == 2000 and st["rebuilds"] >= 2000
    print("C1", seed, {k: f"{v:.2g}" for k, v in worst.items()}, "contacts", len(ow.eval()[2]))


def test_fp64_trajectory_matches_oracle_random_spheres_in_a_box():
    s = W.settle_box(n=2000, seed=2, vel_sigma=0.3)       # 2,000 spheres, 40x40x80 mm box
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s)
    for _ in range(4):
        w.step(75)
        ow.step(75)
        errs, ok = state_close(w, ow, TOL64)
        assert ok, errs
    st = w.stats()
    assert st["steps"] == 300 and st["rebuilds"] >= 300


def _free_running(s, chunks):
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    worst = {}
    for k in chunks:
        w.step(k)
        assert ow.step(k) == 0
        errs, _ = state_close(w, ow, TOL64)
        worst = {a: max(worst.get(a, 0.0), b) for a, b in errs.items()}
    return w, ow, worst


def test_fp64_trajectory_matches_oracle_dense_polydisperse():
    w, ow, worst = _free_running(dense_scene(n=600, seed=8, vel=0.5), (100, 100))
    print("dense free-running", worst)
    assert max(worst.values()) < TOL64, worst
    compare_contacts(w, ow, TOL64)


def test_fp64_trajectory_matches_oracle_clumps_with_walls_and_gravity():
    w, ow, worst = _free_running(W.packed_clumps(n=150, seed=10), (150, 150))
    print("clumps free-running", worst)
    assert max(worst.values()) < TOL64, worst


def test_fp64_trajectory_matches_oracle_in_a_spinning_drum():
    s = W.drum_bed(n=120, seed=1)
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s)
    wall_contacts = 0
    worst = {}
    for _ in range(10):
        w.step(100)
        ow.step(100)
        cs = ow.eval()[2]
        wall_contacts += int(np.sum(cs["j"] < 0))
        errs, _ = state_close(w, ow, TOL64)
        worst = {a: max(worst.get(a, 0.0), b) for a, b in errs.items()}
    print("drum free-running", worst)
    assert max(worst.values()) < TOL64, worst
    assert wall_contacts > 3


def test_fp64_trajectory_matches_oracle_in_a_cone_hopper_with_sink():
    s = W.cone_bed(n=300, seed=13)
    w, ow, worst = _free_running(s, (300, 300, 300))
    print("cone free-running", worst)
    assert max(worst.values()) < TOL64, worst
    assert ow.active.sum() < len(ow.active)          # some spheres went through the sink


# ----------------------------------------------------------------------------- voxel + FP32

def test_voxel_fp32_forces_within_1e4_of_fp64():
    s = dense_scene(n=1500, seed=14)
    w = dem.World.from_scene(s, precision="voxel_fp32")
    ow = oracle.OracleWorld(s)
    gc = w.contacts()
    F, T, oc = ow.eval()
    key_g = {(a, b): k for k, (a, b) in enumerate(zip(gc["i"], gc["j"]))}
    key_o = {(a, b): k for k, (a, b) in enumerate(zip(oc["i"], oc["j"]))}
    common = sorted(set(key_g) & set(key_o))
    # contacts that appear on one side only must be at vanishing overlap
    for k in set(key_g) ^ set(key_o):
        ov = gc["overlap"][key_g[k]] if k in key_g else oc["overlap"][key_o[k]]
        assert ov < 1e-9
    fo = np.array([oc["force"][key_o[k]] for k in common])
    fg = np.array([gc["force"][key_g[k]] for k in common])
    mag = np.linalg.norm(fo, axis=1)
    floor = 1e-3 * np.median(mag)
    err = np.linalg.norm(fg - fo, axis=1) / np.maximum(mag, floor)
    assert len(common) > 500
    assert err.max() <= 1e-4, (err.max(), np.percentile(err, 99))


def test_voxel_fp32_trajectory_close_to_oracle_over_short_run():
    s = dense_scene(n=500, seed=15, vel=0.2)
    w = dem.World.from_scene(s, precision="voxel_fp32")
    ow = oracle.OracleWorld(s)
    w.step(50)
    ow.step(50)
    x, q, v, wb = w.owner_state()
    assert np.max(np.abs(x - ow.x)) < 1e-8            # metres, after 50 steps
    assert rel_err(v, ow.v, float(np.max(np.abs(ow.v)))) < 1e-3


def test_voxel_fp32_derived_owner_constants_stay_close_to_oracle():
    # single spheres with I = 0.4 m R^2 throughout: the voxel-form kernels derive 1/m and
    # 1/I from the mass and radius; one sphere with another inertia makes the world read
    # them instead.  Both runs follow the oracle, with torques from contacts
    s = dense_scene(n=500, seed=16, vel=0.2)
    s2 = dataclasses.replace(s, templates=s.templates + [dataclasses.replace(
        s.templates[0], moi=s.templates[0].moi * 1.25)],
        owner_template=np.where(np.arange(s.n_owner) == 7, len(s.templates), s.owner_template))
    for sc, derived in ((s, 1), (s2, 0)):
        w = dem.World.from_scene(sc, precision="voxel_fp32")
        assert w.stats()["derived_constants"] == derived
        ow = oracle.OracleWorld(sc)
        w.step(50)
        ow.step(50)
        x, q, v, wb = w.owner_state()
        assert np.max(np.abs(x - ow.x)) < 1e-8
        assert rel_err(v, ow.v, float(np.max(np.abs(ow.v)))) < 1e-3
        assert rel_err(wb, ow.wb, float(np.max(np.abs(ow.wb)))) < 1e-3
        assert np.max(np.abs(ow.wb)) > 0.0
    assert dem.World.from_scene(s, precision="fp64").stats()["derived_constants"] == 0


@pytest.mark.parametrize("precision", ["fp64", "voxel_fp32"])
def test_orientation_of_spheres_at_rest_and_turning(precision):
    # a single sphere that does not turn keeps its orientation exactly; one that turns
    # follows the oracle; a spin set to zero mid-run, the bounce off walls and contacts
    # (which start spins) and a checkpoint restore keep both orientation buffers right
    s = W.settle_box(n=600, vel_sigma=0.3, seed=21)
    w = dem.World.from_scene(s, precision=precision)
    ow = oracle.OracleWorld(s, threads=oracle_threads())
    rng = np.random.default_rng(5)
    x, q, v, wb = w.owner_state()
    q = rng.normal(size=q.shape)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    wb = np.where((np.arange(len(wb)) % 3 == 0)[:, None], rng.normal(scale=50.0, size=wb.shape), 0.0)
    w.set_owner_state(0, quat=q, omega=wb)
    q_set = w.owner_state()[1].copy()
    sync_oracle_to_gpu(w, ow, None)
    tol = TOL64 if precision == "fp64" else 1e-4
    for k in (30, 30):
        w.step(k)
        assert ow.step(k) == 0
        st, ok = state_close(w, ow, tol)
        assert ok, st
    x1, q1, v1, w1 = w.owner_state()
    rest = np.all(w1 == 0.0, axis=1) & np.all(wb == 0.0, axis=1)
    assert rest.sum() > 50
    assert np.array_equal(q1[rest], q_set[rest])            # never turned: the same bits
    # stop every spin, then step on: the orientations stay as they are
    blob = w.save_state()
    w.set_owner_state(0, omega=np.zeros_like(w1))
    q_stop = w.owner_state()[1].copy()
    w.step(1)
    q2, w2 = w.owner_state()[1], w.owner_state()[3]
    still = np.all(w2 == 0.0, axis=1)
    assert still.sum() > 50 and np.array_equal(q2[still], q_stop[still])
    # a restore mid-run continues as the run it was taken from
    w.step(10)
    want = w.owner_state()
    w.load_state(blob)
    w.set_owner_state(0, omega=np.zeros_like(w1))
    w.step(11)
    for a, b in zip(w.owner_state(), want):
        assert np.array_equal(a, b)


# ----------------------------------------------------------------------------- schedules, determinism

@pytest.mark.parametrize("precision", ["fp64", "voxel_fp32"])
def test_delayed_schedule_is_bit_identical_to_every_step(precision):
    s = dense_scene(n=1000, seed=16, vel=0.3)
    # same margin_max: it sizes the cells and, in the voxel form, the voxel edge
    a = dem.World.from_scene(s, precision=precision, schedule="every_step", margin_max=5e-5)
    b = dem.World.from_scene(s, precision=precision, schedule="velocity_bound", margin=5e-5, margin_max=5e-5)
    a.step(200)
    b.step(200)
    for xa, xb in zip(a.owner_state(), b.owner_state()):
        assert np.array_equal(xa, xb)
    sb = b.stats()
    assert sb["steps"] == 200
    assert sb["rebuilds"] < 200


def test_runs_are_deterministic():
    s = dense_scene(n=800, seed=17)
    a = dem.World.from_scene(s, precision="voxel_fp32")
    b = dem.World.from_scene(s, precision="voxel_fp32")
    a.step(100)
    b.step(100)
    for xa, xb in zip(a.owner_state(), b.owner_state()):
        assert np.array_equal(xa, xb)


def test_checkpoint_resume_is_bit_exact():
    s = dense_scene(n=600, seed=18)
    a = dem.World.from_scene(s, precision="fp64", schedule="velocity_bound", margin=4e-5, margin_max=4e-5)
    a.step(60)
    blob = a.save_state()
    a.step(60)
    b = dem.World.from_scene(s, precision="fp64", schedule="velocity_bound", margin=4e-5, margin_max=4e-5)
    b.load_state(blob)
    b.step(60)
    for xa, xb in zip(a.owner_state(), b.owner_state()):
        assert np.array_equal(xa, xb)


def test_batch_equals_separate_worlds():
    scenes = [W.column_collapse(n, asp, mu, e, seed=40 + k)
              for k, (n, asp, mu, e) in enumerate([(300, 1.0, 0.3, 0.5), (900, 2.5, 0.6, 0.8), (150, 0.5, 0.2, 0.3)])]
    bt = dem.Batch(scenes, precision="fp64")
    bt.initialize()
    bt.step(100)
    for k, s in enumerate(scenes):
        w = dem.World.from_scene(s, precision="fp64")
        w.step(100)
        for xa, xb in zip(bt.worlds[k].owner_state(), w.owner_state()):
            assert np.array_equal(xa, xb)


# ----------------------------------------------------------------------------- failure paths

def test_divergence_stops_at_the_last_good_step():
    # spheres released from rest accelerate under gravity until one exceeds 5 mm/s
    s = W.settle_box(n=300, box=(0.02, 0.02, 0.02), seed=19, vel_sigma=0.0)
    s.v_err = 0.005
    w = dem.World.from_scene(s, precision="fp64")
    with pytest.raises(dem.DemError) as ei:
        w.step(1000)
    assert ei.value.status == dem.ERR_DIVERGED
    k = w.stats()["steps"]
    assert 300 < k < 1000
    ow = oracle.OracleWorld(s)
    ow._w.v_err = 0.0
    ow.step(k)
    errs, ok = state_close(w, ow, 1e-9)
    assert ok, errs
    assert np.max(np.linalg.norm(w.owner_state()[2], axis=1)) <= s.v_err
    ow.step(1)
    assert np.max(np.linalg.norm(ow.v, axis=1)) > s.v_err     # the next step is the offending one


def test_list_capacity_regrows_on_overflow():
    # small spheres packed around large ones: rows far beyond the initial capacity
    rng = np.random.default_rng(20)
    big = W.sphere_template(3e-3)
    small = W.sphere_template(0.6e-3)
    xb = np.array([[0.02, 0.02, 0.02]])
    dirs = rng.normal(size=(60, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    xs = xb + dirs * (3.55e-3)
    x = np.concatenate([xb, xs])
    s = W.Scene(np.zeros(3), np.full(3, 0.04), np.array([1e7]), np.array([0.3]), np.array([[0.5]]),
                np.array([[0.4]]), [], [big, small], np.array([0] + [1] * 60), None, x,
                np.tile([1.0, 0, 0, 0], (61, 1)), np.zeros((61, 3)), np.zeros((61, 3)), 1e-6, np.zeros(3))
    w = dem.World.from_scene(s, precision="fp64", margin=1e-4, margin_max=1e-4)
    st = w.stats()
    assert st["overflow_regrows"] >= 1 and st["list_capacity"] > 16
    ow = oracle.OracleWorld(s)
    compare_contacts(w, ow, TOL64)
    w.step(20)
    ow.step(20)
    errs, ok = state_close(w, ow, 1e-8)
    assert ok, errs


def test_set_owner_state_forces_a_rebuild_and_keeps_history():
    s = dense_scene(n=500, seed=21)
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s)
    w.step(30)
    ow.step(30)
    x, q, v, wb = w.owner_state()
    x2 = x.copy()
    x2[:, 0] += 1e-7            # a rigid shift keeps every contact
    w.set_owner_state(0, xyz=x2)
    ow.x[:] = x2
    ow.q[:] = q
    ow.v[:] = v
    ow.wb[:] = wb
    w.step(10)
    ow.step(10)
    errs, ok = state_close(w, ow, 1e-8)
    assert ok, errs


def test_state_upload_keeps_the_list_within_the_margin():
    # delayed schedule: an upload adds each owner's displacement to the audit bounds; the
    # list stays where no owner moved past the margin, and the run is the same bits as
    # one without the round trip; a larger shift rebuilds the list, and both follow the
    # oracle
    s = W.dense_lattice(n=900, seed=23, vel_sigma=0.3)
    beta = 5e-5
    kw = dict(precision="fp64", schedule="velocity_bound", margin=beta, margin_max=beta)
    a = dem.World.from_scene(s, **kw)
    b = dem.World.from_scene(s, **kw)
    a.step(50)
    b.step(50)
    r0 = b.stats()["rebuilds"]
    # positions and velocities pass through the host unchanged (the angular velocity is
    # read in the body frame and rotated back, which rounds once a sphere has turned)
    for _ in range(40):
        a.step(1)
        x, q, v, wb = b.owner_state()
        b.set_owner_state(0, xyz=x, vel=v)
        b.step(1)
    for x, y in zip(a.owner_state(), b.owner_state()):
        assert np.array_equal(x, y)
    assert b.stats()["rebuilds"] - r0 <= a.stats()["rebuilds"] - r0 + 1
    # the whole state through the host every step follows the oracle
    c = dem.World.from_scene(s, **kw)
    oc = oracle.OracleWorld(s)
    c.step(50)
    assert oc.step(50) == 0
    for _ in range(20):
        x, q, v, wb = c.owner_state()
        c.set_owner_state(0, xyz=x, quat=q, vel=v, omega=wb)
        c.step(1)
        assert oc.step(1) == 0
    errs, ok = state_close(c, oc, 1e-8)
    assert ok, errs
    for shift, rebuilt in ((0.1 * beta, False), (3.0 * beta, True)):
        w = dem.World.from_scene(s, **kw)
        ow = oracle.OracleWorld(s)
        w.step(29)
        stored = w.contacts()               # the history the 30th step leaves
        w.step(1)
        x, q, v, wb = w.owner_state()
        x2 = x.copy()
        x2[::7, 0] += shift
        n0 = w.stats()["rebuilds"]
        w.set_owner_state(0, xyz=x2)
        sync_oracle_to_gpu(w, ow, stored)
        w.step(1)
        assert (w.stats()["rebuilds"] > n0) == rebuilt
        assert ow.step(1) == 0
        w.step(9)
        assert ow.step(9) == 0
        errs, ok = state_close(w, ow, 1e-8)
        assert ok, (shift, errs)


def test_diagnostics_match_oracle():
    """The GPU's fixed-order FP64 sums against the oracle's compensated sums of the same
    state, at 1e-9 of the summed magnitudes (energies: the sums themselves, every term
    of one sign; momenta: the sum of the terms' magnitudes)."""
    for s, steps in ((dense_scene(n=700, seed=22), 20), (W.packed_clumps(n=150, seed=10), 150)):
        w = dem.World.from_scene(s, precision="fp64")
        ow = oracle.OracleWorld(s)
        w.step(steps)
        sync_oracle_to_gpu(w, ow, None)
        dg = w.diagnostics()
        do = ow.diagnostics()
        for k in ("ke", "pe", "elastic"):
            assert dg[k] == pytest.approx(do[k], rel=TOL64, abs=1e-300), k
        m = ow.mass[:, None]
        p_scale = np.sum(np.abs(m * ow.v), axis=0)
        assert np.all(np.abs(dg["momentum"] - do["momentum"]) <= TOL64 * p_scale + 1e-300)
        L_orb = np.abs(np.cross(ow.x, m * ow.v)).sum(axis=0)
        L_spin = np.sum(np.abs(ow.moi * ow.wb), axis=0).max()
        assert np.all(np.abs(dg["angmom"] - do["angmom"]) <= TOL64 * (L_orb + L_spin) + 1e-300)
        assert do["elastic"] > 0.0


# ----------------------------------------------------------------------------- wall screens

_DELTAS = [-1e-4, -5e-5, -2e-5, -1e-6, -1e-9, -1e-12, 0.0, 1e-12, 1e-9, 1e-6, 2e-5, 5e-5, 1e-4]


def _threshold_scene(kind, R=1e-3, beta=4e-5):
    """Spheres whose gap to one wall is R + beta + delta for each delta above (from well
    outside the FP32 screening band down to a picometre), spaced 4R apart."""
    Em, num, corm, mum = W._single_material(1e7, 0.3, 0.5, 0.4)
    T = R + beta
    pts = []
    if kind == "plane":
        lo, hi = np.array([0.0, 0.0, 0.0]), np.array([0.2, 0.02, 0.05])
        walls = [dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))]
        for k, dl in enumerate(_DELTAS):
            pts.append([0.004 + 4 * R * k, 0.01, T + dl])
    elif kind == "cylinder":
        r0 = 0.05
        lo, hi = np.array([-0.1, -0.06, -0.06]), np.array([0.1, 0.06, 0.06])
        walls = [dict(type=W.CYLINDER, mat=0, p=np.zeros(3), n=np.array([1.0, 0.0, 0.0]), r0=r0)]
        for k, dl in enumerate(_DELTAS):
            phi = 0.37 + 0.45 * k
            rho = r0 - (T + dl)
            pts.append([-0.05 + 4 * R * k, rho * np.cos(phi), rho * np.sin(phi)])
    else:
        r0, z0, r1, z1 = 0.01, 0.0, 0.04, 0.05
        lo, hi = np.array([-0.05, -0.05, -0.01]), np.array([0.05, 0.05, 0.06])
        walls = [dict(type=W.CONE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]), r0=r0, z0=z0, r1=r1, z1=z1)]
        dr, dz = r1 - r0, z1 - z0
        ln = np.hypot(dr, dz)
        inr, inz = -dz / ln, dr / ln
        if inr > 0:
            inr, inz = -inr, -inz
        for k, dl in enumerate(_DELTAS):
            t = 0.2 + 0.05 * k
            rho = r0 + t * dr + (T + dl) * inr
            z = z0 + t * dz + (T + dl) * inz
            phi = 0.3 + 0.47 * k
            pts.append([rho * np.cos(phi), rho * np.sin(phi), z])
    pts = np.array(pts)
    n = len(pts)
    return W.Scene(lo, hi, Em, num, corm, mum, walls, [W.sphere_template(R)], np.zeros(n, np.int64), None, pts,
                   W._identity_quats(n), np.zeros((n, 3)), np.zeros((n, 3)), 1e-6, np.zeros(3), r_max=R)


@pytest.mark.parametrize("precision", ["fp64", "voxel_fp32"])
@pytest.mark.parametrize("kind", ["plane", "cylinder", "cone"])
def test_wall_sets_at_the_threshold_match_the_fp64_predicate(kind, precision):
    beta = 4e-5
    s = _threshold_scene(kind, beta=beta)
    w = dem.World.from_scene(s, precision=precision, margin=beta, margin_max=beta)
    ow = oracle.OracleWorld(s)
    if precision == "fp64":
        p, r = w.sphere_positions()
        ow.rad[:] = r
    else:
        cell, off, L = w.sphere_voxels()
        _, r = w.sphere_positions()
        p = (np.asarray(s.box_lo) + cell.astype(np.float64) * L) + off.astype(np.float64)
        ow.rad[:] = r.astype(np.float32).astype(np.float64)
    si, wi = w.listed_wall_pairs()
    osi, owi = ow.listed_wall_pairs(p, beta)
    # the spheres inside the threshold are listed, those outside are not
    assert 4 <= len(osi) <= len(_DELTAS) - 4
    assert np.array_equal(si, osi) and np.array_equal(wi, owi)


def test_pair_and_busy_step_counters_follow_the_lists():
    # every-step detection: a read-back shows the list built from the current state, the
    # one the next step uses
    s = dense_scene(n=900, seed=8)
    for precision in ("voxel_fp32", "fp64"):
        w = dem.World.from_scene(s, precision=precision, schedule="every_step", margin_max=5e-5)
        prev = w.stats()
        for _ in range(12):
            w.step(1)
            st = w.stats()
            assert st["pair_steps"] - prev["pair_steps"] == prev["listed_pairs"]
            assert st["busy_steps"] - prev["busy_steps"] == prev["spheres_with_entries"]
            prev = st
        assert prev["listed_pairs"] > 100


def test_voxel_forces_on_axis_planes_match_fp64_at_every_overlap():
    # one sphere against each face of a box, overlaps from a nanometre to 10 micrometres
    R = 1e-3
    Em, num, corm, mum = W._single_material(1e7, 0.3, 0.5, 0.4)
    lo, hi = np.zeros(3), np.array([0.05, 0.04, 0.06])
    pts = []
    for i, dl in enumerate((1e-9, 1e-8, 1e-7, 1e-6, 1e-5)):
        for a in range(3):
            for side in (0, 1):
                # the five spheres of a wall 6 mm apart along one in-plane axis
                p = 0.5 * (lo + hi)
                p[(a + 1) % 3] += 0.006 * (i - 2)
                p[a] = lo[a] + (R - dl) if side == 0 else hi[a] - (R - dl)
                pts.append(p)
    pts = np.array(pts)
    n = len(pts)
    rng = np.random.default_rng(51)
    s = W.Scene(lo, hi, Em, num, corm, mum, W.box_walls(lo, hi), [W.sphere_template(R)], np.zeros(n, np.int64),
                None, pts, W._identity_quats(n), rng.normal(scale=0.05, size=(n, 3)),
                rng.normal(scale=20.0, size=(n, 3)), 1e-6, np.zeros(3), r_max=R)
    w = dem.World.from_scene(s, precision="voxel_fp32")
    ow = oracle.OracleWorld(s)
    cell, off, L = w.sphere_voxels()
    # the oracle at the voxel form's own positions (the radius, kept as a float-float pair
    # by the voxel form, is the scene's)
    ow.x[:] = (np.asarray(s.box_lo) + cell.astype(np.float64) * L) + off.astype(np.float64)
    F, T = w.owner_forces()
    Fo, To, oc = ow.eval()
    assert len(oc) == n
    mag = np.linalg.norm(Fo, axis=1)
    err = np.linalg.norm(F - Fo, axis=1) / mag
    assert err.max() <= 1e-4, err.max()


def test_unset_pairs_of_differing_materials_are_rejected():
    """Sec. 3.1 sets restitution and friction per material pair and gives no rule for
    combining two materials: a pair of materials that differ needs its value set."""
    def world(cor_b, mu_b, set_pair):
        w = dem.World((0, 0, 0), (0.02, 0.02, 0.02), precision="fp64")
        a = w.add_material(1e7, 0.3, 0.5, 0.4)
        b = w.add_material(2e7, 0.25, cor_b, mu_b)
        if set_pair:
            w.set_material_pair(dem.PROP_COR, a, b, 0.45)
            w.set_material_pair(dem.PROP_MU, a, b, 0.35)
        w.add_box_walls(a)
        t = w.add_clump_template([[0, 0, 0]], [1e-3], [b], 1e-5, [4e-12] * 3)
        w.add_clumps(t, [[0.005, 0.005, 0.005], [0.0075, 0.005, 0.005]])
        return w
    for cor_b, mu_b in ((0.7, 0.4), (0.5, 0.6)):
        w = world(cor_b, mu_b, False)
        with pytest.raises(dem.DemError) as e:
            w.initialize()
        assert e.value.status == dem.ERR_STATE and "dem_set_material_pair" in str(e.value)
        w.close()
        w = world(cor_b, mu_b, True)
        w.initialize()
        w.step(2)
        w.close()
    # equal CoR and mu need no pair value (E and nu combine by the Hertz-Mindlin rule)
    w = world(0.5, 0.4, False)
    w.initialize()
    w.step(2)
    w.close()


# ----------------------------------------------------------------------------- rolling resistance

def with_rolling(scene, crr):
    nm = len(scene.E)
    return dataclasses.replace(scene, crr=np.full((nm, nm), crr))


def stored_contacts(w):
    c = w.contacts()
    c["age"] = w.contact_rolling()[0]
    return c


ROLLING_SCENES = {
    "dense_polydisperse": (lambda: with_rolling(dense_scene(n=600, seed=8, vel=0.5), 0.08), (100, 300)),
    "clumps_walls_gravity": (lambda: with_rolling(W.packed_clumps(n=150, seed=10), 0.05), (150, 300)),
    "spinning_drum": (lambda: with_rolling(W.drum_bed(n=120, seed=1), 0.1), (400, 800)),
}


@pytest.mark.parametrize("name", sorted(ROLLING_SCENES))
def test_fp64_rolling_resistance_matches_oracle(name):
    """Rolling resistance (Sec. 4.1, F_r / tau_r, with the collision-time gate of the
    default model of Sec. 4.2.1): one-step parity at 1e-9 from the GPU's own states,
    contact ages included (they must agree bit for bit), and the free-running trajectory
    within 1e-9."""
    make, chunks = ROLLING_SCENES[name]
    s = make()
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    free = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    errs, n = one_step_parity(w, ow, None, rolling=True)
    assert one_step_parity.rolling_on == 0             # every contact is younger than its collision time
    assert free.step(1) == 0
    worst = {}
    rolling_on = 0
    for k in chunks:
        w.step(k - 1)
        assert ow.step(k - 1) == 0
        assert free.step(k) == 0
        stored = stored_contacts(w)
        w.step(1)
        assert ow.step(1) == 0
        st, _ = state_close(w, free, TOL64)
        worst = {a: max(worst.get(a, 0.0), b) for a, b in st.items()}
        errs, n = one_step_parity(w, ow, stored, rolling=True)
        rolling_on += one_step_parity.rolling_on
        assert free.step(1) == 0
        assert n > 0
    print(name, "rolling free-running", worst, "contacts with rolling resistance", rolling_on)
    assert max(worst.values()) < TOL64, worst
    assert rolling_on > 0


def test_voxel_fp32_rolling_resistance_within_1e4_of_fp64():
    """The voxel + FP32 form with rolling resistance: per-contact forces and rolling
    forces within 1e-4 of the FP64 oracle on the GPU's own state (the precision form's
    metric, normalised by max(|F64|, 1e-3 median |F64|))."""
    s = with_rolling(dense_scene(n=1200, seed=14, vel=0.3), 0.08)
    w = dem.World.from_scene(s, precision="voxel_fp32")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    w.step(299)
    stored = stored_contacts(w)
    w.step(1)
    sync_oracle_to_gpu(w, ow, stored)
    gc = w.contacts()
    age, trf = w.contact_rolling()
    _, _, oc = ow.eval()
    key_g = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(gc["i"], gc["j"]))}
    key_o = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(oc["i"], oc["j"]))}
    common = sorted(set(key_g) & set(key_o))
    assert len(common) > 300
    fo = np.array([oc["force"][key_o[k]] for k in common])
    mag = np.linalg.norm(fo, axis=1)
    floor = 1e-3 * np.median(mag)
    for got, want in ((gc["force"], oc["force"]), (trf, oc["torque_force"])):
        g = np.array([got[key_g[k]] for k in common])
        o = np.array([want[key_o[k]] for k in common])
        err = np.linalg.norm(g - o, axis=1) / np.maximum(mag, floor)
        assert err.max() <= 1e-4, err.max()
    assert np.sum(np.linalg.norm(np.array([oc["torque_force"][key_o[k]] for k in common]), axis=1) > 0) > 100



# ----------------------------------------------------------------------------- family tags

def family_scene(n=800, seed=33):
    """A dense lattice with families: the bottom fifth held fixed, the top tenth pushed
    down at a prescribed 5 cm/s with a prescribed spin, a middle slab whose contacts with
    family 0 are not resolved."""
    s = dense_scene(n=n, seed=seed, vel=0.2)
    z = np.asarray(s.x)[:, 2]
    fam = np.zeros(len(z), np.uint8)
    fam[z < np.quantile(z, 0.2)] = 1
    fam[z > np.quantile(z, 0.9)] = 2
    fam[(z > np.quantile(z, 0.45)) & (z < np.quantile(z, 0.55))] = 3
    return dataclasses.replace(s, family=fam,
                               family_motion={1: ((0, 0, 0), (0, 0, 0)), 2: ((0, 0, -0.05), (0.0, 0.0, 20.0))},
                               family_masked=[(3, 0)])


def test_fp64_families_match_oracle():
    """Family tags (Sec. 2.2.2): fixed and prescribed families move exactly as prescribed,
    masked contacts are never listed, and everything matches the oracle at 1e-9 (one step
    from the GPU's own states, and free-running)."""
    s = family_scene()
    w = dem.World.from_scene(s, precision="fp64")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    free = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    x0 = np.asarray(s.x)
    one_step_parity(w, ow, None)
    assert free.step(1) == 0
    worst = {}
    for k in (100, 200):
        w.step(k - 1)
        assert ow.step(k - 1) == 0 and free.step(k) == 0
        stored = w.contacts()
        w.step(1)
        assert ow.step(1) == 0
        st, _ = state_close(w, free, TOL64)
        worst = {a: max(worst.get(a, 0.0), b) for a, b in st.items()}
        one_step_parity(w, ow, stored)
        assert free.step(1) == 0
    assert max(worst.values()) < TOL64, worst
    x, q, v, wb = w.owner_state()
    fam = s.family
    assert np.array_equal(x[fam == 1], x0[fam == 1]) and np.all(v[fam == 1] == 0.0)
    assert np.all(v[fam == 2] == np.array([0.0, 0.0, -0.05]))
    # no listed pair joins family 3 to family 0
    gi, gj = w.listed_pairs()
    o = ow.owner
    fi, fj = fam[o[gi]], fam[o[gj]]
    assert not np.any(((fi == 3) & (fj == 0)) | ((fi == 0) & (fj == 3)))
    assert np.any((fi == 3) & (fj == 3)) and np.any((fi == 1) & (fj == 0))


def test_voxel_fp32_families_hold_the_prescribed_motion():
    """The voxel form: a fixed family's positions stay bit for bit, a prescribed one moves
    at its velocity, and the rest stays within the precision form's error of FP64."""
    s = family_scene()
    w = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    ow = oracle.OracleWorld(s, cell_list=True, threads=oracle_threads())
    x_start = w.owner_state()[0]
    w.step(300)
    assert ow.step(300) == 0
    x, q, v, wb = w.owner_state()
    fam = s.family
    assert np.array_equal(x[fam == 1], x_start[fam == 1]) and np.all(v[fam == 1] == 0.0)
    assert np.allclose(v[fam == 2], [0.0, 0.0, np.float32(-0.05)], rtol=0, atol=1e-9)
    assert np.max(np.abs(x - ow.x)) < 1e-6


def test_active_box_leaves_the_active_region_bit_identical():
    """Sec. 6.4: owners outside the active box are held fixed and their contacts with each
    other are dropped.  Contacts between two fixed owners move nothing, so the run equals,
    bit for bit, one where the same owners are fixed with every contact resolved; the box
    tags owners by their centres."""
    s = dense_scene(n=1500, seed=41, vel=0.3)
    lo, hi = np.asarray(s.box_lo), np.asarray(s.box_hi)
    blo = lo + 0.25 * (hi - lo)
    bhi = hi - 0.25 * (hi - lo)
    worlds = []
    for dormant_masked in (True, False):
        w = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
        w.set_family_motion(7, (0, 0, 0), (0, 0, 0))
        if dormant_masked:
            w.set_family_contacts(7, 7, False)
        w.set_active_box(blo, bhi, 0, 7)
        worlds.append(w)
    x0 = worlds[0].owner_state()[0]
    inside = np.all((x0 >= blo) & (x0 <= bhi), axis=1)
    for w in worlds:
        w.step(400)
    a, b = worlds
    for xa, xb in zip(a.owner_state(), b.owner_state()):
        assert np.array_equal(xa, xb)
    assert a.stats()["listed_pairs"] < b.stats()["listed_pairs"]
    x = a.owner_state()[0]
    assert np.array_equal(x[~inside], x0[~inside])
    assert np.any(x[inside] != x0[inside])


# ----------------------------------------------------------------------------- contact force models

@pytest.mark.parametrize("precision,crr", [("fp64", 0.0), ("fp64", 0.08), ("voxel_fp32", 0.0)])
def test_functor_default_model_equals_the_builtin_kernel(precision, crr):
    """The default model through the functor interface (Sec. 4.2's custom-model route,
    pairs evaluated with A the lower id on both sides) gives the built-in kernel's bits."""
    s = dense_scene(n=800, seed=51, vel=0.4)
    if crr:
        s = with_rolling(s, crr)
    a = dem.World.from_scene(s, precision=precision, schedule="velocity_bound")
    b = dem.World.from_scene(dataclasses.replace(s, force_model="hertz_mindlin"), precision=precision,
                             schedule="velocity_bound")
    for _ in range(3):
        a.step(100)
        b.step(100)
        for xa, xb in zip(a.owner_state(), b.owner_state()):
            assert np.array_equal(xa, xb)
    ca, cb = a.contacts(), b.contacts()
    for k in ("i", "j", "force", "history"):
        assert np.array_equal(ca[k], cb[k]), k


BREAK = dict(tension=-2e4, cohesion=2e4, eta=0.1, damping=0.01)


def bonded_lattice(seed=61):
    """A dense lattice whose overlapping neighbours are bonded at their initial overlap
    (unloaded), with random velocities that stretch, shear and break bonds (Sec. 6.3)."""
    return dataclasses.replace(dense_scene(n=343, seed=seed, vel=0.3), force_model="bonded_breakage",
                               model_params=BREAK)


def bond_initial_contacts(w, ow):
    c = w.contacts()
    pair = c["j"] >= 0
    i, j, ov = c["i"][pair], c["j"][pair], c["overlap"][pair]
    wc = np.zeros((len(i), 4))
    wc[:, 0] = 1.0
    wc[:, 1] = ov
    w.set_contact_wildcards(i, j, wc)
    for o in ow:
        o.set_wildcards(i, j, wc)
    return len(i)


def test_fp64_bonded_breakage_matches_oracle():
    """The bonded, breakable contact (Sec. 6.3) on the GPU against the oracle at 1e-9:
    one step from the GPU's own states (history, ages and bond wildcards synced) and the
    free-running run, while bonds stretch across gaps and break."""
    s = bonded_lattice()
    w = dem.World.from_scene(s, precision="fp64", margin=5e-5)
    ow = oracle.OracleWorld(s, threads=oracle_threads())
    free = oracle.OracleWorld(s, threads=oracle_threads())
    nb = bond_initial_contacts(w, (ow, free))
    assert nb > 500
    worst = {}
    for k in (1, 100, 200):
        if k > 1:
            w.step(k - 1)
            assert ow.step(k - 1) == 0 and free.step(k - 1) == 0
        c0 = w.contacts()
        wc0 = w.contact_wildcards()
        w.step(1)
        assert ow.step(1) == 0 and free.step(1) == 0
        st, _ = state_close(w, free, TOL64)
        worst = {a: max(worst.get(a, 0.0), b) for a, b in st.items()}
        # one step from the GPU's own state: history, age and bond wildcards carried in
        ow.x[:], ow.q[:], ow.v[:], ow.wb[:] = w.owner_state()
        ow.set_history(c0["i"], c0["j"], c0["history"], age=wc0[:, 3])
        pair = c0["j"] >= 0
        ow.set_wildcards(c0["i"][pair], c0["j"][pair], wc0[pair][:, 4:8])
        gc = w.contacts()
        gw = w.contact_wildcards()
        Fg, Tg = w.owner_forces()
        Fo, To, oc = ow.eval()
        assert np.array_equal(gc["i"], oc["i"]) and np.array_equal(gc["j"], oc["j"])
        fs = np.abs(oc["force"]).max(axis=1, keepdims=True) + 1e-300
        assert rel_err(gc["force"], oc["force"], fs) < TOL64
        assert np.array_equal(gw[:, 4] > 0, np.asarray(oc["wc"])[:, 0] > 0)        # bond states agree
        assert rel_err(Fg, Fo, owner_scale(ow, oc, Fo)) < TOL64
        assert rel_err(Tg, To, torque_scale(ow, oc)) < TOL64
    assert max(worst.values()) < TOL64, worst
    bonds = np.sum(free.wildcards()[:, 0] > 0)
    broken = nb - bonds
    print("bonded breakage: bonds", nb, "left", bonds, "free-running", worst)
    assert 0 < broken < nb


# ----------------------------------------------------------------------------- mesh facets

def test_fp64_mesh_facets_match_oracle():
    """Sphere-facet contacts with a static facet floor and a turning paddle mesh (Sec. 2.4,
    Sec. 5): the listed sets (facets found through their cell bins) equal the oracle's
    brute-force set, and forces and states match at 1e-9, one step from the GPU's own
    states and free-running."""
    s = W.paddle_bed(n=300, seed=3)
    beta = 4e-5
    w = dem.World.from_scene(s, precision="fp64", margin=beta)
    ow = oracle.OracleWorld(s, threads=oracle_threads())
    free = oracle.OracleWorld(s, threads=oracle_threads())
    n_regular = 6
    facet_hits = 0
    worst = {}
    one_step_parity(w, ow, None)
    assert free.step(1) == 0
    for k in (300, 600, 900):
        w.step(k - 1)
        assert ow.step(k - 1) == 0 and free.step(k - 1) == 0
        p, r = w.sphere_positions()
        si, wi = w.listed_wall_pairs()
        osi, owi = ow.listed_wall_pairs(p, beta)
        assert np.array_equal(si, osi) and np.array_equal(wi, owi)
        stored = w.contacts()
        w.step(1)
        assert ow.step(1) == 0 and free.step(1) == 0
        st, _ = state_close(w, free, TOL64)
        worst = {a: max(worst.get(a, 0.0), b) for a, b in st.items()}
        facet_hits += int(np.sum(w.contacts()["j"] <= -1 - n_regular))
        one_step_parity(w, ow, stored)
        assert free.step(1) == 0
    print("paddle bed free-running", worst, "facet contacts", facet_hits)
    assert max(worst.values()) < TOL64, worst
    assert facet_hits > 10


def test_voxel_fp32_mesh_facets_stay_close_to_fp64():
    s = W.paddle_bed(n=300, seed=3)
    w = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    ow = oracle.OracleWorld(s, threads=oracle_threads())
    w.step(400)
    assert ow.step(400) == 0
    x = w.owner_state()[0]
    assert np.max(np.abs(x - ow.x)) < 1e-6
    c = w.contacts()
    assert np.sum(c["j"] <= -7) > 10


def test_large_state_upload_in_pieces_is_checked_whole():
    # from 2^20 owners the upload is copied in four pieces, each checked for non-finite
    # values as it lands: a NaN in the last piece rejects the whole upload with nothing
    # applied; without it every piece lands at its place (FP64 positions, orientations and
    # velocities come back exactly); a ragged range overwrites only itself
    s = W.dense_lattice(n=1_100_000, seed=5, vel_sigma=0.3)
    w = dem.World.from_scene(s, precision="fp64", schedule="velocity_bound")
    try:
        w.step(2)
        x, q, v, wb = w.owner_state()
        rng = np.random.default_rng(0)
        x2 = x + rng.uniform(-1e-7, 1e-7, size=x.shape)
        v2 = v + 0.01
        w2 = 0.5 * wb
        bad = v2.copy()
        bad[-3, 1] = np.nan
        with pytest.raises(dem.DemError) as ei:
            w.set_owner_state(0, xyz=x2, quat=q, vel=bad, omega=w2)
        assert ei.value.status == dem.ERR_ARG
        for a, b in zip(w.owner_state(), (x, q, v, wb)):
            assert np.array_equal(a, b)
        w.set_owner_state(0, xyz=x2, quat=q, vel=v2, omega=w2)
        xa, qa, va, wa = w.owner_state()
        assert np.array_equal(xa, x2) and np.array_equal(qa, q) and np.array_equal(va, v2)
        np.testing.assert_allclose(wa, w2, rtol=1e-12, atol=1e-9 * float(np.abs(w2).max()))
        f, m = 33_333, 1_050_000                    # a ragged range, in four pieces too
        w.set_owner_state(f, xyz=x[f:f + m], vel=v[f:f + m])
        xb, _, vb, _ = w.owner_state()
        ex, ev = x2.copy(), v2.copy()
        ex[f:f + m] = x[f:f + m]
        ev[f:f + m] = v[f:f + m]
        assert np.array_equal(xb, ex) and np.array_equal(vb, ev)
        w.step(2)                                   # and it steps on from there
        assert np.all(np.isfinite(w.owner_state()[0]))
    finally:
        w.close()
