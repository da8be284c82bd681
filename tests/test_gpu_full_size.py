"""Parity at the full size of the bench workload, on sampled outputs.

The 4,000,000-sphere settling column (R ~ U[0.8, 1.2] mm, 0.3 x 0.3 x 1.2 m box, dt = 2e-6 s)
runs in the launch configuration the bench times: voxel positions with FP32 arithmetic,
velocity-bound delayed detection on the second stream, audited every step, and the
tuning the bench's autotuner picks at this size on a GB300 (the two-kernel force step,
128-thread contact blocks, a detection margin of 0.35 of margin_max).  The oracle
cannot step four million spheres, so it evaluates sampled windows of the GPU's own state
one by one: every owner whose centre lies in a cube around a sampled sphere, with the
tangential history the GPU carried into the step.  A sphere in the inner core of a
window has all its possible partners inside the window (a partner's centre lies within
R_i + R_j <= 2 r_max), so the oracle's brute-force contacts of core spheres are complete
and must equal the GPU's: the same contact set (a contact seen by one side only must be
at vanishing overlap) and forces within 1e-4 of the FP64 oracle (error normalised by
max(|F64|, 1e-3 median |F64|), the metric of the precision form).  A contact the delayed
list had missed would show as a set difference, since the GPU reports contacts from the
list in use.

``test_window_sampling_reproduces_whole_world_contacts`` (CPU) checks the sampling
method itself: windows cut from an oracle run reproduce that run's own contacts exactly.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2311_04648_gb300 import workloads as W

N_FULL = 4_000_000
STEPS = 2500           # mid-run: the column has closed many lattice gaps (the bench tunes here too)
N_WINDOWS = 800
TOL = 1e-4


def window_centres(x, cs, n, seed):
    """Centres of n windows: spheres drawn from the contacts (a quarter of them from wall
    contacts) so that every window holds contacts to compare."""
    rng = np.random.default_rng(seed)
    wall = np.unique(cs["i"][cs["j"] < 0])
    pair = np.unique(cs["i"][cs["j"] >= 0])
    nw = min(len(wall), n // 4)
    pick = np.concatenate([rng.choice(wall, nw, replace=False) if nw else np.zeros(0, np.int64),
                           rng.choice(pair, min(len(pair), n - nw), replace=False)])
    return x[pick]


def in_boxes(x, centres, half):
    """Mask of the points within ``half`` (per axis) of any centre.  Points are binned in
    cubes of edge 2 half, so a box around a centre meets at most two cubes per axis."""
    sel = np.zeros(len(x), bool)
    if len(x) == 0 or len(centres) == 0:
        return sel
    edge = 2.0 * half
    lo = x.min(axis=0)
    cell = np.floor((x - lo) / edge).astype(np.int64)
    dims = cell.max(axis=0) + 2
    key = (cell[:, 0] * dims[1] + cell[:, 1]) * dims[2] + cell[:, 2]
    order = np.argsort(key, kind="stable")
    skey = key[order]
    for c in centres:
        a = np.floor((c - half - lo) / edge).astype(np.int64)
        b = np.floor((c + half - lo) / edge).astype(np.int64)
        for cx in range(a[0], b[0] + 1):
            for cy in range(a[1], b[1] + 1):
                for cz in range(a[2], b[2] + 1):
                    k = (cx * dims[1] + cy) * dims[2] + cz
                    ids = order[np.searchsorted(skey, k):np.searchsorted(skey, k, side="right")]
                    sel[ids[np.all(np.abs(x[ids] - c) <= half, axis=1)]] = True
    return sel


def oracle_window_contacts(scene, x, q, v, wb, sub, hist):
    """The oracle's contacts among the owners ``sub`` (sorted global ids; one sphere per
    owner) at the given state, with the stored tangential history ``hist`` (global ids,
    as ``dem.World.contacts`` reports it) carried in; ids returned global."""
    sc = dataclasses.replace(scene, owner_template=np.asarray(scene.owner_template)[sub],
                             owner_scale=np.asarray(scene.owner_scale)[sub],
                             x=x[sub], q=q[sub], v=v[sub], wb=wb[sub])
    ow = oracle.OracleWorld(sc, cell_list=True)
    loc = np.full(len(x), -1, np.int64)
    loc[sub] = np.arange(len(sub))
    hi, hj = np.asarray(hist["i"]), np.asarray(hist["j"])
    li = loc[hi]
    lj = np.where(hj >= 0, loc[np.maximum(hj, 0)], hj)
    keep = (li >= 0) & ((hj < 0) | (lj >= 0))
    ow.set_history(li[keep], lj[keep], np.asarray(hist["history"])[keep])
    _, _, oc = ow.eval()
    gi = sub[oc["i"]]
    gj = np.where(oc["j"] >= 0, sub[np.maximum(oc["j"], 0)], oc["j"])
    return dict(i=gi, j=gj, force=np.array(oc["force"]), overlap=np.array(oc["overlap"]))


def compare_core(gc, oc, core, tol):
    """Contacts touching a core sphere: equal sets up to vanishing overlaps, forces within
    ``tol`` of the oracle's.  Returns (compared contacts, wall contacts, max error, p99)."""
    def index(c):
        out = {}
        for k, (a, b) in enumerate(zip(c["i"], c["j"])):
            if core[a] or (b >= 0 and core[b]):
                out[(int(a), int(b))] = k
        return out
    kg, ko = index(gc), index(oc)
    for key in set(kg) ^ set(ko):
        ov = gc["overlap"][kg[key]] if key in kg else oc["overlap"][ko[key]]
        assert ov < 1e-9, (key, ov, key in kg)
    common = sorted(set(kg) & set(ko))
    fo = np.array([oc["force"][ko[k]] for k in common]).reshape(-1, 3)
    fg = np.array([gc["force"][kg[k]] for k in common]).reshape(-1, 3)
    mag = np.linalg.norm(fo, axis=1)
    floor = 1e-3 * np.median(mag) if len(mag) else 0.0
    err = np.linalg.norm(fg - fo, axis=1) / np.maximum(mag, floor + 1e-300)
    emax = float(err.max()) if len(err) else 0.0
    p99 = float(np.percentile(err, 99)) if len(err) else 0.0
    assert emax <= tol, (emax, p99)
    return len(common), sum(1 for k in common if k[1] < 0), emax, p99


def sampled_parity(scene, state, c0, c1, n_windows, seed=11):
    """Windows around sampled contacts of state k+1 (``c1``), history from state k
    (``c0``, the history each contact stores for the next step)."""
    x, q, v, wb = state
    r_max = float(scene.r_max)
    core_half = 1.5 * r_max
    half = core_half + 2.0 * r_max + 1e-4
    centres = window_centres(x, c1, n_windows, seed)
    sub = np.flatnonzero(in_boxes(x, centres, half))
    core = in_boxes(x, centres, core_half)
    oc = oracle_window_contacts(scene, x, q, v, wb, sub, c0)
    return compare_core(c1, oc, core, TOL)


def test_window_sampling_reproduces_whole_world_contacts():
    """The sampling method against the whole-world oracle: a dense 4,000-sphere lattice in a
    walled box stepped by the oracle, windows cut from its state with its own history."""
    s = W.dense_lattice(n=4000, seed=21)
    ow = oracle.OracleWorld(s, cell_list=True)
    assert ow.step(20) == 0
    c0 = ow.eval()[2]
    hist0 = dict(i=np.array(c0["i"]), j=np.array(c0["j"]), history=np.array(c0["ut"]))
    assert ow.step(1) == 0
    c1 = ow.eval()[2]
    gc = dict(i=np.array(c1["i"]), j=np.array(c1["j"]), force=np.array(c1["force"]),
              overlap=np.array(c1["overlap"]))
    state = (ow.x.copy(), ow.q.copy(), ow.v.copy(), ow.wb.copy())
    n, n_wall, emax, _ = sampled_parity(s, state, hist0, gc, 40)
    assert n > 100 and n_wall > 5
    assert emax == 0.0            # the same FP64 arithmetic on the same inputs
    # a contact missing from the compared side is caught
    r_max = float(s.r_max)
    core = in_boxes(state[0], window_centres(state[0], gc, 40, 11), 1.5 * r_max)
    k = int(np.flatnonzero(core[gc["i"]] & (gc["overlap"] > 1e-6))[0])
    dropped = {key: np.delete(val, k, axis=0) for key, val in gc.items()}
    with pytest.raises(AssertionError):
        sampled_parity(s, state, hist0, dropped, 40)


def test_in_boxes_matches_a_direct_scan():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 2.0, size=(20000, 3))
    centres = rng.uniform(-1.2, 2.2, size=(30, 3))
    direct = np.zeros(len(x), bool)
    for c in centres:
        direct |= np.all(np.abs(x - c) <= 0.17, axis=1)
    assert np.array_equal(in_boxes(x, centres, 0.17), direct)


@pytest.mark.gpu
def test_full_size_bench_workload_matches_oracle_on_sampled_windows():
    from paper_2311_04648_gb300 import dem
    s = W.settling_column(n=N_FULL)
    w = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    try:
        w.set_tuning(contact_block=128, fused_block=0, margin=0.35 * w.tuning()["margin"])
        w.step(STEPS)
        c0 = w.contacts()                      # the first read-back allocates its buffer
        again = w.contacts()
        w.step(1)
        st = w.stats()
        state = w.owner_state()
        c1 = w.contacts()
    finally:
        w.close()
    # a read-back gives the same answer whether or not its buffer was just allocated
    for key in c0:
        assert np.array_equal(c0[key], again[key]), key
    assert st["steps"] == STEPS + 1
    assert st["rebuilds"] > 1                  # the delayed list was rebuilt along the way
    assert np.all(np.isfinite(state[0]))
    n, n_wall, emax, p99 = sampled_parity(s, state, c0, c1, N_WINDOWS)
    print(f"full size: {len(c1['i'])} contacts, {n} compared ({n_wall} with walls), "
          f"force error max {emax:.3g} p99 {p99:.3g}")
    assert n > 600 and n_wall > 100
