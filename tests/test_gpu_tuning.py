"""GPU: captured CUDA graphs, launch shapes, detection cell size, detection placement and
the autotuner change timing only: every configuration gives bit-identical states."""
import os

import numpy as np
import pytest

from paper_2311_04648_gb300 import dem, workloads as W

pytestmark = pytest.mark.gpu


def _state(w):
    return w.owner_state()


def test_graphs_tunings_and_inline_detection_are_bit_identical():
    s = W.dense_lattice(n=800, seed=31, vel_sigma=0.3)
    beta = 5e-5
    ref = dem.World.from_scene(s, precision="voxel_fp32", schedule="every_step", margin_max=beta)
    ref.step(150)
    want = _state(ref)
    runs = []
    a = dem.World.from_scene(s, precision="voxel_fp32", schedule="every_step", margin_max=beta)
    a.set_graphs(False)
    runs.append(a)
    b = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    b.set_tuning(contact_block=32, integrate_block=512, narrow_block=256, detect_inline=1, fused_block=0)
    runs.append(b)
    c = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    c.set_tuning(contact_block=128, integrate_block=128, narrow_block=64, detect_inline=0, cell_factor=2.0,
                 fused_block=256)
    runs.append(c)
    f = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    f.set_tuning(contact_block=32, contact_lean=1, integrate_staged=1, fused_block=0)
    runs.append(f)
    e = dem.World.from_scene(s, precision="voxel_fp32", schedule="every_step", margin_max=beta)
    e.set_tuning(cell_factor=1.5)
    runs.append(e)
    g = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    g.set_tuning(margin=0.35 * beta)             # fewer listed pairs, more rebuilds
    assert g.tuning()["margin"] == 0.35 * beta
    with pytest.raises(Exception):
        g.set_tuning(margin=2.0 * beta)          # above margin_max
    runs.append(g)
    for w in runs:
        w.step(150)
        for x, y in zip(_state(w), want):
            assert np.array_equal(x, y)
    assert g.stats()["rebuilds"] > b.stats()["rebuilds"]
    # margins changed in mid-run
    m = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    for k, fm in ((40, 0.5), (50, 1.0), (60, 0.35)):
        m.set_tuning(margin=fm * beta)
        m.step(k)
    for x, y in zip(_state(m), want):
        assert np.array_equal(x, y)
    assert c.stats()["cell_size"] > 1.9 * ref.stats()["cell_size"]
    # a cell size change in mid-run, in the FP64 form as well
    for prec in ("voxel_fp32", "fp64"):
        p = dem.World.from_scene(s, precision=prec, schedule="velocity_bound", margin=beta, margin_max=beta)
        q = dem.World.from_scene(s, precision=prec, schedule="velocity_bound", margin=beta, margin_max=beta)
        p.step(70)
        p.set_tuning(cell_factor=3.0)
        p.step(40)
        p.set_tuning(cell_factor=1.0)
        p.step(40)
        q.step(150)
        for x, y in zip(_state(p), _state(q)):
            assert np.array_equal(x, y)
        assert p.listed_pairs()[0].tolist() == q.listed_pairs()[0].tolist()


def test_autotune_restores_the_state_and_reuses_its_cache(tmp_path):
    s = W.dense_lattice(n=600, seed=32, vel_sigma=0.3)
    beta = 5e-5
    w = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    w.step(20)
    before = _state(w)
    steps_before = w.stats()["steps"]
    cache = os.path.join(str(tmp_path), "tune.jsonl")
    t = w.autotune(steps=40, cache_path=cache)
    assert t["step_ms"] > 0
    assert w.tuning()["contact_block"] == t["contact_block"]
    for x, y in zip(_state(w), before):
        assert np.array_equal(x, y)
    assert w.stats()["steps"] == steps_before
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1
    # a second world of the same shape takes the cached choice without trials
    w2 = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    t2 = w2.autotune(steps=40, cache_path=cache)
    for k in ("contact_block", "integrate_block", "narrow_block", "detect_inline"):
        assert t2[k] == t[k]
    assert t2["cell_factor"] == pytest.approx(t["cell_factor"], abs=1e-3)
    assert t2["step_ms"] == pytest.approx(t["step_ms"], abs=1e-6)
    assert 0.0 < t["margin"] <= beta and w.tuning()["margin"] == t["margin"]
    assert t2["margin"] == t["margin"] and w2.tuning()["margin"] == t["margin"]
    assert len(open(cache).read().strip().splitlines()) == 1
    # tuned runs continue exactly like untuned ones
    w.step(60)
    u = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    u.step(80)
    for x, y in zip(_state(w), _state(u)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("kind", ["spheres", "clumps"])
def test_staged_integration_is_bit_identical(kind):
    s = W.dense_lattice(n=700, seed=33, vel_sigma=0.3) if kind == "spheres" else W.packed_clumps(n=200, seed=34)
    beta = 5e-5
    a = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    b = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    # the two-kernel path (the staged integration is not part of the fused step)
    a.set_tuning(fused_block=0)
    b.set_tuning(integrate_staged=1, fused_block=0)
    assert b.tuning()["integrate_staged"] == 1
    a.step(60)
    b.step(60)
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    # switch back and forth in mid-run
    b.set_tuning(integrate_staged=0)
    a.step(20)
    b.step(20)
    b.set_tuning(integrate_staged=1)
    a.step(20)
    b.step(20)
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    assert a.stats()["audit_fallbacks"] == b.stats()["audit_fallbacks"]


def test_staged_integration_in_a_batch_of_scenes():
    scenes = [W.dense_lattice(n=150 + 97 * k, seed=40 + k, vel_sigma=0.3) for k in range(3)]
    beta = 5e-5
    p = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    q = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    p.initialize()
    q.initialize()
    p.worlds[0].set_tuning(fused_block=0)
    q.worlds[0].set_tuning(integrate_staged=1, fused_block=0)
    p.step(50)
    q.step(50)
    for wp, wq in zip(p.worlds, q.worlds):
        for x, y in zip(_state(wp), _state(wq)):
            assert np.array_equal(x, y)


def test_staged_integration_is_refused_by_the_fp64_form():
    s = W.dense_lattice(n=200, seed=35)
    w = dem.World.from_scene(s, precision="fp64", schedule="every_step")
    w.set_tuning(integrate_staged=1)
    assert w.tuning()["integrate_staged"] == 0


@pytest.mark.parametrize("prec", ["voxel_fp32", "fp64"])
def test_fused_step_is_bit_identical(prec):
    # one kernel summing each sphere's contact forces in registers and integrating it
    # against contact forces and integration as two kernels; every block size, switched
    # in mid-run, both schedules
    s = W.dense_lattice(n=900, seed=36, vel_sigma=0.3)
    beta = 5e-5
    for sched in ("every_step", "velocity_bound"):
        kw = dict(precision=prec, schedule=sched, margin_max=beta)
        if sched != "every_step":
            kw["margin"] = beta
        a = dem.World.from_scene(s, **kw)
        a.set_tuning(fused_block=0)
        for k in (50, 20, 50):              # the same calls as below: the same cycles
            a.step(k)
        want = _state(a)
        # read in the same order for every world: stats() rebuilds a stale list
        want_pairs = a.listed_pairs()[0].tolist()
        want_fallbacks = a.stats()["audit_fallbacks"]
        for fb in (64, 128, 256):
            b = dem.World.from_scene(s, **kw)
            b.set_tuning(fused_block=fb)
            assert b.tuning()["fused_block"] == fb
            b.step(50)
            b.set_tuning(fused_block=0)
            b.step(20)
            b.set_tuning(fused_block=fb)
            b.step(50)
            for x, y in zip(_state(b), want):
                assert np.array_equal(x, y)
            assert b.listed_pairs()[0].tolist() == want_pairs
            assert b.stats()["audit_fallbacks"] == want_fallbacks


@pytest.mark.parametrize("prec", ["voxel_fp32", "fp64"])
def test_contact_kernel_integration_is_bit_identical(prec):
    # the contact kernel integrating the owners with listed partners (the integration
    # kernel the rest) against every owner integrated by the integration kernel: both
    # contact builds, switched in mid-run, both schedules
    s = W.dense_lattice(n=900, seed=37, vel_sigma=0.3)
    beta = 5e-5
    for sched in ("every_step", "velocity_bound"):
        kw = dict(precision=prec, schedule=sched, margin_max=beta)
        if sched != "every_step":
            kw["margin"] = beta
        a = dem.World.from_scene(s, **kw)
        a.set_tuning(fused_block=0, contact_integrates=0)
        for k in (50, 20, 50):
            a.step(k)
        want = _state(a)
        want_pairs = a.listed_pairs()[0].tolist()
        want_fallbacks = a.stats()["audit_fallbacks"]
        for lean in (0, 1):
            b = dem.World.from_scene(s, **kw)
            b.set_tuning(fused_block=0, contact_integrates=1, contact_lean=lean)
            assert b.tuning()["contact_integrates"] == 1
            b.step(50)
            b.set_tuning(fused_block=0, contact_integrates=0, contact_lean=lean)
            b.step(20)
            b.set_tuning(fused_block=0, contact_integrates=1, contact_lean=lean)
            b.step(50)
            for x, y in zip(_state(b), want):
                assert np.array_equal(x, y)
            assert b.listed_pairs()[0].tolist() == want_pairs
            assert b.stats()["audit_fallbacks"] == want_fallbacks


def test_contact_kernel_integration_with_a_sink_in_a_batch_and_ignored_for_clumps():
    s = W.cone_bed(n=300, seed=13)
    a = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    b = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    a.set_tuning(fused_block=0, contact_integrates=0)
    b.set_tuning(fused_block=0, contact_integrates=1)
    a.step(900)
    b.step(900)
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    scenes = [W.dense_lattice(n=150 + 97 * k, seed=45 + k, vel_sigma=0.3) for k in range(3)]
    beta = 5e-5
    p = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    q = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    p.initialize()
    q.initialize()
    p.worlds[0].set_tuning(fused_block=0, contact_integrates=0)
    q.worlds[0].set_tuning(fused_block=0, contact_integrates=1)
    p.step(60)
    q.step(60)
    for wp, wq in zip(p.worlds, q.worlds):
        for x, y in zip(_state(wp), _state(wq)):
            assert np.array_equal(x, y)
    c = dem.World.from_scene(W.packed_clumps(n=100, seed=38), precision="voxel_fp32", schedule="every_step")
    c.set_tuning(contact_integrates=1)
    assert c.tuning()["contact_integrates"] == 0


def test_fused_step_with_a_sink_and_walls_is_bit_identical():
    s = W.cone_bed(n=300, seed=13)        # some spheres pass the sink within 900 steps
    a = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    b = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    a.set_tuning(fused_block=0)
    b.set_tuning(fused_block=128)
    a.step(900)
    b.step(900)
    sa, sb = _state(a), _state(b)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    removed = np.all(sa[2] == 0.0, axis=1) & np.all(sa[3] == 0.0, axis=1)
    assert removed.sum() > 0                # removed spheres keep zero velocities
    ca, cb = a.contacts(), b.contacts()
    for k in ("i", "j", "force"):
        assert np.array_equal(ca[k], cb[k])


def test_fused_step_in_a_batch_and_ignored_for_clumps():
    scenes = [W.dense_lattice(n=150 + 97 * k, seed=45 + k, vel_sigma=0.3) for k in range(3)]
    beta = 5e-5
    p = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    q = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    p.initialize()
    q.initialize()
    p.worlds[0].set_tuning(fused_block=0)
    q.worlds[0].set_tuning(fused_block=256)
    p.step(60)
    q.step(60)
    for wp, wq in zip(p.worlds, q.worlds):
        for x, y in zip(_state(wp), _state(wq)):
            assert np.array_equal(x, y)
    c = dem.World.from_scene(W.packed_clumps(n=100, seed=38), precision="voxel_fp32", schedule="every_step")
    c.set_tuning(fused_block=128)
    assert c.tuning()["fused_block"] == 0
    with pytest.raises(Exception):
        c.set_tuning(fused_block=96)


@pytest.mark.parametrize("prec", ["voxel_fp32", "fp64"])
@pytest.mark.parametrize("scene", ["dense", "clumps", "drum", "cone", "paddle"])
def test_counting_sort_binning_equals_radix_sort_binning(prec, scene):
    # the detection's two ways of ordering spheres by cell build the same contact lists
    # (rows sorted by partner), so the runs are the same bits: single spheres, clumps,
    # walls, a sink and turning facets, both schedules
    s = {"dense": lambda: W.dense_lattice(n=900, seed=39, vel_sigma=0.3),
         "clumps": lambda: W.packed_clumps(n=120, seed=40),
         "drum": lambda: W.drum_bed(n=150, seed=41),
         "cone": lambda: W.cone_bed(n=300, seed=13),
         "paddle": lambda: W.paddle_bed(n=300, seed=3)}[scene]()
    for sched in ("every_step", "velocity_bound"):
        runs = []
        for bn in (1, 2):
            w = dem.World.from_scene(s, precision=prec, schedule=sched)
            w.set_tuning(binning=bn)
            assert w.tuning()["binning"] == bn
            w.step(150)
            runs.append((_state(w), w.listed_pairs()[0].tolist(), w.listed_wall_pairs()[0].tolist(),
                         w.stats()["rebuilds"]))
        (sa, pa, wa, ra), (sb, pb, wb, rb) = runs
        for x, y in zip(sa, sb):
            assert np.array_equal(x, y)
        assert pa == pb and wa == wb and ra == rb


@pytest.mark.parametrize("prec", ["voxel_fp32", "fp64"])
@pytest.mark.parametrize("scene", ["dense", "clumps", "cone", "paddle", "families"])
def test_staged_narrow_phase_builds_the_same_lists(prec, scene):
    # the narrow phase reading its candidates from ranges staged in shared memory against
    # reading them from L1/L2: the same lists and the same runs, bit for bit
    s = {"dense": lambda: W.dense_lattice(n=900, seed=39, vel_sigma=0.3),
         "clumps": lambda: W.packed_clumps(n=120, seed=40),
         "cone": lambda: W.cone_bed(n=300, seed=13),
         "paddle": lambda: W.paddle_bed(n=300, seed=3),
         "families": lambda: W.dense_lattice(n=400, seed=47, vel_sigma=0.3)}[scene]()
    runs = []
    for staged in (0, 1):
        w = dem.World.from_scene(s, precision=prec, schedule="velocity_bound")
        if scene == "families":
            w.set_family(0, np.arange(s.n_owner) % 3)
            w.set_family_contacts(1, 2, False)
        w.set_tuning(narrow_staged=staged)
        assert w.tuning()["narrow_staged"] == staged
        w.step(120)
        runs.append((_state(w), w.listed_pairs()[0].tolist(), w.listed_wall_pairs()[0].tolist()))
    (sa, pa, wa), (sb, pb, wb) = runs
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    assert pa == pb and wa == wb and len(pa) > 0


def test_counting_sort_binning_with_families_in_a_batch():
    scenes = [W.dense_lattice(n=150 + 97 * k, seed=45 + k, vel_sigma=0.3) for k in range(3)]
    beta = 5e-5
    out = []
    for bn in (1, 2):
        b = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
        b.initialize()
        b.worlds[0].set_tuning(binning=bn)
        b.step(80)
        out.append([_state(w) for w in b.worlds])
    for wa, wb in zip(*out):
        for x, y in zip(wa, wb):
            assert np.array_equal(x, y)
    s = W.dense_lattice(n=400, seed=47, vel_sigma=0.3)
    fam = np.arange(s.n_owner) % 3
    res = []
    for bn in (1, 2):
        w = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
        w.set_family(0, fam)
        w.set_family_contacts(1, 2, False)
        w.set_tuning(binning=bn)
        w.step(100)
        res.append((_state(w), w.listed_pairs()[0].tolist()))
    for x, y in zip(res[0][0], res[1][0]):
        assert np.array_equal(x, y)
    assert res[0][1] == res[1][1]
    with pytest.raises(Exception):
        w.set_tuning(binning=3)


@pytest.mark.parametrize("prec", ["voxel_fp32", "fp64"])
def test_two_pass_contact_step_is_bit_identical(prec):
    # screening and evaluation passes against the single contact kernel: both schedules,
    # switched in mid-run; with a wide margin the rows pass 32 entries (the entry mask's
    # high word)
    for s, beta in ((W.dense_lattice(n=900, seed=37, vel_sigma=0.3), 5e-5),
                    (W.dense_lattice(n=700, seed=41, vel_sigma=0.3), 1.2e-3)):
        for sched in ("every_step", "velocity_bound"):
            kw = dict(precision=prec, schedule=sched, margin_max=beta)
            if sched != "every_step":
                kw["margin"] = beta
            a = dem.World.from_scene(s, **kw)
            a.set_tuning(fused_block=0, contact_integrates=0, contact_screen=0)
            for k in (50, 20, 50):
                a.step(k)
            b = dem.World.from_scene(s, **kw)
            b.set_tuning(fused_block=0, contact_integrates=0, contact_screen=1)
            assert b.tuning()["contact_screen"] == 1
            b.step(50)
            b.set_tuning(fused_block=0, contact_integrates=0, contact_screen=0)
            b.step(20)
            b.set_tuning(fused_block=0, contact_integrates=0, contact_screen=1)
            b.step(50)
            for x, y in zip(_state(b), _state(a)):
                assert np.array_equal(x, y)
            ca, cb = a.contacts(), b.contacts()
            assert len(ca["i"]) > 100
            for k in ca:
                assert np.array_equal(ca[k], cb[k]), k
            assert b.listed_pairs()[0].tolist() == a.listed_pairs()[0].tolist()
            sa, sb = a.stats(), b.stats()
            assert sa["audit_fallbacks"] == sb["audit_fallbacks"] and sa["rebuilds"] == sb["rebuilds"]
            if beta > 1e-4 and sched != "every_step":
                assert sb["list_max_row"] > 32      # the every-step lists use no margin


def test_two_pass_contact_step_with_a_sink_in_a_batch_and_ignored_for_clumps():
    s = W.cone_bed(n=300, seed=13)
    a = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    b = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound")
    a.set_tuning(fused_block=0, contact_integrates=0, contact_screen=0)
    b.set_tuning(fused_block=0, contact_integrates=0, contact_screen=1)
    a.step(900)
    b.step(900)
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    v = _state(b)[2]
    assert np.count_nonzero(np.all(v == 0.0, axis=1)) > 0     # the sink removed some
    scenes = [W.dense_lattice(n=150 + 97 * k, seed=45 + k, vel_sigma=0.3) for k in range(3)]
    beta = 5e-5
    p = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    q = dem.Batch(scenes, schedule="velocity_bound", margin=beta, margin_max=beta)
    p.initialize()
    q.initialize()
    p.worlds[0].set_tuning(fused_block=0, contact_integrates=0, contact_screen=0)
    q.worlds[0].set_tuning(fused_block=0, contact_integrates=0, contact_screen=1)
    p.step(60)
    q.step(60)
    for wp, wq in zip(p.worlds, q.worlds):
        for x, y in zip(_state(wp), _state(wq)):
            assert np.array_equal(x, y)
    c = dem.World.from_scene(W.packed_clumps(n=100, seed=38), precision="voxel_fp32", schedule="every_step")
    c.set_tuning(contact_screen=1)
    assert c.tuning()["contact_screen"] == 0
