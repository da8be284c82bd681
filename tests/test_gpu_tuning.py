"""GPU: captured CUDA graphs, launch shapes, detection placement and the autotuner change
timing only: every configuration gives bit-identical states."""
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
    b.set_tuning(contact_block=32, integrate_block=512, narrow_block=256, detect_inline=1)
    runs.append(b)
    c = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    c.set_tuning(contact_block=128, integrate_block=128, narrow_block=64, detect_inline=0)
    runs.append(c)
    for w in runs:
        w.step(150)
        for x, y in zip(_state(w), want):
            assert np.array_equal(x, y)


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
    assert t2["step_ms"] == pytest.approx(t["step_ms"], abs=1e-6)
    assert len(open(cache).read().strip().splitlines()) == 1
    # tuned runs continue exactly like untuned ones
    w.step(60)
    u = dem.World.from_scene(s, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    u.step(80)
    for x, y in zip(_state(w), _state(u)):
        assert np.array_equal(x, y)
