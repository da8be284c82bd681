"""The seeded input generators against the recipes they implement: sizes, value ranges,
no overlap at the start, every sphere inside its container.  Overlaps are checked with the
oracle's brute-force listed set at zero margin, or along the lattice where the workload is
too large for that."""
import math

import numpy as np

import oracle
from paper_2311_04648_gb300 import workloads as W


def radii(scene):
    return np.asarray(scene.owner_scale, np.float64) * 1e-3      # single-sphere templates of R = 1 mm


def test_settling_column_at_full_size_follows_its_recipe():
    s = W.settling_column()                      # 4,000,000 spheres, the bench workload
    n = 4_000_000
    assert s.n_owner == n and s.n_sphere == n
    assert s.meta["nx"] == 122 and s.meta["ny"] == 122 and s.meta["layers"] == 269
    r = radii(s)
    assert 0.8e-3 <= r.min() and r.max() <= 1.2e-3
    x = np.asarray(s.x)
    # the outer lattice sites sit R_max from the walls, moved by up to the 0.02 mm jitter
    assert np.all(x - r[:, None] > s.box_lo - 0.02e-3) and np.all(x + r[:, None] < s.box_hi + 0.02e-3)
    assert 0.6 < x[:, 2].max() < 0.7                                    # ~0.66 m of column
    assert abs(np.std(np.asarray(s.v)) - 0.05) < 1e-3
    # no overlap: the nearest sites are the lattice neighbours along x, y and z
    nx, per = s.meta["nx"], s.meta["nx"] * s.meta["ny"]
    idx = np.arange(n)
    for step, same_line in ((1, idx % nx != nx - 1), (nx, (idx % per) // nx != s.meta["ny"] - 1), (per, None)):
        i = idx[: n - step]
        if same_line is not None:
            i = i[same_line[: n - step]]
        d = np.linalg.norm(x[i + step] - x[i], axis=1)
        assert np.all(d > r[i] + r[i + step])


def test_cone_hopper_spheres_start_inside_the_cone_without_overlap():
    s = W.cone_hopper(n=5000)
    r = radii(s)
    x = np.asarray(s.x)
    cone = s.walls[0]
    assert cone["type"] == W.CONE and cone["r0"] == 10 * 2e-3            # orifice 10 R_max
    tan = math.tan(math.radians(30.0))
    rho = np.hypot(x[:, 0], x[:, 1])
    # distance to the wall in the (rho, z) half plane, the wall 30 degrees from vertical
    gap = (cone["r0"] + x[:, 2] * tan - rho) * math.cos(math.radians(30.0))
    assert np.all(gap > r)
    pi, pj = oracle.listed_pairs_f64(x, r, np.arange(len(r)), 0.0)
    assert len(pi) == 0


def test_clump_drum_clumps_start_inside_the_drum_without_overlap():
    s = W.clump_drum(n_clumps=3000)
    ow = oracle.OracleWorld(s)
    p = ow.sphere_positions()
    rad = ow.rad
    assert len(s.templates) == 2 and {len(t.radii) for t in s.templates} == {3, 4}   # rods, tetrahedra
    comp = np.asarray(s.owner_scale) * 1e-3
    assert 1e-3 <= comp.min() and comp.max() <= 2e-3
    radial = np.hypot(p[:, 1], p[:, 2])
    assert np.all(radial + rad < 0.6)
    half = s.meta["length"] / 2
    assert np.all(np.abs(p[:, 0]) + rad < half)
    pi, pj = oracle.listed_pairs_f64(p, rad, ow.owner, 0.0)          # spheres of different clumps
    assert len(pi) == 0


def test_batch_scenes_follow_their_distributions():
    scenes = W.batch_scenes()
    assert len(scenes) == 512
    counts = np.array([sc.n_owner for sc in scenes])
    assert counts.min() >= 1000 and counts.max() <= 50_000
    # log-uniform on [1e3, 5e4]: mean (5e4 - 1e3) / ln 50 = 12.5k per scene
    assert abs(counts.mean() / ((5e4 - 1e3) / math.log(50.0)) - 1.0) < 0.1
    mu = np.array([float(np.asarray(sc.mu).ravel()[0]) for sc in scenes])
    e = np.array([float(np.asarray(sc.cor).ravel()[0]) for sc in scenes])
    aspect = np.array([sc.meta["aspect"] for sc in scenes])
    assert 0.2 <= mu.min() and mu.max() <= 0.8
    assert 0.3 <= e.min() and e.max() <= 0.9
    assert 0.5 <= aspect.min() and aspect.max() <= 4.0
    for sc in scenes[:8]:                        # no overlap at the start
        r = radii(sc)
        assert 0.9e-3 <= r.min() and r.max() <= 1.1e-3
        pi, _ = oracle.listed_pairs_f64(np.asarray(sc.x), r, np.arange(len(r)), 0.0)
        assert len(pi) == 0


def test_mixer_bed_starts_clear_of_blades_hub_floor_and_container():
    # the bed start of the Sec. 5 mixer: every element inside the container, above the
    # floor and clear of the 2,892 facets at their pose at t = 0 (the oracle's brute-force
    # sphere-wall listing at zero margin), for spheres and three-sphere rods
    for clump, n in (("sphere", 20_000), ("rod3", 8_000)):
        s = W.mixer(n=n, clump=clump, start="bed")
        assert s.n_owner == n and s.meta["start"] == "bed"
        assert sum(1 for w in s.walls if w["type"] == W.TRIANGLE) == 2892
        ow = oracle.OracleWorld(s, threads=oracle.max_threads())
        p = ow.sphere_positions()
        si, wi = ow.listed_wall_pairs(p, 0.0)
        assert len(si) == 0
        assert p[:, 2].min() > 0.0 and np.hypot(p[:, 0], p[:, 1]).max() < 0.5
        # the bed reaches down among the blades (z from 0.02 to 0.12 m)
        assert np.sum(p[:, 2] < 0.12) > n // 10
