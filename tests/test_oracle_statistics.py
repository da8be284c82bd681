"""Pins of the bulk statistics (packing fraction, coordination) against closed forms, and of
the oracle's grid enumeration against its plain all-pairs loop."""
import math

import numpy as np
import pytest

import oracle
from oracle import statistics as S
from paper_2311_04648_gb300 import workloads as W

PI = math.pi


# ------------------------------------------------------------------ disc slices

def test_disc_inside_rectangle_is_the_full_disc():
    assert S.disc_rect_area(1.5, -2, 2, -3, 3) == pytest.approx(PI * 2.25, rel=1e-14)


@pytest.mark.parametrize("d", [-0.9, -0.3, 0.0, 0.25, 0.7, 0.99])
def test_disc_cut_by_one_line_is_a_circular_segment(d):
    r = 1.3
    dd = d * r
    seg = r * r * math.acos(dd / r) - dd * math.sqrt(r * r - dd * dd)     # part with x >= dd
    assert S.disc_rect_area(r, dd, 5, -5, 5) == pytest.approx(seg, rel=1e-13, abs=1e-15)
    assert S.disc_rect_area(r, -5, 5, dd, 5) == pytest.approx(seg, rel=1e-13, abs=1e-15)
    assert S.disc_rect_area(r, -5, -dd, -5, 5) == pytest.approx(seg, rel=1e-13, abs=1e-15)


def test_disc_quarter_and_inscribed_square():
    r = 0.8
    assert S.disc_rect_area(r, 0, 1, 0, 1) == pytest.approx(PI * r * r / 4, rel=1e-14)
    a = r / math.sqrt(2)
    assert S.disc_rect_area(r, -a, a, -a, a) == pytest.approx(4 * a * a, rel=1e-13)
    # a rectangle wholly inside the disc
    assert S.disc_rect_area(r, -0.3, 0.2, -0.1, 0.4) == pytest.approx(0.5 * 0.5, rel=1e-13)


def test_disc_rectangle_areas_add_up():
    rng = np.random.default_rng(11)
    for _ in range(50):
        r = rng.uniform(0.2, 2)
        x0, x1 = np.sort(rng.uniform(-2.5, 2.5, 2))
        y0, y1 = np.sort(rng.uniform(-2.5, 2.5, 2))
        xm = rng.uniform(x0, x1)
        whole = S.disc_rect_area(r, x0, x1, y0, y1)
        parts = S.disc_rect_area(r, x0, xm, y0, y1) + S.disc_rect_area(r, xm, x1, y0, y1)
        assert whole == pytest.approx(parts, rel=1e-12, abs=1e-14)


# ------------------------------------------------------------------ clipped balls

def test_ball_volumes_of_symmetric_cuts():
    R, c = 0.7, np.array([0.1, -0.2, 0.3])
    full = 4 / 3 * PI * R ** 3
    far = 10.0
    assert S.sphere_box_volume(c, R, c - far, c + far) == pytest.approx(full, rel=1e-14)
    lo, hi = c - far, c + far
    assert S.sphere_box_volume(c, R, [c[0], lo[1], lo[2]], hi) == pytest.approx(full / 2, rel=1e-12)
    assert S.sphere_box_volume(c, R, [c[0], c[1], lo[2]], hi) == pytest.approx(full / 4, rel=1e-12)
    assert S.sphere_box_volume(c, R, c, hi) == pytest.approx(full / 8, rel=1e-12)
    assert S.sphere_box_volume(c, R, c + R, hi) == 0.0


@pytest.mark.parametrize("h", [0.05, 0.3, 0.7, 1.1, 1.6])
def test_ball_cut_by_a_plane_is_a_spherical_cap(h):
    R = 0.8
    c = np.zeros(3)
    cap = PI * h * h * (3 * R - h) / 3
    for axis in range(3):
        lo = -10 * np.ones(3)
        lo[axis] = R - h
        assert S.sphere_box_volume(c, R, lo, 10 * np.ones(3)) == pytest.approx(cap, rel=1e-12)


def test_ball_slab_between_two_planes():
    R, z0, z1 = 1.0, -0.35, 0.6
    slab = PI * (R * R * (z1 - z0) - (z1 ** 3 - z0 ** 3) / 3)
    assert S.sphere_box_volume([0, 0, 0], R, [-5, -5, z0], [5, 5, z1]) == pytest.approx(slab, rel=1e-12)


def test_cube_inside_the_ball_is_the_cube():
    # corners at distance sqrt(3) * 0.5 < 1: the clipped ball is the cube itself
    assert S.sphere_box_volume([0, 0, 0], 1.0, [-0.5] * 3, [0.5] * 3) == pytest.approx(1.0, rel=1e-12)
    # an off-centre box with every corner inside the ball
    lo, hi = np.array([-0.2, -0.5, 0.1]), np.array([0.4, 0.3, 0.6])
    assert S.sphere_box_volume([0, 0, 0], 1.0, lo, hi) == pytest.approx(float(np.prod(hi - lo)), rel=1e-12)


def test_clipped_ball_volumes_add_up():
    rng = np.random.default_rng(12)
    for _ in range(25):
        R = rng.uniform(0.3, 1.0)
        lo = rng.uniform(-1.2, 0.0, 3)
        hi = rng.uniform(0.0, 1.2, 3)
        axis = int(rng.integers(3))
        m = rng.uniform(lo[axis], hi[axis])
        hi_a, lo_b = hi.copy(), lo.copy()
        hi_a[axis] = m
        lo_b[axis] = m
        whole = S.sphere_box_volume([0, 0, 0], R, lo, hi)
        parts = S.sphere_box_volume([0, 0, 0], R, lo, hi_a) + S.sphere_box_volume([0, 0, 0], R, lo_b, hi)
        assert whole == pytest.approx(parts, rel=1e-11, abs=1e-15)


def test_simple_cubic_lattice_packs_pi_over_six():
    a, k = 2.0e-3, 4
    g = np.arange(k + 1) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    centres = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    radii = np.full(len(centres), a / 2)
    phi = S.packing_fraction(centres, radii, [0, 0, 0], [k * a] * 3)
    assert phi == pytest.approx(PI / 6, rel=1e-11)


def test_coordination_counts_each_contact_at_both_ends():
    centres = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [5, 5, 5]], np.float64)
    ci = np.array([0, 1, 0, 2])
    cj = np.array([1, 2, -1, -3])        # two wall contacts, ignored
    z, n = S.coordination(centres, ci, cj, [-0.5] * 3, [2.5, 0.5, 0.5])
    assert n == 3 and z == pytest.approx(4 / 3)


# ------------------------------------------------------------------ oracle grid enumeration

def _same_run(scene, steps):
    a = oracle.OracleWorld(scene, cell_list=True)
    b = oracle.OracleWorld(scene)
    assert a.step(steps) == 0 and b.step(steps) == 0
    for f in ("x", "v", "wb", "q", "active"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    ha, hb = a.history(), b.history()
    for u, w in zip(ha, hb):
        assert np.array_equal(u, w)
    return len(ha[0])


def test_grid_enumeration_is_bit_identical_for_colliding_spheres():
    sc = W.settling_column(n=1500, column_width=0.02, vel_sigma=0.4, seed=21)
    assert _same_run(sc, 200) > 20


def test_grid_enumeration_is_bit_identical_for_clumps_and_walls():
    sc = W.packed_clumps(n=300, seed=22)
    assert _same_run(sc, 150) > 20


def test_grid_enumeration_is_bit_identical_with_a_sink():
    sc = W.cone_bed(n=600, seed=23)
    a = oracle.OracleWorld(sc, cell_list=True)
    b = oracle.OracleWorld(sc)
    assert a.step(1000) == 0 and b.step(1000) == 0
    assert (a.active == 0).sum() > 0          # the sink has removed owners
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.active, b.active)


# ------------------------------------------------------------------ oracle threads

def _same_run_threads(scene, steps, cell_list):
    a = oracle.OracleWorld(scene, cell_list=cell_list, threads=4)
    b = oracle.OracleWorld(scene, cell_list=cell_list)
    assert a.step(steps) == 0 and b.step(steps) == 0
    for f in ("x", "v", "wb", "q", "active"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    ha, hb = a.history(), b.history()
    for u, w in zip(ha, hb):
        assert np.array_equal(u, w)
    Fa, Ta, ca = a.eval()
    Fb, Tb, cb = b.eval()
    assert np.array_equal(Fa, Fb) and np.array_equal(Ta, Tb) and np.array_equal(ca, cb)
    return len(ha[0])


@pytest.mark.parametrize("cell_list", [False, True])
def test_threaded_oracle_is_bit_identical_for_clumps_and_walls(cell_list):
    """Contacts found on four threads, reduced serially: the one-thread results."""
    assert _same_run_threads(W.packed_clumps(n=300, seed=22), 120, cell_list) > 20


def test_threaded_oracle_is_bit_identical_with_a_sink():
    sc = W.cone_bed(n=600, seed=23)
    a = oracle.OracleWorld(sc, cell_list=True, threads=4)
    b = oracle.OracleWorld(sc, cell_list=True)
    assert a.step(1000) == 0 and b.step(1000) == 0
    assert (a.active == 0).sum() > 0
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.active, b.active)


def test_history_set_sorts_unsorted_entries():
    sc = W.packed_clumps(n=100, seed=24)
    ow = oracle.OracleWorld(sc)
    assert ow.step(60) == 0
    i, j, ut = ow.history()
    assert len(i) > 5
    perm = np.random.default_rng(1).permutation(len(i))
    ow2 = oracle.OracleWorld(sc)
    ow2.set_history(i[perm], j[perm], ut[perm])
    i2, j2, ut2 = ow2.history()
    assert np.array_equal(i, i2) and np.array_equal(j, j2) and np.array_equal(ut, ut2)
