"""Pins of the FP64 CPU oracle to what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a closed form, an
invariant, a special case or a brute-force enumeration that a plausible mistake in the
oracle (dropped term, wrong sign or index, transposed operand) would break.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_2311_04648_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def one_material(E=1e7, nu=0.3, e=0.5, mu=0.4):
    return (np.array([E]), np.array([nu]), np.array([[e]]), np.array([[mu]]))


def make_scene(x, v=None, wb=None, q=None, templates=None, owner_t=None, scale=None, walls=(), g=(0, 0, 0),
               h=1e-6, mat=one_material(), **kw):
    x = np.asarray(x, np.float64).reshape(-1, 3)
    M = len(x)
    if templates is None:
        templates = [W.sphere_template(1e-3)]
    if owner_t is None:
        owner_t = np.zeros(M, np.int64)
    if q is None:
        q = np.zeros((M, 4)); q[:, 0] = 1
    v = np.zeros((M, 3)) if v is None else np.asarray(v, np.float64).reshape(M, 3)
    wb = np.zeros((M, 3)) if wb is None else np.asarray(wb, np.float64).reshape(M, 3)
    E, nu, cor, mu = mat
    return W.Scene(np.full(3, -1.0), np.full(3, 1.0), E, nu, cor, mu, list(walls), templates,
                   np.asarray(owner_t, np.int64), scale, x, np.asarray(q, np.float64), v, wb, h,
                   np.asarray(g, np.float64), **kw)


# ----------------------------------------------------------------------------- pairs

def numpy_pairs(p, rad, owner, beta):
    n = len(rad)
    out = []
    for i in range(n):
        d = p[i] - p[i + 1:]
        s = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        t = (rad[i] + rad[i + 1:]) + 2.0 * beta
        hit = (s < t * t) & (owner[i + 1:] != owner[i])
        for j in np.nonzero(hit)[0]:
            out.append((i, i + 1 + j))
    return out


def test_listed_pairs_match_direct_enumeration():
    rng = np.random.default_rng(11)
    n = 400
    p = rng.uniform(0, 0.02, size=(n, 3))
    rad = rng.uniform(0.8e-3, 1.2e-3, size=n)
    owner = np.arange(n) // 3            # clumps of 3 spheres: same-owner pairs excluded
    for beta in (0.0, 5e-5):
        pi, pj = oracle.listed_pairs_f64(p, rad, owner, beta)
        got = list(zip(pi.tolist(), pj.tolist()))
        assert got == numpy_pairs(p, rad, owner, beta)
        assert len(got) > 100
        assert got == sorted(got)


def test_listed_pairs_voxel_f32_matches_float32_enumeration():
    rng = np.random.default_rng(12)
    n = 300
    L = np.float32(2.5e-3)
    cell = rng.integers(0, 6, size=(n, 3)).astype(np.int32)
    off = (rng.random((n, 3)) * float(L)).astype(np.float32)
    rad = rng.uniform(0.8e-3, 1.2e-3, size=n).astype(np.float32)
    owner = np.arange(n)
    beta = np.float32(5e-5)
    pi, pj = oracle.listed_pairs_voxel_f32(cell, off, L, rad, owner, beta)
    want = []
    for i in range(n):
        dc = (cell[i] - cell[i + 1:]).astype(np.float32)
        d = dc * L + (off[i] - off[i + 1:])
        s = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        t = (rad[i] + rad[i + 1:]) + np.float32(2) * beta
        for j in np.nonzero(s < t * t)[0]:
            want.append((i, i + 1 + j))
    assert list(zip(pi.tolist(), pj.tolist())) == want
    # the FP64 set on the same positions differs only for pairs within rounding of the threshold
    p64 = cell.astype(np.float64) * float(L) + off.astype(np.float64)
    qi, qj = oracle.listed_pairs_f64(p64, rad.astype(np.float64), owner, float(beta))
    a = set(zip(pi.tolist(), pj.tolist()))
    b = set(zip(qi.tolist(), qj.tolist()))
    for (i, j) in a ^ b:
        d = np.linalg.norm(p64[i] - p64[j])
        t = float(rad[i]) + float(rad[j]) + 2 * float(beta)
        assert abs(d - t) < 1e-6 * t


def test_contacts_are_the_listed_set_at_zero_margin_and_inside_any_margin():
    s = W.settle_box(n=250, box=(0.015, 0.015, 0.015), seed=5, gap=-2e-4)  # overlapping placement
    ow = oracle.OracleWorld(s)
    p = ow.sphere_positions()
    F, T, cs = ow.eval()
    sph = cs[cs["j"] >= 0]
    contact = set(zip(sph["i"].tolist(), sph["j"].tolist()))
    assert len(contact) > 50
    assert np.all(sph["overlap"] > 0)
    li, lj = oracle.listed_pairs_f64(p, ow.rad, ow.owner, 1e-5)
    assert contact <= set(zip(li.tolist(), lj.tolist()))
    # every listed pair at zero margin with a strictly positive overlap is a contact
    li0, lj0 = oracle.listed_pairs_f64(p, ow.rad, ow.owner, 0.0)
    for i, j in zip(li0.tolist(), lj0.tolist()):
        d = np.linalg.norm(p[i] - p[j])
        if (ow.rad[i] + ow.rad[j]) - d > 0:
            assert (i, j) in contact


# ----------------------------------------------------------------------------- Hertz head-on

def headon_run(v0, e, R=1e-3, E=1e7, nu=0.3, steps_per_tc=4000, rho=W.RHO):
    m = rho * 4 / 3 * math.pi * R ** 3
    mbar = m / 2
    Rbar = R / 2
    Es = E / (2 * (1 - nu ** 2))
    tc = 2.868 * (mbar ** 2 / (Rbar * Es ** 2 * v0)) ** 0.2
    h = tc / steps_per_tc
    s = W.two_spheres(R=R, v0=v0, E=E, nu=nu, e=e, h=h, gap=0.0, rho=rho)
    s.x[0, 0] += 0.0
    ow = oracle.OracleWorld(s)
    dmax = 0.0
    t_in = None
    t_out = None
    for k in range(4 * steps_per_tc):
        F, T, cs = ow.eval()
        if len(cs):
            dmax = max(dmax, float(cs["overlap"].max()))
            if t_in is None:
                t_in = k * h
        elif t_in is not None:
            t_out = k * h
            break
        ow.step(1)
    vrel = ow.v[1, 0] - ow.v[0, 0]
    return dict(dmax=dmax, tc=t_out - t_in, e_out=vrel / v0, mbar=mbar, Rbar=Rbar, Es=Es, h=h)


def test_hertz_headon_undamped_matches_closed_form():
    """Hertz impact: delta_max = (15 mbar v0^2 / (16 E* sqrt(Rbar)))^(2/5) and duration
    t_c = 2 (delta_max / v0) * (2/5) B(2/5, 1/2); restitution 1 without damping."""
    v0 = 1.0
    r = headon_run(v0, e=1.0)
    dmax = (15 * r["mbar"] * v0 ** 2 / (16 * r["Es"] * math.sqrt(r["Rbar"]))) ** 0.4
    beta_fn = math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
    tc = 2 * dmax / v0 * 0.4 * beta_fn
    assert r["dmax"] == pytest.approx(dmax, rel=2e-3)
    assert r["tc"] == pytest.approx(tc, rel=2e-3)
    assert r["e_out"] == pytest.approx(1.0, abs=2e-3)
    # the worked numbers for this material at 1 m/s: delta_max ~ 7.0e-5 m, t_c ~ 2.07e-4 s
    assert dmax == pytest.approx(7.05e-5, rel=1e-2)
    assert tc == pytest.approx(2.07e-4, rel=1e-2)


def ode_restitution(e, v0, mbar, Rbar, Es):
    """Normal-only 1-D impact in the overlap x: the normal force on A is
    k_n x + g_n (u.n) with u.n = -x' (A approaches B against the normal), so
    m x'' = -(k_n(x) x - g_n(x) x'), integrated by classical RK4 with 2e5 steps per
    contact: an independent integrator for the oracle's first-order 3-D step."""
    le = math.log(max(e, 1e-12))
    b = le / math.sqrt(le * le + math.pi ** 2)

    def acc(x, xd):
        if x <= 0:
            return 0.0
        sn = 2 * Es * math.sqrt(Rbar * x)
        kn = 2.0 / 3.0 * sn
        gn = 2 * math.sqrt(5.0 / 6.0) * b * math.sqrt(sn * mbar)
        return -(kn * x - gn * xd) / mbar

    tc = 2.868 * (mbar ** 2 / (Rbar * Es ** 2 * v0)) ** 0.2
    n = 200_000
    h = 2 * tc / n
    x, xd = 0.0, v0
    for _ in range(n):
        k1x, k1v = xd, acc(x, xd)
        k2x, k2v = xd + 0.5 * h * k1v, acc(x + 0.5 * h * k1x, xd + 0.5 * h * k1v)
        k3x, k3v = xd + 0.5 * h * k2v, acc(x + 0.5 * h * k2x, xd + 0.5 * h * k2v)
        k4x, k4v = xd + h * k3v, acc(x + h * k3x, xd + h * k3v)
        x += h / 6 * (k1x + 2 * k2x + 2 * k3x + k4x)
        xd += h / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
        if x < 0 and xd < 0:
            break
    return -xd / v0


@pytest.mark.slow
def test_hertz_headon_damped_velocity_independent_and_matches_1d_solve():
    """The damping of Sec. 4.1 scales as delta^(1/4), which makes the outcome independent of
    the impact speed; the 3-D oracle must converge to the 1-D normal impact."""
    outs = [headon_run(v0, e=0.5, steps_per_tc=2000) for v0 in (0.1, 1.0, 5.0)]
    es = [o["e_out"] for o in outs]
    assert max(es) - min(es) < 1e-3
    assert 0.4 < es[0] < 1.0
    r = outs[1]
    e_ode = ode_restitution(0.5, 1.0, r["mbar"], r["Rbar"], r["Es"])
    assert es[1] == pytest.approx(e_ode, abs=2e-3)
    # monotone in the input restitution coefficient
    e_lo = headon_run(1.0, e=0.2, steps_per_tc=2000)["e_out"]
    e_hi = headon_run(1.0, e=0.8, steps_per_tc=2000)["e_out"]
    assert e_lo < es[1] < e_hi < 1.0


def test_mixer_material_restitution_velocity_independent():
    gm = read_golden("mixer_material_sec5.txt")
    rs = [headon_run(v0, e=gm["cor"], E=gm["E_pa"], nu=gm["nu"], rho=gm["density_kgpm3"], steps_per_tc=1500)["e_out"]
          for v0 in (0.5, 2.0)]
    assert abs(rs[0] - rs[1]) < 1e-3
    assert 0.0 < rs[0] < 1.0


# ----------------------------------------------------------------------------- balance laws

def test_linear_and_angular_momentum_conserved_without_walls():
    s = W.free_spheres(n=150, box=0.0135, vel_sigma=0.8, seed=3, h=2e-6)
    ow = oracle.OracleWorld(s)
    d0 = ow.diagnostics()
    m = ow.mass
    scale_p = float(np.sum(m * np.linalg.norm(ow.v, axis=1)))
    scale_l = float(np.sum(np.linalg.norm(np.cross(ow.x, m[:, None] * ow.v), axis=1))) + \
        float(np.sum(ow.moi[:, 0] * np.linalg.norm(ow.wb, axis=1)))
    ncont = 0
    for _ in range(10):
        ow.step(40)
        ncont += len(ow.eval()[2])
    assert ncont > 20
    d1 = ow.diagnostics()
    assert np.max(np.abs(d1["momentum"] - d0["momentum"])) < 1e-12 * scale_p
    assert np.max(np.abs(d1["angmom"] - d0["angmom"])) < 1e-11 * scale_l


def test_energy_conserved_when_elastic_and_frictionless():
    s = W.settle_box(n=150, box=(0.0135, 0.0135, 0.0135), seed=4, vel_sigma=0.3, e=1.0, mu=0.0, h=2e-7, gap=1e-5)
    ow = oracle.OracleWorld(s)

    def emech():
        d = ow.diagnostics()
        return d["ke"] + d["pe"] + d["elastic"]

    ke0 = ow.diagnostics()["ke"]
    e0 = emech()
    worst = 0.0
    for _ in range(20):
        ow.step(100)
        worst = max(worst, abs(emech() - e0))
    assert worst < 1e-3 * ke0


def test_energy_non_increasing_with_damping_and_friction():
    s = W.settle_box(n=150, box=(0.0135, 0.0135, 0.0135), seed=4, vel_sigma=0.3, e=0.5, mu=0.4, h=5e-7, gap=1e-5)
    ow = oracle.OracleWorld(s)
    d = ow.diagnostics()
    prev = d["ke"] + d["pe"] + d["elastic"]
    e0 = abs(prev)
    first = prev
    for _ in range(20):
        ow.step(50)
        d = ow.diagnostics()
        cur = d["ke"] + d["pe"] + d["elastic"]
        assert cur <= prev + 1e-6 * e0
        prev = cur
    assert prev < first - 1e-3 * abs(first)


# ----------------------------------------------------------------------------- statics

def test_static_stack_settles_to_hertz_overlaps():
    """A vertical column of k spheres on a floor: the contact under n spheres carries
    W = n m g and settles to delta = (3 W / (4 E* sqrt(Rbar)))^(2/3), with Rbar = R/2
    between spheres and Rbar = R at the floor (wall curvature infinite)."""
    k, R, E, nu, g = 5, 1e-3, 1e7, 0.3, 9.81
    x = np.array([[0.0, 0.0, R + 2 * R * i] for i in range(k)])
    floor = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    s = make_scene(x, walls=[floor], g=(0, 0, -g), h=1e-6, mat=one_material(E=E, nu=nu, e=0.1, mu=0.3))
    ow = oracle.OracleWorld(s)
    ow.step(120000)
    F, T, cs = ow.eval()
    m = ow.mass[0]
    Es_ss = E / (2 * (1 - nu ** 2))
    Es_sw = E / (2 * (1 - nu ** 2))          # wall made of the same material
    got = {}
    for c in cs:
        got[(int(c["i"]), int(c["j"]))] = float(c["overlap"])
    for i in range(k - 1):
        Wn = (k - 1 - i) * m * g
        want = (3 * Wn / (4 * Es_ss * math.sqrt(R / 2))) ** (2 / 3)
        assert got[(i, i + 1)] == pytest.approx(want, rel=1e-6)
    want_floor = (3 * k * m * g / (4 * Es_sw * math.sqrt(R))) ** (2 / 3)
    assert got[(0, -1)] == pytest.approx(want_floor, rel=1e-6)
    assert np.max(np.abs(ow.v)) < 1e-9


# ----------------------------------------------------------------------------- friction

def incline_run(alpha_deg, t_end=1.5):
    gd = read_golden("incline_sec4_3_1.txt")
    r, m, mu = gd["radius_m"], gd["mass_kg"], gd["mu"]
    rho = m / (4 / 3 * math.pi * r ** 3)
    tpl = W.sphere_template(r, rho=rho)
    a = math.radians(alpha_deg)
    g = 9.81 * np.array([-math.sin(a), 0.0, -math.cos(a)])
    Es = gd["E_pa"] / (2 * (1 - gd["nu"] ** 2))
    d0 = (3 * m * 9.81 * math.cos(a) / (4 * Es * math.sqrt(r))) ** (2 / 3)
    x = np.array([[0.0, 0.0, r - d0]])
    plane = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    h = 2e-5
    s = make_scene(x, v=[[gd["v0_up_incline_mps"], 0, 0]], templates=[tpl], walls=[plane], g=g, h=h,
                   mat=one_material(E=gd["E_pa"], nu=gd["nu"], e=gd["cor"], mu=mu))
    ow = oracle.OracleWorld(s)
    ts, vs, slips, arms = [], [], [], []
    n = int(t_end / h)
    for k in range(0, n, 50):
        ow.step(50)
        qw, qx, qy, qz = ow.q[0]
        Rm = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
                       [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
                       [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])
        wg = Rm @ ow.wb[0]
        F, T, cs = ow.eval()
        # slip = velocity of the material point of the sphere at the contact point
        arm = np.array(cs["point"][0]) - ow.x[0]
        ts.append((k + 50) * h)
        vs.append(ow.v[0, 0])
        slips.append(ow.v[0, 0] + np.cross(wg, arm)[0])
        arms.append(np.linalg.norm(arm))
    return np.array(ts), np.array(vs), np.array(slips), mu, a, float(np.mean(arms[len(arms) // 2:])), r


@pytest.mark.parametrize("alpha", [30.0, 38.0])
def test_incline_below_threshold_ends_in_pure_rolling(alpha):
    """Sec. 4.3.1 with C_r = 0: pure rolling iff tan(alpha) <= 3.5 mu; rolling down an
    incline accelerates at (5/7) g sin(alpha)."""
    ts, vs, slips, mu, a, arm, r = incline_run(alpha)
    assert math.tan(a) < 3.5 * mu
    late = ts > ts[-1] * 0.6
    assert np.max(np.abs(slips[late])) < 1e-3 * np.max(np.abs(vs[late]))
    acc = np.polyfit(ts[late], vs[late], 1)[0]
    assert acc == pytest.approx(-5.0 / 7.0 * 9.81 * math.sin(a), rel=5e-3)


@pytest.mark.parametrize("alpha", [45.0, 55.0])
def test_incline_above_threshold_slips_at_the_coulomb_rate(alpha):
    """Above the threshold the contact slides: the slip speed at the contact point grows at
    g (sin(alpha) - mu cos(alpha) (1 + a^2 / (2/5 r^2))) for Coulomb friction mu N acting
    at the lever arm a (= r minus half the overlap; 3.5 mu for a = r), MOI 2/5 m r^2."""
    ts, vs, slips, mu, a, arm, r = incline_run(alpha)
    assert math.tan(a) > 3.5 * mu
    late = ts > ts[-1] * 0.5
    rate = np.polyfit(ts[late], slips[late], 1)[0]
    want = -9.81 * (math.sin(a) - mu * math.cos(a) * (1 + arm * arm / (0.4 * r * r)))
    assert rate == pytest.approx(want, rel=2e-3)
    acc = np.polyfit(ts[late], vs[late], 1)[0]
    assert acc == pytest.approx(-9.81 * (math.sin(a) - mu * math.cos(a)), rel=1e-2)


def test_history_lifetime_created_at_zero_and_dropped_on_separation():
    """Contact wildcards (Sec. 4.2): allocated at zero when a contact appears, freed when it
    vanishes.  An oblique frictional graze builds a history which disappears after."""
    R = 1e-3
    x = np.array([[0.0, 0.0, 0.0], [2 * R + 1e-7, 0.3 * R, 0.0]])
    s = make_scene(x, v=[[0.5, 0, 0], [-0.5, 0, 0]], h=1e-7, mat=one_material(e=0.5, mu=0.5))
    ow = oracle.OracleWorld(s)
    seen = False
    for _ in range(6000):
        ow.step(1)
        i, j, ut = ow.history()
        if len(i):
            seen = True
            assert (i[0], j[0]) == (0, 1)
            assert np.abs(ut[0, 2]) < 1e-15 and np.linalg.norm(ut[0]) > 0
        elif seen:
            break
    assert seen
    assert len(ow.history()[0]) == 0
    # the history is orthogonal to the current normal after every update
    F, T, cs = ow.eval()
    assert len(cs) == 0


# ----------------------------------------------------------------------------- rigid bodies

def test_torque_free_symmetric_top_precesses_at_euler_rate():
    """Euler's equations for I2 = I3: omega_1 is constant and (omega_2, omega_3) rotates at
    lambda = (I2 - I1) omega_1 / I2; the gyroscopic sign decides the direction."""
    tpl = W.rod_template(1e-3)
    I1, I2 = tpl.moi[0], tpl.moi[1]
    w0 = np.array([200.0, 30.0, 0.0])
    h = 1e-6
    s = make_scene([[0, 0, 0]], wb=[w0], templates=[tpl], h=h)
    ow = oracle.OracleWorld(s)
    d0 = ow.diagnostics()
    n = 20000
    ow.step(n)
    t = n * h
    lam = (I2 - I1) * w0[0] / I2
    want = np.array([w0[0], w0[1] * math.cos(lam * t), -w0[1] * math.sin(lam * t)])
    assert np.allclose(ow.wb[0], want, atol=2e-3 * np.linalg.norm(w0))
    d1 = ow.diagnostics()
    assert np.linalg.norm(d1["angmom"]) == pytest.approx(np.linalg.norm(d0["angmom"]), rel=1e-3)


def test_quaternion_rotation_about_a_principal_axis_is_exact():
    """Constant body rate about a principal axis: after n steps the orientation is the
    rotation by n h |omega| about that axis (each step composes an exact rotation)."""
    tpl = W.rod_template(1e-3)
    w = 37.0
    h = 1e-5
    s = make_scene([[0, 0, 0]], wb=[[0.0, 0.0, w]], templates=[tpl], h=h)
    ow = oracle.OracleWorld(s)
    n = 5000
    ow.step(n)
    ang = n * h * w
    want = np.array([math.cos(ang / 2), 0.0, 0.0, math.sin(ang / 2)])
    assert np.allclose(ow.q[0], want, atol=1e-12)
    # a sphere offset rotates with the body: local +x goes to (cos, sin, 0)
    p = ow.sphere_positions()
    assert np.allclose(p[2], [2e-3 * math.cos(ang), 2e-3 * math.sin(ang), 0.0], atol=1e-15)


def test_clump_mass_properties_are_the_parallel_axis_sums():
    R = 1e-3
    for tpl in (W.rod_template(R), W.tetra_template(R)):
        m1 = W.RHO * 4 / 3 * math.pi * R ** 3
        I = np.zeros((3, 3))
        for c in tpl.rel_xyz:
            I += 0.4 * m1 * R * R * np.eye(3) + m1 * (np.dot(c, c) * np.eye(3) - np.outer(c, c))
        assert np.allclose(np.diag(I), tpl.moi, rtol=1e-12)
        assert np.allclose(I - np.diag(np.diag(I)), 0, atol=1e-20)
        assert np.allclose(tpl.rel_xyz.sum(axis=0), 0, atol=1e-18)
        d = np.linalg.norm(tpl.rel_xyz[:, None] - tpl.rel_xyz[None], axis=-1)
        assert np.isclose(np.min(d[d > 0]), 2 * R)


# ----------------------------------------------------------------------------- walls

def test_sphere_resting_on_plane_and_in_drum_settles_to_hertz_overlap():
    R, E, nu, g = 1e-3, 1e7, 0.3, 9.81
    Es = E / (2 * (1 - nu ** 2))
    m = W.RHO * 4 / 3 * math.pi * R ** 3
    want = (3 * m * g / (4 * Es * math.sqrt(R))) ** (2 / 3)
    plane = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    drum = dict(type=W.CYLINDER, mat=0, p=np.zeros(3), n=np.array([1.0, 0.0, 0.0]), r0=0.05)
    for wall, x0 in ((plane, [0.0, 0.0, R]), (drum, [0.0, 0.0, -0.05 + R])):
        s = make_scene([x0], walls=[wall], g=(0, 0, -g), h=1e-6, mat=one_material(E=E, nu=nu, e=0.1, mu=0.3))
        ow = oracle.OracleWorld(s)
        ow.step(120000)
        F, T, cs = ow.eval()
        assert len(cs) == 1 and cs["j"][0] == -1
        assert cs["overlap"][0] == pytest.approx(want, rel=1e-6)


def test_spinning_wall_drags_a_resting_sphere_along_its_surface_velocity():
    R = 1e-3
    plane = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]), omega=np.array([0, 0, 5.0]))
    s = make_scene([[0.01, 0.0, R - 1e-6]], walls=[plane], g=(0, 0, -9.81), h=1e-6)
    ow = oracle.OracleWorld(s)
    ow.step(200)
    vwall = np.cross([0, 0, 5.0], [0.01, 0.0, 0.0])          # +y at this point
    assert ow.v[0, 1] > 0 and abs(ow.v[0, 0]) < 1e-3 * ow.v[0, 1]
    assert np.dot(ow.v[0], vwall) > 0


def cone_min_distance(pt, r0, z0, r1, z1, nseg=4000):
    z = pt[2]
    rho = math.hypot(pt[0], pt[1])
    lo, hi = 0.0, 1.0
    for _ in range(3):                   # sample, then resample around the best point
        t = np.linspace(lo, hi, nseg)
        d = np.hypot(rho - (r0 + t * (r1 - r0)), z - (z0 + t * (z1 - z0)))
        k = int(np.argmin(d))
        step = (hi - lo) / (nseg - 1)
        lo, hi = max(0.0, t[k] - 2 * step), min(1.0, t[k] + 2 * step)
    return float(d[k])


def test_cone_wall_overlap_matches_sampled_surface_distance():
    r0, z0, r1, z1 = 0.02, 0.0, 0.0777, 0.1
    cone = dict(type=W.CONE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]), r0=r0, z0=z0, r1=r1, z1=z1)
    rng = np.random.default_rng(2)
    R = 1e-3
    tan = (r1 - r0) / (z1 - z0)
    checked = 0
    for _ in range(40):
        z = rng.uniform(0.01, 0.09)
        phi = rng.uniform(0, 2 * math.pi)
        rw = r0 + z * tan
        rho = rw - rng.uniform(0.2, 1.0) * R * math.cos(math.atan(tan))
        pt = np.array([rho * math.cos(phi), rho * math.sin(phi), z])
        s = make_scene([pt], walls=[cone], h=1e-6)
        ow = oracle.OracleWorld(s)
        F, T, cs = ow.eval()
        dist = cone_min_distance(pt, r0, z0, r1, z1)
        if R - dist > 1e-6:
            assert len(cs) == 1
            assert cs["overlap"][0] == pytest.approx(R - dist, abs=2e-8)
            # the normal points from the wall towards the axis side and lies in the meridian plane
            n = cs["normal"][0]
            assert n[0] * pt[0] + n[1] * pt[1] < 0
            checked += 1
    assert checked > 20


def test_sink_removes_owners_below_the_plane():
    x = np.array([[0.0, 0.0, 0.001], [0.0, 0.01, 0.5]])
    s = make_scene(x, v=[[0, 0, -5.0], [0, 0, 0]], g=(0, 0, -9.81), h=1e-5,
                   sink=(np.zeros(3), np.array([0.0, 0.0, 1.0])))
    ow = oracle.OracleWorld(s)
    ow.step(40)
    assert ow.active.tolist() == [0, 1]
    z_frozen = ow.x[0, 2]
    ow.step(10)
    assert ow.x[0, 2] == z_frozen and ow.x[1, 2] < 0.5


def test_clump_collisions_conserve_linear_momentum_and_nearly_angular():
    """Rods and tetrahedra colliding without walls or gravity: forces are pairwise
    antisymmetric, so linear momentum is constant to rounding; the explicit gyroscopic
    update conserves angular momentum only to O(h)."""
    s = W.free_clumps(n=60, box=0.045, vel_sigma=1.5, seed=9, h=2e-6)
    ow = oracle.OracleWorld(s)
    d0 = ow.diagnostics()
    m = ow.mass
    scale_p = float(np.sum(m * np.linalg.norm(ow.v, axis=1)))
    n_contacts = 0
    for _ in range(400):
        ow.step(10)
        n_contacts += len(ow.eval()[2])
    assert n_contacts > 5
    d1 = ow.diagnostics()
    assert np.max(np.abs(d1["momentum"] - d0["momentum"])) < 1e-12 * scale_p
    assert np.linalg.norm(d1["angmom"] - d0["angmom"]) < 1e-2 * np.linalg.norm(d0["angmom"])


def test_gyroscopic_angular_momentum_drift_is_first_order_in_h():
    """The explicit body-frame update drifts |L| by O(h): halving h halves the drift."""
    tpl = W.rod_template(1e-3)
    drift = []
    for h in (4e-6, 2e-6):
        s = make_scene([[0, 0, 0]], wb=[[300.0, 80.0, -40.0]], templates=[tpl], h=h)
        ow = oracle.OracleWorld(s)
        L0 = ow.diagnostics()["angmom"].copy()
        ow.step(int(round(0.02 / h)))
        drift.append(np.linalg.norm(ow.diagnostics()["angmom"] - L0))
    assert 1.8 < drift[0] / drift[1] < 2.2


def test_sphere_launched_on_a_floor_slides_then_rolls_at_five_sevenths():
    """A sphere resting on a floor at its static overlap, launched at v0 without spin:
    it slides with deceleration mu g while friction spins it up, w R = (5/2) mu g t, until
    the contact point stops slipping at t = 2 v0 / (7 mu g).  From then on it rolls at
    (5/7) v0, its angular momentum about the contact line being conserved."""
    R, E, nu, mu, v0, g, h = 1e-3, 1e9, 0.3, 0.3, 0.1, 9.81, 1e-6
    m = W.sphere_template(R).mass
    ds = (3 * m * g / (4 * (E / (2 * (1 - nu ** 2))) * math.sqrt(R))) ** (2 / 3)
    floor = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    s = make_scene([[0.0, 0.0, R - ds]], v=[[v0, 0.0, 0.0]], walls=[floor], g=(0, 0, -g), h=h,
                   mat=one_material(E=E, nu=nu, e=0.5, mu=mu))
    ow = oracle.OracleWorld(s)
    t_roll = 2 * v0 / (7 * mu * g)
    n = int(0.25 * t_roll / h)
    for k in (1, 2, 3):                              # sliding
        assert ow.step(n) == 0
        t = k * n * h
        assert ow.v[0, 0] == pytest.approx(v0 - mu * g * t, rel=1e-6)
        assert ow.wb[0, 1] * R == pytest.approx(2.5 * mu * g * t, rel=1e-4)
    assert ow.step(int(1.5 * t_roll / h)) == 0      # rolling
    assert ow.v[0, 0] == pytest.approx(5.0 / 7.0 * v0, rel=1e-4)
    assert ow.wb[0, 1] * R == pytest.approx(ow.v[0, 0], rel=1e-4)


@pytest.mark.parametrize("mu,vn,vt", [(0.1, 1.0, 2.0), (0.3, 0.5, 3.0)])
def test_oblique_impact_in_gross_sliding_follows_the_coulomb_impulse(mu, vn, vt):
    """A sphere hits a plane obliquely, elastic (e = 1) and fast enough along the plane
    that its contact point slides for the whole impact (vt > 7 mu vn for a solid sphere).
    Coulomb friction then transmits a tangential impulse of exactly mu times the normal
    one, so the tangential velocity changes by mu times the normal velocity change.  The
    spin gained is that impulse times the lever arm over I = (2/5) m R^2.  The arm runs
    from R down to R - delta_max/2, the contact point being the middle of the overlap, so
    the spin lies between 2.5 mu dv_n (R - delta_max/2)/R^2 and 2.5 mu dv_n / R."""
    R, E, nu, h = 1e-3, 1e9, 0.3, 1e-8
    assert vt > 7 * mu * vn
    floor = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    s = make_scene([[0.0, 0.0, R + 1e-7]], v=[[vt, 0.0, -vn]], walls=[floor], h=h,
                   mat=one_material(E=E, nu=nu, e=1.0, mu=mu))
    ow = oracle.OracleWorld(s)
    m = ow.mass[0]
    Es = E / (2 * (1 - nu ** 2))                     # the plane is of the same material
    dmax = (15 * m * vn ** 2 / (16 * Es * math.sqrt(R))) ** 0.4
    tc = 2 * dmax / vn * 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
    assert ow.step(int((1e-7 / vn + 1.5 * tc) / h)) == 0
    assert len(ow.eval()[2]) == 0                    # the impact is over
    dvn = ow.v[0, 2] + vn
    dvt = ow.v[0, 0] - vt
    assert dvn == pytest.approx(2 * vn, rel=1e-6)    # elastic
    assert -dvt / dvn == pytest.approx(mu, rel=1e-9)
    spin = ow.wb[0, 1]
    hi = 2.5 * mu * dvn / R
    assert hi * (1 - dmax / (2 * R)) < spin < hi


def stack_run(mu, gap_frac, m2, t_end=3.0, h=5e-5):
    """The three-sphere stack of Sec. 4.3.2 with C_r = 0, run to t_end; returns the top
    sphere's height, the largest speed and the statics threshold tan(theta/2)."""
    g = read_golden("stacking_sec4_3_2.txt")
    R, m1 = g["radius_m"], g["bottom_mass_kg"]
    a = R + 0.5 * gap_frac * R                      # bottom centres at x = -a, +a
    sin_t = a / (2 * R)                             # theta: contact normal from vertical
    x = np.array([[-a, 0.0, R], [a, 0.0, R], [0.0, 0.0, R + 2 * R * math.sqrt(1 - sin_t ** 2)]])
    vol = 4.0 / 3.0 * math.pi * R ** 3
    tpls = [W.sphere_template(R, rho=m1 / vol), W.sphere_template(R, rho=m2 / vol)]
    floor = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    s = make_scene(x, templates=tpls, owner_t=[0, 0, 1], walls=[floor], g=(0, 0, -9.81), h=h,
                   mat=one_material(E=1e7, nu=0.3, e=0.5, mu=mu))
    ow = oracle.OracleWorld(s)
    assert ow.step(int(round(t_end / h))) == 0
    return ow.x[2, 2], float(np.max(np.abs(ow.v))), math.tan(0.5 * math.asin(sin_t)), R


@pytest.mark.parametrize("gap_frac,m2", [(0.2, 1.0), (0.2, 3.0), (0.5, 0.3)])
def test_three_sphere_stack_stands_iff_friction_exceeds_tan_half_angle(gap_frac, m2):
    """Statics of the stack without rolling resistance.  On a bottom sphere, torques about
    its centre make the floor's friction equal the friction T at the top contact, and the
    horizontal balance gives T = N tan(theta/2), N being the normal force there.  The top
    sphere's vertical balance gives N = m2 g / 2, because cos(theta) + tan(theta/2)
    sin(theta) = 1.  The floor then carries more than N, so its friction limit holds
    whenever the top contact's does.  The stack can stand iff mu >= tan(theta/2),
    whatever the masses.  It stands 4% above the threshold and collapses 4% below."""
    R = read_golden("stacking_sec4_3_2.txt")["radius_m"]
    thr = math.tan(0.5 * math.asin((R + 0.5 * gap_frac * R) / (2 * R)))
    z_hi, v_hi, thr_run, _ = stack_run(1.04 * thr, gap_frac, m2)
    z_lo, v_lo, _, _ = stack_run(0.96 * thr, gap_frac, m2)
    assert thr_run == thr
    assert z_hi > 2.0 * R and v_hi < 1e-9            # standing, at rest
    assert z_lo < 1.01 * R                           # the top sphere reached the floor


@pytest.mark.parametrize("nu", [0.2, 0.3, 0.45])
def test_tangential_to_normal_stiffness_is_mindlins_ratio(nu):
    """Mindlin: for like materials the tangential stiffness of a Hertzian contact is
    2(1 - nu)/(2 - nu) times the incremental normal stiffness dF_n/d(delta).  Undamped
    (e = 1) so that the tangential force is the spring alone; one step of tangential
    sliding velocity builds the displacement."""
    R, E, h, delta = 1e-3, 1e7, 1e-7, 2e-5
    x = np.array([[0.0, 0.0, 0.0], [2 * R - delta, 0.0, 0.0]])
    s = make_scene(x, v=[[0.0, 0.01, 0.0], [0.0, 0.0, 0.0]], h=h, mat=one_material(E=E, nu=nu, e=1.0, mu=10.0))
    ow = oracle.OracleWorld(s)
    F, T, cs = ow.eval()
    assert len(cs) == 1
    c = cs[0]
    n = np.array(c["normal"])
    f = np.array(c["force"])
    ft = f - np.dot(f, n) * n
    kt = np.linalg.norm(ft) / np.linalg.norm(c["ut"])
    fn = abs(np.dot(f, n))
    kn_incr = 1.5 * fn / c["overlap"]              # F_n ~ delta^(3/2)
    assert kt / kn_incr == pytest.approx(2 * (1 - nu) / (2 - nu), rel=1e-9)


def _contact_stiffness(mats, E, nu, R=1e-3, delta=2e-5, h=1e-7):
    """Normal (F_n / delta^(3/2)) and tangential (|F_t| / |u_t|) stiffness of one undamped,
    frictionally locked contact between spheres of materials mats[0] and mats[1], from one
    step of tangential sliding."""
    tpls = [W.sphere_template(R, mat=0), W.sphere_template(R, mat=1)]
    x = np.array([[0.0, 0.0, 0.0], [2 * R - delta, 0.0, 0.0]])
    mat = (np.asarray(E, np.float64), np.asarray(nu, np.float64), np.ones((2, 2)), np.full((2, 2), 10.0))
    s = make_scene(x, v=[[0.0, 0.01, 0.0], [0.0, 0.0, 0.0]], templates=tpls, owner_t=list(mats), h=h, mat=mat)
    cs = oracle.OracleWorld(s).eval()[2]
    assert len(cs) == 1
    n = np.array(cs[0]["normal"])
    f = np.array(cs[0]["force"])
    fn = abs(np.dot(f, n))
    ft = f - np.dot(f, n) * n
    return fn / cs[0]["overlap"] ** 1.5, np.linalg.norm(ft) / np.linalg.norm(cs[0]["ut"])


def test_unlike_material_stiffnesses_are_the_two_half_space_compliances_in_series():
    """Hertz and Mindlin: each body of a contact deforms as an elastic half-space, so at a
    given contact radius the contact's normal and tangential compliances are the sums of
    the two bodies' compliances ((1 - nu^2)/E and (2 - nu)/G per body, G = E/(2(1 + nu))).
    With the geometry fixed, a like-material contact has twice one body's compliance, so
    1/k(A, B) = (1/k(A, A) + 1/k(B, B)) / 2 for both stiffnesses."""
    E, nu = [1e7, 4.5e7], [0.22, 0.41]
    kn_aa, kt_aa = _contact_stiffness((0, 0), E, nu)
    kn_bb, kt_bb = _contact_stiffness((1, 1), E, nu)
    kn_ab, kt_ab = _contact_stiffness((0, 1), E, nu)
    assert 1.0 / kn_ab == pytest.approx(0.5 * (1.0 / kn_aa + 1.0 / kn_bb), rel=1e-9)
    assert 1.0 / kt_ab == pytest.approx(0.5 * (1.0 / kt_aa + 1.0 / kt_bb), rel=1e-9)
    # and the pair is symmetric in its two bodies
    kn_ba, kt_ba = _contact_stiffness((1, 0), E, nu)
    assert kn_ba == pytest.approx(kn_ab, rel=1e-12) and kt_ba == pytest.approx(kt_ab, rel=1e-12)


def test_hertz_headon_unlike_materials_and_radii():
    """Hertz impact of unlike spheres: delta_max = (15 mbar v^2 / (16 E* sqrt(Rbar)))^(2/5)
    with 1/E* = sum (1 - nu_i^2)/E_i, Rbar = R1 R2/(R1 + R2), mbar = m1 m2/(m1 + m2)."""
    R1, R2, E1, E2, n1, n2, v0 = 1e-3, 1.7e-3, 1e7, 3e7, 0.25, 0.4, 0.8
    t1 = W.sphere_template(R1, mat=0)
    t2 = W.sphere_template(R2, mat=1)
    m1, m2 = t1.mass, t2.mass
    mbar = m1 * m2 / (m1 + m2)
    Rbar = R1 * R2 / (R1 + R2)
    Es = 1.0 / ((1 - n1 ** 2) / E1 + (1 - n2 ** 2) / E2)
    dmax = (15 * mbar * v0 ** 2 / (16 * Es * math.sqrt(Rbar))) ** 0.4
    tc = 2 * dmax / v0 * 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
    h = tc / 4000
    x = np.array([[0.0, 0.0, 0.0], [R1 + R2, 0.0, 0.0]])
    v = np.array([[v0 * m2 / (m1 + m2), 0, 0], [-v0 * m1 / (m1 + m2), 0, 0]])
    mat = (np.array([E1, E2]), np.array([n1, n2]), np.ones((2, 2)), np.zeros((2, 2)))
    s = make_scene(x, v=v, templates=[t1, t2], owner_t=[0, 1], h=h, mat=mat)
    ow = oracle.OracleWorld(s)
    best = 0.0
    for _ in range(3 * 4000):
        ow.step(1)
        cs = ow.eval()[2]
        if len(cs):
            best = max(best, float(cs["overlap"][0]))
        elif best > 0:
            break
    assert best == pytest.approx(dmax, rel=2e-3)
    assert ow.v[1, 0] - ow.v[0, 0] == pytest.approx(v0, rel=2e-3)   # elastic: speed of separation = v0



# ----------------------------------------------------------------------------- rolling resistance

def rolling_incline_run(alpha_deg, crr, v0, t_end, mu=None):
    """A sphere (the Sec. 4.3.1 incline parameters) set rolling without slip at v0 along
    the incline (negative: down-slope), rolling resistance C_r = crr."""
    gd = read_golden("incline_sec4_3_1.txt")
    r, m = gd["radius_m"], gd["mass_kg"]
    mu = gd["mu"] if mu is None else mu
    rho = m / (4 / 3 * math.pi * r ** 3)
    a = math.radians(alpha_deg)
    g = 9.81 * np.array([-math.sin(a), 0.0, -math.cos(a)])
    Es = gd["E_pa"] / (2 * (1 - gd["nu"] ** 2))
    d0 = (3 * m * 9.81 * math.cos(a) / (4 * Es * math.sqrt(r))) ** (2 / 3)
    arm0 = r - 0.5 * d0
    plane = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    h = 2e-5
    s = make_scene([[0.0, 0.0, r - d0]], v=[[v0, 0, 0]], wb=[[0, v0 / arm0, 0]],
                   templates=[W.sphere_template(r, rho=rho)], walls=[plane], g=g, h=h,
                   mat=one_material(E=gd["E_pa"], nu=gd["nu"], e=gd["cor"], mu=mu), crr=np.array([[crr]]))
    ow = oracle.OracleWorld(s)
    ts, vs, xs, slips, arms = [], [], [], [], []
    for k in range(0, int(t_end / h), 50):
        assert ow.step(50) == 0
        qw, qx, qy, qz = ow.q[0]
        Rm = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
                       [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
                       [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])
        F, T, cs = ow.eval()
        arm = np.array(cs["point"][0]) - ow.x[0]
        ts.append((k + 50) * h)
        vs.append(ow.v[0, 0])
        xs.append(ow.x[0, 0])
        slips.append(ow.v[0, 0] + np.cross(Rm @ ow.wb[0], arm)[0])
        arms.append(np.linalg.norm(arm))
    return np.array(ts), np.array(vs), np.array(xs), np.array(slips), a, float(np.mean(arms)), r


@pytest.mark.parametrize("alpha", [7.0, 15.0, 25.0, 30.0])
def test_rolling_resistance_on_an_incline_rolls_at_the_closed_form_rate(alpha):
    """Sec. 4.3.1 with C_r = 0.1, mu = 0.25: between tan(alpha) = C_r and 3.5 mu - 2.5 C_r
    the sphere rolls without slip.  Rolling resistance C_r N acts at the contact arm a, so
    the friction F_t and the rolling equations m dv/dt = m g sin(alpha) - F_t and
    I dw/dt = a (F_t - C_r N), with v = a w and N = m g cos(alpha), give
    dv/dt = g (sin(alpha) - C_r cos(alpha)) / (1 + I / (m a^2)), I = (2/5) m r^2."""
    crr, mu = 0.1, 0.25
    ts, vs, xs, slips, a, arm, r = rolling_incline_run(alpha, crr, -0.2 if alpha > 7 else 0.0, 1.5)
    assert crr < math.tan(a) < 3.5 * mu - 2.5 * crr
    late = ts > ts[-1] * 0.4
    assert np.max(np.abs(slips[late])) < 1e-6 * np.max(np.abs(vs[late]))
    acc = np.polyfit(ts[late], vs[late], 1)[0]
    assert acc == pytest.approx(-9.81 * (math.sin(a) - crr * math.cos(a)) / (1 + 0.4 * r * r / arm ** 2), rel=1e-6)


def test_rolling_resistance_stops_a_sphere_below_tan_alpha_equal_to_cr():
    """Sec. 4.3.1: stationary iff tan(alpha) <= (mu_s / mu_k) C_r (here mu_s = mu_k): a
    sphere rolling down a 4 degree incline with C_r = 0.1 decelerates at
    g (C_r cos - sin) / (1 + I / (m a^2)) and then stays put."""
    crr = 0.1
    ts, vs, xs, slips, a, arm, r = rolling_incline_run(4.0, crr, -0.2, 2.0)
    assert math.tan(a) < crr
    early = (ts > 0.1) & (ts < 0.4)            # after the first contact's transient, before it stops
    acc = np.polyfit(ts[early], vs[early], 1)[0]
    assert acc == pytest.approx(9.81 * (crr * math.cos(a) - math.sin(a)) / (1 + 0.4 * r * r / arm ** 2), rel=1e-6)
    last = ts > 1.5
    assert np.max(np.abs(vs[last])) < 1e-3 * 0.2
    assert np.ptp(xs[last]) < 1e-4 * r


def test_rolling_resistance_slips_above_the_mixed_threshold():
    """Sec. 4.3.1: pure rolling only while tan(alpha) <= 3.5 mu_s - 2.5 C_r (0.625 for
    mu = 0.25, C_r = 0.1); at 35 degrees the contact point slides."""
    ts, vs, xs, slips, a, arm, r = rolling_incline_run(35.0, 0.1, -0.2, 1.0)
    assert math.tan(a) > 3.5 * 0.25 - 2.5 * 0.1
    late = ts > ts[-1] * 0.5
    assert np.max(np.abs(slips[late])) > 0.1 * np.max(np.abs(vs[late]))


def stack_statics_critical_mass(mu, crr, gap_frac, R, m1, g=9.81):
    """Largest top mass m2 for which the three-sphere stack can stand with friction mu and
    rolling resistance C_r, by the statics of a bottom sphere (rolling resistance acting
    as a torque limit C_r N R at each of its two contacts).  With theta the angle of the
    top contact normal from vertical and N = m2 g / 2 + x its normal force, the top
    sphere's balance fixes the tangential force there, f = (x cos + (m2 g / 2)(cos - 1))
    / sin, the bottom sphere's horizontal balance the floor friction
    F = (-x - (m2 g / 2)(1 - cos)) / sin, its torque balance the rolling torque needed,
    R x / tan(theta/2), and the floor carries m1 g + m2 g / 2.  The stack stands iff some
    x >= 0 meets |f| <= mu N, |F| <= mu (m1 g + m2 g / 2) and the rolling torque limit
    C_r R (N + m1 g + m2 g / 2).  (C_r = 0 leaves x = 0: mu >= tan(theta/2).)"""
    st = (R + 0.5 * gap_frac * R) / (2 * R)
    ct = math.sqrt(1 - st * st)
    cot2 = 1.0 / math.tan(0.5 * math.asin(st))

    def stands(m2):
        W2 = 0.5 * m2 * g
        x_min = W2 * (1 - ct - mu * st) / (ct + mu * st)            # |f| <= mu N
        x_max = crr * (2 * W2 + m1 * g) / (cot2 - crr) if cot2 > crr else math.inf
        x_f = mu * st * (m1 * g + W2) - W2 * (1 - ct)                # floor friction
        return max(x_min, 0.0) <= min(x_max, x_f)

    lo, hi = 1e-4, 1e3
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if stands(mid) else (lo, mid)
    return lo


def stack_run_rolling(mu, crr, gap_frac, m2, t_end=3.0, h=5e-5):
    g = read_golden("stacking_sec4_3_2.txt")
    R, m1 = g["radius_m"], g["bottom_mass_kg"]
    a = R + 0.5 * gap_frac * R
    sin_t = a / (2 * R)
    x = np.array([[-a, 0.0, R], [a, 0.0, R], [0.0, 0.0, R + 2 * R * math.sqrt(1 - sin_t ** 2)]])
    vol = 4.0 / 3.0 * math.pi * R ** 3
    tpls = [W.sphere_template(R, rho=m1 / vol), W.sphere_template(R, rho=m2 / vol)]
    floor = dict(type=W.PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]))
    s = make_scene(x, templates=tpls, owner_t=[0, 0, 1], walls=[floor], g=(0, 0, -9.81), h=h,
                   mat=one_material(E=1e7, nu=0.3, e=0.5, mu=mu), crr=np.array([[crr]]))
    ow = oracle.OracleWorld(s)
    assert ow.step(int(round(t_end / h))) == 0
    return ow.x[2, 2], R


@pytest.mark.parametrize("gap_frac,mu,crr", [(0.2, 0.2, 0.05), (0.2, 0.2, 0.03), (0.5, 0.25, 0.05)])
def test_three_sphere_stack_with_rolling_resistance_follows_its_statics(gap_frac, mu, crr):
    """Sec. 4.3.2: with rolling resistance the stack carries a top mass up to a critical
    value that grows with C_r (here mu < tan(theta/2), so friction alone cannot hold it).
    The run stands at 0.85 of the statics' critical mass and collapses at 1.15 of it."""
    g = read_golden("stacking_sec4_3_2.txt")
    R, m1 = g["radius_m"], g["bottom_mass_kg"]
    assert mu < math.tan(0.5 * math.asin((R + 0.5 * gap_frac * R) / (2 * R)))
    mc = stack_statics_critical_mass(mu, crr, gap_frac, R, m1)
    assert mc > stack_statics_critical_mass(mu, 0.5 * crr, gap_frac, R, m1) > 0.0
    z_lo, _ = stack_run_rolling(mu, crr, gap_frac, 0.85 * mc)
    z_hi, _ = stack_run_rolling(mu, crr, gap_frac, 1.15 * mc)
    assert z_lo > 2.0 * R                  # standing
    assert z_hi < 1.01 * R                 # the top sphere reached the floor


def test_rolling_resistance_waits_for_the_collision_time_and_acts_on_torques_only():
    """The default model of Sec. 4.2.1: no rolling resistance during a contact's first
    collision time; after it, a force of C_r |F_n| along w_B x r_B - w_A x r_A that enters
    the torques only (the contact force and the owners' force sums are unchanged)."""
    R, crr = 1e-3, 0.2
    x = np.array([[0.0, 0.0, 0.0], [2 * R - 2e-5, 0.0, 0.0]])
    wb = np.array([[0.0, 0.0, 30.0], [0.0, 0.0, 0.0]])
    s = make_scene(x, wb=wb, h=1e-7, mat=one_material(e=0.5, mu=0.4), crr=np.array([[crr]]))
    s0 = make_scene(x, wb=wb, h=1e-7, mat=one_material(e=0.5, mu=0.4))
    ow, ow0 = oracle.OracleWorld(s), oracle.OracleWorld(s0)
    F, T, cs = ow.eval()
    F0, T0, cs0 = ow0.eval()
    assert len(cs) == 1 and cs["age"][0] == pytest.approx(1e-7)
    assert np.all(np.array(cs["torque_force"][0]) == 0.0) and np.array_equal(T, T0)
    # a contact that has lasted a long time: the rolling force is on
    ow.set_history([0], [1], [[0.0, 0.0, 0.0]], age=[1.0])
    F, T, cs = ow.eval()
    fr = np.array(cs["torque_force"][0])
    fn = abs(np.dot(np.array(cs["force"][0]), np.array(cs["normal"][0])))
    assert np.linalg.norm(fr) == pytest.approx(crr * fn, rel=1e-9)
    # along w_B x r_B - w_A x r_A: A spins about +z, its contact point (r_A = +a x) moves
    # along +y, so the force on A points along -y
    assert fr[1] / np.linalg.norm(fr) == pytest.approx(-1.0, abs=1e-12)
    assert np.array_equal(F, F0)
    arm = np.array(cs["point"][0]) - x[0]
    assert T[0] - T0[0] == pytest.approx(np.cross(arm, fr), rel=1e-9, abs=1e-18)
    assert T[1] - T0[1] == pytest.approx(np.cross(np.array(cs["point"][0]) - x[1], -fr), rel=1e-9, abs=1e-18)


# ----------------------------------------------------------------------------- family tags

def test_a_fixed_family_holds_still_and_carries_a_sphere_at_the_hertz_overlap():
    """Sec. 2.2.2: a family prescribed to zero velocity stays put; a sphere resting on a
    fixed sphere settles to the static Hertz overlap delta = (3 W / (4 E* sqrt(Rbar)))^(2/3)
    with W = m g and Rbar = R / 2."""
    R, E, nu = 1e-3, 1e7, 0.3
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2 * R]])
    s = make_scene(x, g=(0, 0, -9.81), h=2e-6, mat=one_material(E=E, nu=nu, e=0.3, mu=0.3),
                   family=np.array([1, 0]), family_motion={1: ((0, 0, 0), (0, 0, 0))})
    ow = oracle.OracleWorld(s)
    assert ow.step(150000) == 0
    assert np.array_equal(ow.x[0], x[0]) and np.all(ow.v[0] == 0.0)
    m = ow.mass[1]
    Es = E / (2 * (1 - nu * nu))
    want = (3 * m * 9.81 / (4 * Es * math.sqrt(R / 2))) ** (2 / 3)
    assert (2 * R - (ow.x[1, 2] - ow.x[0, 2])) == pytest.approx(want, rel=1e-6)


def test_a_prescribed_velocity_bounces_a_sphere_off_at_twice_its_speed():
    """A family prescribed to move at V does not respond to forces: an elastic,
    frictionless head-on hit on a free sphere at rest sends it off at 2 V (the relative
    motion of an elastic Hertz contact is reversed; the prescribed body is not slowed)."""
    R = 1e-3
    V = 0.3
    x = np.array([[0.0, 0.0, 0.0], [2 * R + 1e-5, 0.0, 0.0]])
    s = make_scene(x, v=[[V, 0, 0], [0, 0, 0]], h=1e-8, mat=one_material(e=1.0, mu=0.0),
                   family=np.array([2, 0]), family_motion={2: ((V, 0, 0), None)})
    ow = oracle.OracleWorld(s)
    n = 40000
    assert ow.step(n) == 0
    assert len(ow.eval()[2]) == 0                       # the contact is over
    assert ow.v[0, 0] == V
    assert ow.x[0, 0] == pytest.approx(n * 1e-8 * V, rel=1e-12)
    assert ow.v[1, 0] == pytest.approx(2 * V, rel=1e-4)
    assert np.all(np.abs(ow.v[1, 1:]) < 1e-12)


def test_a_prescribed_spin_turns_the_owner_at_that_rate():
    """A family prescribed to spin at w (global frame) turns by h |w| per step about w
    whatever torque acts, and reads back its body-frame angular velocity R(q)^T w."""
    R = 1e-3
    w = np.array([0.0, 3.0, 4.0])
    s = make_scene([[0.0, 0.0, 0.0]], h=1e-5, family=np.array([5]), family_motion={5: (None, w)})
    ow = oracle.OracleWorld(s)
    n = 2000
    assert ow.step(n) == 0
    ang = n * 1e-5 * 5.0
    ax = w / 5.0
    want = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax])
    assert np.allclose(ow.q[0], want, atol=1e-12)
    qw, qx, qy, qz = ow.q[0]
    Rm = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
                   [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
                   [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])
    assert np.allclose(Rm @ ow.wb[0], w, atol=1e-12)


def test_masked_families_pass_through_each_other():
    """Sec. 2.2.2: contacts between masked families are not resolved; the same spheres in
    unmasked families collide."""
    R = 1e-3
    x = np.array([[0.0, 0.0, 0.0], [2 * R + 1e-5, 0.0, 0.0]])
    v = [[0.5, 0, 0], [-0.5, 0, 0]]
    base = dict(v=v, h=1e-7, mat=one_material(e=0.5, mu=0.3), family=np.array([3, 4]))
    through = oracle.OracleWorld(make_scene(x, family_masked=[(3, 4)], **base))
    hit = oracle.OracleWorld(make_scene(x, **base))
    assert through.step(40000) == 0 and hit.step(40000) == 0
    assert np.array_equal(through.v, np.array(v, np.float64))
    assert through.x[0, 0] > through.x[1, 0]           # they have crossed
    assert hit.v[0, 0] < 0 and hit.v[1, 0] > 0          # they bounced


def test_contacts_among_fixed_owners_change_nothing():
    """The active-box reading (Sec. 6.4): owners outside the box are fixed and their
    mutual contacts are not resolved.  Contacts between two fixed owners move nothing, so
    masking them leaves every trajectory bit-identical."""
    sc = W.dense_lattice(n=600, seed=31, vel_sigma=0.3)
    z = np.asarray(sc.x)[:, 2]
    fam = np.where(z < np.median(z), 1, 0).astype(np.uint8)
    fixed = {1: ((0, 0, 0), (0, 0, 0))}
    a = oracle.OracleWorld(dataclasses.replace(sc, family=fam, family_motion=fixed, family_masked=[(1, 1)]))
    b = oracle.OracleWorld(dataclasses.replace(sc, family=fam, family_motion=fixed))
    assert a.step(200) == 0 and b.step(200) == 0
    for f in ("x", "v", "wb", "q"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert len(a.eval()[2]) < len(b.eval()[2])          # fewer contacts resolved
    moved = np.any(a.x != np.asarray(sc.x), axis=1)
    assert not np.any(moved[fam == 1]) and np.any(moved[fam == 0])


# ----------------------------------------------------------------------------- bonded breakage

BRK = dict(tension=-1e5, cohesion=2e5, eta=0.1, damping=0.01)


def bonded_pair_run(v_b, steps, R=1e-3, E=1e7, nu=0.3, mu=0.4, h=1e-6, sample=50, params=BRK):
    """Two touching spheres bonded at zero load (Sec. 6.3 model): A held fixed, B moved
    at the prescribed velocity v_b; returns per sample the centre distance, the contact
    force on A and whether the pair still interacts."""
    x = np.array([[0.0, 0.0, 0.0], [2 * R, 0.0, 0.0]])
    s = make_scene(x, h=h, mat=one_material(E=E, nu=nu, e=0.5, mu=mu), family=np.array([1, 2]),
                   family_motion={1: ((0, 0, 0), (0, 0, 0)), 2: (v_b, (0, 0, 0))},
                   force_model="bonded_breakage", model_params=params)
    ow = oracle.OracleWorld(s)
    ow.set_wildcards([0], [1], [[1.0, 0.0, 0.0, 0.0]])
    out = []
    for k in range(steps // sample):
        assert ow.step(sample) == 0
        F, T, cs = ow.eval()
        d = float(np.linalg.norm(ow.x[1] - ow.x[0]))
        if len(cs):
            out.append((d, np.array(cs["force"][0]), float(cs["wc"][0][0])))
        else:
            out.append((d, np.zeros(3), 0.0))
    return out, ow


def test_bonded_contact_in_tension_peaks_at_its_strength_and_breaks_at_three_times_yield():
    """Sec. 6.3 (Eq. of k_n): a bond pulled apart carries k_n D up to its strength
    F_b = sigma_t A (A = pi R^2, k_n = E* Rbar), softens linearly to zero at three times
    the yield separation D_y = F_b / k_n, and breaks there."""
    R, E, nu = 1e-3, 1e7, 0.3
    V = 0.01
    out, ow = bonded_pair_run((V, 0, 0), 40000, R=R, E=E, nu=nu)
    Es = E / (2 * (1 - nu * nu))
    kn = Es * R / 2
    Fb = BRK["tension"] * math.pi * R * R
    Dy = Fb / kn
    sep = np.array([d - 2 * R for d, _, _ in out])
    fx = np.array([f[0] for _, f, _ in out])             # pull on A towards B (+x)
    damp = BRK["damping"] * math.sqrt(0.5 * ow.mass[0] * kn) * V
    alive = fx > 0
    assert fx.max() == pytest.approx(-Fb + damp, rel=2e-3)
    k_peak = int(np.argmax(fx))
    assert sep[k_peak] == pytest.approx(-Dy, rel=2e-2)
    # halfway down the softening branch at twice the yield separation
    mid = int(np.argmin(np.abs(sep - 2 * (-Dy))))
    assert fx[mid] == pytest.approx(-0.5 * Fb + damp, rel=2e-2)
    # the bond is gone once the separation passes 3 D_y, and nothing pulls afterwards
    last_alive = int(np.flatnonzero(alive)[-1])
    step_sep = V * 1e-6 * 50
    assert sep[last_alive] <= 3 * (-Dy) + step_sep and sep[last_alive + 1] >= 3 * (-Dy) - step_sep
    assert np.all(fx[last_alive + 1:] == 0.0)


def test_bonded_contact_in_shear_breaks_at_its_cohesion():
    """Sec. 6.3: the tangential spring k_t = nu k_n carries the shear until it exceeds
    mu |F| + c A (c the cohesion).  Sheared sideways by u at speed V, the pair's centre
    distance grows to sqrt(4 R^2 + u^2), so the bond also carries a tension
    k_n (sqrt(4 R^2 + u^2) - 2 R); it breaks where k_t u + g_t V (the spring plus its
    damping) first exceeds mu times that tension plus c A."""
    R, E, nu = 1e-3, 1e7, 0.3
    V = 0.01
    par = dict(BRK, cohesion=2e4)          # breaks in shear long before the normal gap matters
    out, ow = bonded_pair_run((0, V, 0), 12000, R=R, E=E, nu=nu, sample=10, params=par)
    kn = E / (2 * (1 - nu * nu)) * R / 2
    kt = nu * kn
    m = ow.mass[0]
    beta = math.log(0.5) / math.sqrt(math.log(0.5) ** 2 + math.pi ** 2)
    gt = -2 * math.sqrt(5 / 6) * beta * math.sqrt(0.5 * m * kt)
    cA = par["cohesion"] * math.pi * R * R

    def excess(u):
        return kt * u + gt * V - (0.4 * kn * (math.sqrt(4 * R * R + u * u) - 2 * R) + cA)
    lo, hi = 0.0, 1e-3
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if excess(mid) > 0 else (mid, hi)
    u_break = hi
    state = np.array([st for _, _, st in out])
    k = int(np.flatnonzero(state <= 0.0)[0])            # first sample without the bond
    assert k * 10 * 1e-6 * V <= u_break <= (k + 1) * 10 * 1e-6 * V + 1e-12
    # the tangential part of the force just before the break: the spring and its damping
    u = k * 10 * 1e-6 * V
    n = np.array([-2 * R, -u, 0.0]) / math.sqrt(4 * R * R + u * u)
    f = out[k - 1][1]
    ft = np.linalg.norm(f - np.dot(f, n) * n)
    assert ft == pytest.approx(kt * (u + 1e-6 * V) + gt * V, rel=1e-3)


def test_bonded_cluster_conserves_linear_momentum():
    """Action and reaction: a free cluster of bonded spheres of unequal radii (no walls, no
    gravity) keeps its total linear momentum to rounding while bonds stretch and break."""
    rng = np.random.default_rng(5)
    R = 1e-3
    x = np.array([[0.0, 0.0, 0.0], [1.95 * R, 0.0, 0.0], [0.9 * R, 1.7 * R, 0.0], [0.9 * R, 0.6 * R, 1.6 * R]])
    v = rng.normal(scale=0.2, size=(4, 3))
    scale = np.array([1.0, 0.9, 1.1, 0.95])
    s = make_scene(x, v=v, scale=scale, h=1e-6, mat=one_material(e=0.5, mu=0.4),
                   force_model="bonded_breakage", model_params=BRK)
    ow = oracle.OracleWorld(s)
    pairs = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]
    ow.set_wildcards([a for a, _ in pairs], [b for _, b in pairs], [[1.0, 0.0, 0.0, 0.0]] * len(pairs))
    p0 = (ow.mass[:, None] * ow.v).sum(axis=0)
    assert ow.step(3000) == 0
    p1 = (ow.mass[:, None] * ow.v).sum(axis=0)
    scale_p = (ow.mass[:, None] * np.abs(v)).sum()
    assert np.all(np.abs(p1 - p0) <= 1e-12 * scale_p)


# ----------------------------------------------------------------------------- mesh facets

def facet(tri, p=(0, 0, 0), omega=(0, 0, 0), mat=0):
    return dict(type=oracle.WALL_TRIANGLE, mat=mat, p=np.asarray(p, np.float64), n=np.zeros(3),
                omega=np.asarray(omega, np.float64), tri=np.asarray(tri, np.float64).reshape(9))


def sampled_distance(c, tri, n=400):
    """Distance from c to a triangle by dense barycentric sampling (brute force)."""
    a, b, cc = np.asarray(tri, np.float64).reshape(3, 3)
    u, v = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    keep = u + v <= 1
    pts = a + u[keep, None] * (b - a) + v[keep, None] * (cc - a)
    return float(np.min(np.linalg.norm(pts - c, axis=1)))


def test_facet_gap_is_the_distance_to_the_closest_point_in_every_region():
    """Sec. 2.4 meshes: a sphere's gap to a facet is its centre's distance to the facet's
    closest point, whichever region (face, one of three edges, one of three vertices) that
    point lies in; brute-force sampling of the triangle agrees."""
    tri = [[0.0, 0.0, 0.0], [4e-3, 0.0, 0.0], [0.5e-3, 3e-3, 0.0]]
    R = 1e-3
    rng = np.random.default_rng(3)
    centres = np.concatenate([rng.uniform([-2e-3, -2e-3, -1.5e-3], [6e-3, 5e-3, 1.5e-3], size=(60, 3)),
                              [[-0.4e-3, -0.3e-3, 0.2e-3], [4.5e-3, -0.2e-3, 0.1e-3], [0.4e-3, 3.4e-3, -0.1e-3],
                               [2e-3, -0.6e-3, 0.0], [1.5e-3, 1e-3, 0.6e-3]]])
    for c in centres:
        d = sampled_distance(c, tri)
        s = make_scene([c], walls=[facet(tri)])
        ow = oracle.OracleWorld(s)
        F, T, cs = ow.eval()
        if d < R - 2e-5:
            assert len(cs) == 1
            assert cs["overlap"][0] == pytest.approx(R - d, abs=2e-5)
            nrm = np.array(cs["normal"][0])
            q = c - d * nrm                               # back to the facet
            assert sampled_distance(q, tri) < 2e-5
        elif d > R + 2e-5:
            assert len(cs) == 0


def test_sphere_resting_on_a_facet_settles_to_the_hertz_overlap():
    """A horizontal facet carries a sphere like a plane (Rbar = R): the static overlap is
    (3 m g / (4 E* sqrt(R)))^(2/3)."""
    R, E, nu = 1e-3, 1e7, 0.3
    tri = [[-5e-3, -5e-3, 0.0], [5e-3, -5e-3, 0.0], [0.0, 6e-3, 0.0]]
    s = make_scene([[0.0, 0.0, R]], walls=[facet(tri)], g=(0, 0, -9.81), h=2e-6,
                   mat=one_material(E=E, nu=nu, e=0.3, mu=0.3))
    ow = oracle.OracleWorld(s)
    assert ow.step(150000) == 0
    m = ow.mass[0]
    want = (3 * m * 9.81 / (4 * E / (2 * (1 - nu * nu)) * math.sqrt(R))) ** (2 / 3)
    assert R - ow.x[0, 2] == pytest.approx(want, rel=1e-6)


def test_a_turning_facet_moves_by_its_rotation():
    """A facet turning with omega about p sits at p + R(omega t)(v - p) at time t: a
    resting sphere's gap follows the analytic distance to the rotated triangle, and the
    facet drags a touching sphere along its surface velocity omega x (c - p)."""
    tri = np.array([[3e-3, -2e-3, 0.0], [9e-3, -2e-3, 0.0], [6e-3, 4e-3, 0.0]])
    w = np.array([0.0, 0.0, 20.0])
    c = np.array([[5e-3, 3e-3, 0.9e-3]])
    s = make_scene(c, walls=[facet(tri, omega=w)], h=1e-5, family=np.array([1]),
                   family_motion={1: ((0, 0, 0), (0, 0, 0))})
    ow = oracle.OracleWorld(s)
    for n in (0, 40, 90):
        if n:
            assert ow.step(n - ow._w.step) == 0
        t = ow._w.step * 1e-5
        th = 20.0 * t
        Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
        rot = tri @ Rz.T
        d = sampled_distance(c[0], rot, n=600)
        F, T, cs = ow.eval()
        if d < 1e-3:
            assert cs["overlap"][0] == pytest.approx(1e-3 - d, abs=2e-5)
            # the facet's surface velocity at the contact point enters the tangential force
            u_b = np.cross(w, np.array(cs["point"][0]))
            assert np.linalg.norm(u_b) > 0
        else:
            assert len(cs) == 0
