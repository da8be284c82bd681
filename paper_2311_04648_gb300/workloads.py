"""Seeded synthetic scenes shaped like the paper's workloads.

This module holds scene *descriptions* only (geometry, materials, initial state drawn
from seeded generators); it contains none of the DEM method's arithmetic.  It is the one
module that both the CUDA library's tests/benchmarks and the CPU oracle's tests consume.

Scenes (SI units throughout):
  - ``settle_box``      : N monodisperse spheres placed by random sequential addition
                          without overlap in a walled box (2,000 spheres, R = 1 mm,
                          40 x 40 x 80 mm box, dt = 1e-6 s).
  - ``settling_column`` : polydisperse spheres (R ~ U[0.8, 1.2] mm) on a jittered cubic
                          lattice in a 0.3 x 0.3 x 1.2 m walled box, small random initial
                          velocities, dt = 2e-6 s; ``column_width`` restricts the same
                          generator to a central column (the 20k-sphere sub-box).
  - ``clump_drum``      : 3-sphere rods and 4-sphere tetrahedra (component R ~ U[1, 2] mm)
                          in a drum of radius 0.6 m spinning at 1 rad/s about x.
  - ``cone_hopper``     : polydisperse spheres (R ~ U[1, 2] mm) above a 30-degree conical
                          hopper with a sink below the orifice.
  - ``column_collapse`` : one granular column of a batch of independent scenes.
Material: rho = 2600 kg/m^3, E = 1e7 Pa, nu = 0.3 unless stated.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

RHO = 2600.0
PLANE, CYLINDER, CONE, TRIANGLE = 0, 1, 2, 3


@dataclass
class Template:
    rel_xyz: np.ndarray          # (n, 3) component centres about the centre of mass, principal frame
    radii: np.ndarray            # (n,)
    mats: np.ndarray             # (n,) material ids
    mass: float
    moi: np.ndarray              # (3,) principal moments


@dataclass
class Scene:
    box_lo: np.ndarray
    box_hi: np.ndarray
    E: np.ndarray
    nu: np.ndarray
    cor: np.ndarray              # (nm, nm)
    mu: np.ndarray               # (nm, nm)
    walls: list
    templates: list
    owner_template: np.ndarray   # (M,)
    owner_scale: np.ndarray | None
    x: np.ndarray                # (M, 3)
    q: np.ndarray                # (M, 4) (w, x, y, z)
    v: np.ndarray                # (M, 3)
    wb: np.ndarray               # (M, 3) body-frame angular velocity
    h: float
    g: np.ndarray
    gyroscopic: bool = True
    sink: tuple | None = None
    v_err: float = 0.0
    r_max: float = 0.0
    name: str = ""
    meta: dict = field(default_factory=dict)
    crr: np.ndarray | None = None    # (nm, nm) rolling resistance coefficients; None: zero
    family: np.ndarray | None = None  # (M,) family tag per owner (0..255); None: all 0
    family_motion: dict | None = None  # family -> (v or None, w or None): prescribed velocities
    family_masked: list | None = None  # (a, b) family pairs whose contacts are not resolved
    force_model: str | None = None     # None / "hertz_mindlin" or "bonded_breakage"
    model_params: dict | None = None   # bonded_breakage: tension, cohesion, eta, damping

    @property
    def n_owner(self):
        return len(self.owner_template)

    @property
    def n_sphere(self):
        counts = np.array([len(t.radii) for t in self.templates], np.int64)
        return int(counts[np.asarray(self.owner_template, np.int64)].sum())


def sphere_template(R: float, mat: int = 0, rho: float = RHO) -> Template:
    m = rho * 4.0 / 3.0 * math.pi * R ** 3
    I = 0.4 * m * R * R
    return Template(np.zeros((1, 3)), np.array([R]), np.array([mat], np.int32), m, np.array([I, I, I]))


def rod_template(R: float, mat: int = 0, rho: float = RHO) -> Template:
    """Three tangent collinear spheres along x (spacing 2R)."""
    m1 = rho * 4.0 / 3.0 * math.pi * R ** 3
    i1 = 0.4 * m1 * R * R
    xs = np.array([[-2 * R, 0, 0], [0, 0, 0], [2 * R, 0, 0]], np.float64)
    Ixx = 3 * i1
    Iyy = 3 * i1 + 2 * m1 * (2 * R) ** 2
    return Template(xs, np.full(3, R), np.full(3, mat, np.int32), 3 * m1, np.array([Ixx, Iyy, Iyy]))


def tetra_template(R: float, mat: int = 0, rho: float = RHO) -> Template:
    """Four tangent spheres on the vertices of a regular tetrahedron of edge 2R."""
    m1 = rho * 4.0 / 3.0 * math.pi * R ** 3
    i1 = 0.4 * m1 * R * R
    a = 2 * R / (2 * math.sqrt(2))   # vertices (+-a,+-a,+-a) with an even number of minus signs
    xs = np.array([[a, a, a], [a, -a, -a], [-a, a, -a], [-a, -a, a]], np.float64)
    d2 = 2 * a * a                   # squared distance of each vertex from any coordinate axis
    I = 4 * i1 + 4 * m1 * d2
    return Template(xs, np.full(4, R), np.full(4, mat, np.int32), 4 * m1, np.array([I, I, I]))


def _single_material(E, nu, e, mu):
    return (np.array([E], np.float64), np.array([nu], np.float64),
            np.array([[e]], np.float64), np.array([[mu]], np.float64))


def box_walls(lo, hi, mat=0):
    walls = []
    for a in range(3):
        n = np.zeros(3); n[a] = 1.0
        walls.append(dict(type=PLANE, mat=mat, p=np.array(lo, np.float64), n=n.copy()))
        walls.append(dict(type=PLANE, mat=mat, p=np.array(hi, np.float64), n=-n))
    return walls


def _identity_quats(M):
    q = np.zeros((M, 4))
    q[:, 0] = 1.0
    return q


def _random_quats(rng, M):
    q = rng.normal(size=(M, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def settle_box(n=2000, R=1e-3, box=(0.04, 0.04, 0.08), E=1e7, nu=0.3, e=0.5, mu=0.4,
               seed=1, vel_sigma=0.0, h=1e-6, gap=1e-5, g=(0.0, 0.0, -9.81), walls=True) -> Scene:
    """Random sequential addition of monodisperse spheres without overlap (reject if the
    centre distance is below 2R + gap), optionally with N(0, vel_sigma^2) velocities."""
    rng = np.random.default_rng(seed)
    lo = np.zeros(3)
    hi = np.array(box, np.float64)
    pts = np.empty((n, 3))
    cell = 2 * R + gap
    grid = {}
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > 200 * n:
            raise RuntimeError("random sequential addition did not converge")
        c = lo + R + gap + rng.random(3) * (hi - lo - 2 * (R + gap))
        key = tuple((c // cell).astype(int))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for m in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        if np.sum((pts[m] - c) ** 2) < (2 * R + gap) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts[k] = c
            grid.setdefault(key, []).append(k)
            k += 1
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    v = rng.normal(scale=vel_sigma, size=(n, 3)) if vel_sigma > 0 else np.zeros((n, 3))
    return Scene(lo, hi, Em, num, corm, mum, box_walls(lo, hi) if walls else [], [sphere_template(R)],
                 np.zeros(n, np.int64), None, pts, _identity_quats(n), v, np.zeros((n, 3)), h,
                 np.array(g, np.float64), r_max=R, name=f"settle_box_n{n}_seed{seed}")


def settling_column(n=4_000_000, box=(0.3, 0.3, 1.2), r_lo=0.8e-3, r_hi=1.2e-3, spacing=2.45e-3,
                    jitter=0.02e-3, vel_sigma=0.05, seed=3, E=1e7, nu=0.3, e=0.5, mu=0.4, h=2e-6,
                    column_width=None) -> Scene:
    """Jittered cubic lattice filled layer by layer from z = r_hi upward; R ~ U[r_lo, r_hi].
    With ``column_width`` the lattice is restricted to a central square column of that
    width (same generator, fewer sites per layer), the box shrunk to it."""
    rng = np.random.default_rng(seed)
    lo = np.zeros(3)
    hi = np.array(box, np.float64)
    if column_width is not None:
        cx = 0.5 * (lo[0] + hi[0])
        cy = 0.5 * (lo[1] + hi[1])
        lo = np.array([cx - column_width / 2, cy - column_width / 2, 0.0])
        hi = np.array([cx + column_width / 2, cy + column_width / 2, box[2]])
    nx = int(math.floor((hi[0] - lo[0] - 2 * r_hi) / spacing)) + 1
    ny = int(math.floor((hi[1] - lo[1] - 2 * r_hi) / spacing)) + 1
    per_layer = nx * ny
    layers = int(math.ceil(n / per_layer))
    zmax = r_hi + (layers - 1) * spacing
    if zmax + r_hi > hi[2]:
        raise ValueError("column does not fit the box")
    ii = np.arange(n)
    lz = ii // per_layer
    rem = ii % per_layer
    ly = rem // nx
    lx = rem % nx
    x0 = lo[0] + r_hi + 0.5 * (hi[0] - lo[0] - 2 * r_hi - (nx - 1) * spacing)
    y0 = lo[1] + r_hi + 0.5 * (hi[1] - lo[1] - 2 * r_hi - (ny - 1) * spacing)
    pts = np.stack([x0 + lx * spacing, y0 + ly * spacing, lo[2] + r_hi + lz * spacing], axis=1)
    pts += rng.uniform(-jitter, jitter, size=(n, 3))
    R = rng.uniform(r_lo, r_hi, size=n)
    v = rng.normal(scale=vel_sigma, size=(n, 3))
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    tpl = sphere_template(1e-3)
    return Scene(lo, hi, Em, num, corm, mum, box_walls(lo, hi), [tpl], np.zeros(n, np.int64), R / 1e-3,
                 pts, _identity_quats(n), v, np.zeros((n, 3)), h, np.array([0.0, 0.0, -9.81]),
                 r_max=r_hi, name=f"settling_column_n{n}", meta=dict(nx=nx, ny=ny, layers=layers))


def clump_drum(n_clumps=20_000_000, drum_radius=0.6, omega=1.0, r_lo=1e-3, r_hi=2e-3, mu=0.5, e=0.5,
               E=1e7, nu=0.3, fill=0.40, solid_fraction=0.55, seed=4, h=2e-6, length=None) -> Scene:
    """Half 3-sphere rods, half 4-sphere tetrahedra, component R ~ U[r_lo, r_hi] per clump,
    in a drum about the x axis, placed on a lattice (filled from the bottom) with random
    orientations.  The drum length L is chosen so that the clumps at the stated solid
    fraction fill ``fill`` of the drum volume, unless the lattice needs a longer drum:
    randomly oriented clumps on a lattice whose pitch clears the longest clump hold only
    a few percent solids, so a large clump count sets L by the lattice instead (the
    effective fill at the stated solid fraction is recorded in ``meta``)."""
    rng = np.random.default_rng(seed)
    kinds = rng.random(n_clumps) < 0.5           # True: rod, False: tetra
    Rc = rng.uniform(r_lo, r_hi, size=n_clumps)
    vol = np.where(kinds, 3.0, 4.0) * (4.0 / 3.0) * math.pi * Rc ** 3
    length_fill = float(vol.sum() / solid_fraction / (fill * math.pi * drum_radius ** 2))
    spacing = 6.2 * r_hi             # a rod spans 6R: lattice pitch above the largest clump extent
    if length is None:
        length = length_fill
        ys_all = np.arange(-drum_radius + spacing, drum_radius - spacing, spacing)
        Yf, Zf = np.meshgrid(ys_all, ys_all, indexing="ij")
        per_slice = int(np.count_nonzero((Yf ** 2 + Zf ** 2) < (drum_radius - spacing) ** 2))
        slices = len(np.arange(-length / 2 + spacing / 2, length / 2 - spacing / 2 + 1e-12, spacing))
        if per_slice * slices < n_clumps:
            length = (math.ceil(n_clumps / per_slice) + 1) * spacing
    # lattice sites inside the lower half disc (y, z) times x
    ys = np.arange(-drum_radius + spacing, drum_radius - spacing, spacing)
    zs = np.arange(-drum_radius + spacing, 0.0, spacing)
    Y, Z = np.meshgrid(ys, zs, indexing="ij")
    ok = (Y ** 2 + Z ** 2) < (drum_radius - spacing) ** 2
    yz = np.stack([Y[ok], Z[ok]], axis=1)
    xs = np.arange(-length / 2 + spacing / 2, length / 2 - spacing / 2 + 1e-12, spacing)
    nsite = len(xs) * len(yz)
    if nsite < n_clumps:
        # stack further up into the upper half if the lower half is full
        zs2 = np.arange(-drum_radius + spacing, drum_radius - spacing, spacing)
        Y, Z = np.meshgrid(ys, zs2, indexing="ij")
        ok = (Y ** 2 + Z ** 2) < (drum_radius - spacing) ** 2
        yz = np.stack([Y[ok], Z[ok]], axis=1)
        order = np.argsort(yz[:, 1], kind="stable")
        yz = yz[order]
        nsite = len(xs) * len(yz)
        if nsite < n_clumps:
            raise ValueError("drum too short for the requested clumps")
    # fill from the bottom: sites ordered by z then y then x
    order = np.lexsort((yz[:, 0], yz[:, 1]))
    yz = yz[order]
    site = np.arange(n_clumps)
    iyz = site // len(xs)
    ix = site % len(xs)
    pts = np.stack([xs[ix], yz[iyz, 0], yz[iyz, 1]], axis=1)
    q = _random_quats(rng, n_clumps)
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    templates = [rod_template(1e-3), tetra_template(1e-3)]
    owner_t = np.where(kinds, 0, 1).astype(np.int64)
    axis = np.array([1.0, 0.0, 0.0])
    walls = [dict(type=CYLINDER, mat=0, p=np.zeros(3), n=axis, r0=drum_radius, omega=omega * axis),
             dict(type=PLANE, mat=0, p=np.array([-length / 2, 0, 0]), n=axis.copy(), omega=omega * axis),
             dict(type=PLANE, mat=0, p=np.array([length / 2, 0, 0]), n=-axis, omega=omega * axis)]
    lo = np.array([-length / 2, -drum_radius, -drum_radius])
    hi = np.array([length / 2, drum_radius, drum_radius])
    return Scene(lo, hi, Em, num, corm, mum, walls, templates, owner_t, Rc / 1e-3, pts, q,
                 np.zeros((n_clumps, 3)), np.zeros((n_clumps, 3)), h, np.array([0.0, 0.0, -9.81]),
                 r_max=r_hi, name=f"clump_drum_n{n_clumps}",
                 meta=dict(length=length, length_fill=length_fill,
                           fill_effective=float(vol.sum() / solid_fraction / (math.pi * drum_radius ** 2 * length))))


def cone_hopper(n=10_000_000, r_lo=1e-3, r_hi=2e-3, half_angle_deg=30.0, e=0.5, mu=0.4, E=1e7, nu=0.3,
                seed=6, h=2e-6, vel_sigma=0.0) -> Scene:
    """Polydisperse spheres on a lattice inside a conical hopper (wall 30 degrees from the
    vertical, orifice radius 10 R_max) with a sink plane below the orifice."""
    rng = np.random.default_rng(seed)
    spacing = 2 * r_hi * 1.05
    r_orifice = 10 * r_hi
    tan = math.tan(math.radians(half_angle_deg))
    # choose the fill height so that the cone frustum holds n sites at lattice density
    z = 0.0
    count = 0
    site_z = []
    while count < n:
        rz = r_orifice + (z + spacing) * tan - spacing
        m = int(math.floor(2 * rz / spacing))
        layer = m * m if m > 0 else 0
        # sites inside the disc of radius rz
        if m > 0:
            c = (np.arange(m) - (m - 1) / 2) * spacing
            X, Y = np.meshgrid(c, c, indexing="ij")
            inside = int(np.count_nonzero(X ** 2 + Y ** 2 < rz ** 2))
        else:
            inside = 0
        site_z.append((z, rz, inside))
        count += inside
        z += spacing
    pts = []
    need = n
    for (zl, rz, inside) in site_z:
        m = int(math.floor(2 * rz / spacing))
        c = (np.arange(m) - (m - 1) / 2) * spacing
        X, Y = np.meshgrid(c, c, indexing="ij")
        sel = X ** 2 + Y ** 2 < rz ** 2
        layer = np.stack([X[sel], Y[sel], np.full(int(sel.sum()), zl + spacing)], axis=1)
        take = min(need, len(layer))
        pts.append(layer[:take])
        need -= take
        if need == 0:
            break
    pts = np.concatenate(pts, axis=0)
    z_top = float(pts[:, 2].max()) + 4 * r_hi
    R = rng.uniform(r_lo, r_hi, size=n)
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    axis = np.array([0.0, 0.0, 1.0])
    r_top = r_orifice + z_top * tan
    walls = [dict(type=CONE, mat=0, p=np.zeros(3), n=axis, r0=r_orifice, z0=0.0, r1=r_top, z1=z_top)]
    lo = np.array([-r_top, -r_top, -0.05])
    hi = np.array([r_top, r_top, z_top])
    v = rng.normal(scale=vel_sigma, size=(n, 3)) if vel_sigma > 0 else np.zeros((n, 3))
    return Scene(lo, hi, Em, num, corm, mum, walls, [sphere_template(1e-3)], np.zeros(n, np.int64), R / 1e-3,
                 pts, _identity_quats(n), v, np.zeros((n, 3)), h, np.array([0.0, 0.0, -9.81]),
                 sink=(np.array([0.0, 0.0, -0.02]), axis.copy()), r_max=r_hi, name=f"cone_hopper_n{n}",
                 meta=dict(r_orifice=r_orifice, z_top=z_top))


def column_collapse(n, aspect, mu, e, seed, r_lo=0.9e-3, r_hi=1.1e-3, E=1e7, nu=0.3, h=2e-6,
                    solid_fraction=0.55) -> Scene:
    """A granular column of N spheres with aspect ratio a = height/width, depth 10 R_max,
    on a floor with a flume of length (a + 3) w; the confining wall is absent from t = 0."""
    rng = np.random.default_rng(seed)
    vbar = (4.0 / 3.0) * math.pi * ((r_lo + r_hi) / 2) ** 3
    D = 10 * r_hi
    w = math.sqrt(n * vbar / (solid_fraction * aspect * D))
    H = aspect * w
    spacing = 2 * r_hi * 1.02
    nx = max(1, int(math.floor((w - 2 * r_hi) / spacing)) + 1)
    ny = max(1, int(math.floor((D - 2 * r_hi) / spacing)) + 1)
    per = nx * ny
    ii = np.arange(n)
    lz = ii // per
    rem = ii % per
    ly = rem // nx
    lx = rem % nx
    pts = np.stack([r_hi + lx * spacing, r_hi + ly * spacing, r_hi + lz * spacing], axis=1)
    pts += rng.uniform(-0.01 * r_hi, 0.01 * r_hi, size=(n, 3))
    R = rng.uniform(r_lo, r_hi, size=n)
    L = (aspect + 3) * w
    top = max(H, float(pts[:, 2].max()) + r_hi) * 1.5
    lo = np.zeros(3)
    hi = np.array([max(L, float(pts[:, 0].max()) + 2 * r_hi), D, top])
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    walls = [dict(type=PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0])),
             dict(type=PLANE, mat=0, p=np.zeros(3), n=np.array([1.0, 0.0, 0.0])),
             dict(type=PLANE, mat=0, p=np.zeros(3), n=np.array([0.0, 1.0, 0.0])),
             dict(type=PLANE, mat=0, p=np.array([0.0, D, 0.0]), n=np.array([0.0, -1.0, 0.0])),
             dict(type=PLANE, mat=0, p=np.array([hi[0], 0.0, 0.0]), n=np.array([-1.0, 0.0, 0.0]))]
    return Scene(lo, hi, Em, num, corm, mum, walls, [sphere_template(1e-3)], np.zeros(n, np.int64), R / 1e-3,
                 pts, _identity_quats(n), np.zeros((n, 3)), np.zeros((n, 3)), h, np.array([0.0, 0.0, -9.81]),
                 r_max=r_hi, name=f"column_collapse_n{n}", meta=dict(aspect=aspect, width=w))


def batch_scenes(n_scenes=512, n_lo=1000, n_hi=50_000, seed=5):
    """Independent column collapses: N log-uniform in [n_lo, n_hi], mu ~ U[0.2, 0.8],
    e ~ U[0.3, 0.9], aspect ~ U[0.5, 4]."""
    rng = np.random.default_rng(seed)
    Ns = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_scenes))).astype(int)
    mus = rng.uniform(0.2, 0.8, size=n_scenes)
    es = rng.uniform(0.3, 0.9, size=n_scenes)
    aspects = rng.uniform(0.5, 4.0, size=n_scenes)
    return [column_collapse(int(Ns[k]), float(aspects[k]), float(mus[k]), float(es[k]), seed=1000 + k)
            for k in range(n_scenes)]


def two_spheres(R=1e-3, v0=1.0, E=1e7, nu=0.3, e=1.0, mu=0.0, h=1e-7, gap=1e-6, rho=RHO) -> Scene:
    """Head-on pair along x closing at speed v0, no gravity, no walls."""
    m = rho * 4.0 / 3.0 * math.pi * R ** 3
    x = np.array([[-(R + gap / 2), 0.0, 0.0], [R + gap / 2, 0.0, 0.0]])
    v = np.array([[v0 / 2, 0.0, 0.0], [-v0 / 2, 0.0, 0.0]])
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    return Scene(np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0]), Em, num, corm, mum, [],
                 [sphere_template(R, rho=rho)], np.zeros(2, np.int64), None, x, _identity_quats(2), v,
                 np.zeros((2, 3)), h, np.zeros(3), r_max=R, name="two_spheres", meta=dict(mass=m))


def free_spheres(n=200, R=1e-3, box=0.03, vel_sigma=0.5, E=1e7, nu=0.3, e=0.7, mu=0.3, seed=7, h=1e-6) -> Scene:
    """Spheres with random velocities, no walls, no gravity (momentum tests)."""
    s = settle_box(n=n, R=R, box=(box, box, box), E=E, nu=nu, e=e, mu=mu, seed=seed, vel_sigma=vel_sigma,
                   h=h, g=(0.0, 0.0, 0.0), walls=False)
    rng = np.random.default_rng(seed + 100)
    s.wb = rng.normal(scale=vel_sigma / R, size=(n, 3))
    s.name = f"free_spheres_n{n}"
    return s


def free_clumps(n=60, R=1e-3, box=0.03, vel_sigma=0.5, E=1e7, nu=0.3, e=0.7, mu=0.3, seed=8, h=1e-6,
                g=(0.0, 0.0, 0.0), walls=False) -> Scene:
    """Rods and tetrahedra with random poses and velocities (on a coarse lattice)."""
    rng = np.random.default_rng(seed)
    sp = 7.0 * R
    m = int(math.floor(box / sp))
    sites = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    if len(sites) < n:
        raise ValueError("box too small")
    sel = rng.permutation(len(sites))[:n]
    x = (sites[sel] + 0.5) * sp
    kinds = (np.arange(n) % 2).astype(np.int64)
    q = _random_quats(rng, n)
    v = rng.normal(scale=vel_sigma, size=(n, 3))
    wb = rng.normal(scale=vel_sigma / R, size=(n, 3))
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    lo = np.zeros(3)
    hi = np.full(3, box)
    return Scene(lo, hi, Em, num, corm, mum, box_walls(lo, hi) if walls else [],
                 [rod_template(R), tetra_template(R)], kinds, None, x, q, v, wb, h, np.array(g, np.float64),
                 r_max=R, name=f"free_clumps_n{n}")


# ----------------------------------------------------------------------------- contact-rich test beds

def dense_lattice(n=1000, R=1e-3, spacing=1.97e-3, jitter=0.05e-3, scale_spread=0.03, vel_sigma=0.2,
                  omega_sigma=100.0, e=0.5, mu=0.4, E=1e7, nu=0.3, seed=0, h=1e-6, walls=True,
                  g=(0.0, 0.0, -9.81), wall_overlap=0.02e-3) -> Scene:
    """A jittered cubic lattice of spacing below 2R (many lattice neighbours overlap),
    radii R * U[1 - s, 1 + s], random velocities and spins; the box walls touch the
    outer layers with a small overlap."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n ** (1.0 / 3.0)))
    idx = np.arange(n)
    pts = np.stack([idx % m, (idx // m) % m, idx // (m * m)], axis=1).astype(np.float64) * spacing
    pts += rng.uniform(-jitter, jitter, size=(n, 3))
    scale = rng.uniform(1.0 - scale_spread, 1.0 + scale_spread, size=n)
    rad = R * scale
    lo = np.min(pts - rad[:, None], axis=0) + wall_overlap
    hi = np.max(pts + rad[:, None], axis=0) - wall_overlap
    pad = 0.0 if walls else 5 * R
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    v = rng.normal(scale=vel_sigma, size=(n, 3))
    wb = rng.normal(scale=omega_sigma, size=(n, 3))
    return Scene(lo - pad, hi + pad, Em, num, corm, mum, box_walls(lo, hi) if walls else [], [sphere_template(R)],
                 np.zeros(n, np.int64), scale, pts, _identity_quats(n), v, wb, h, np.array(g, np.float64),
                 r_max=float(rad.max()), name=f"dense_lattice_n{n}_seed{seed}")


def packed_clumps(n=150, R=1e-3, fill=0.15, max_overlap=0.12, vel_sigma=0.3, omega_sigma=100.0, e=0.5, mu=0.4,
                  E=1e7, nu=0.3, seed=0, h=1e-6, walls=True, g=(0.0, 0.0, -9.81)) -> Scene:
    """Rods and tetrahedra placed by random sequential addition with random orientations
    in a box holding them at solid fraction ``fill``; spheres of different clumps may
    overlap by up to ``max_overlap`` R, so many pairs start in contact."""
    rng = np.random.default_rng(seed)
    tpls = [rod_template(R), tetra_template(R)]
    kinds = rng.integers(0, 2, size=n).astype(np.int64)
    vol = float(np.sum(np.where(kinds == 0, 3, 4))) * (4.0 / 3.0) * math.pi * R ** 3
    side = (vol / fill) ** (1.0 / 3.0)
    lo = np.zeros(3)
    hi = np.full(3, side)
    xs, qs, cents = [], [], []
    allp = np.zeros((0, 3))
    for k in range(n):
        t = tpls[int(kinds[k])]
        for _ in range(5000):
            q = _random_quats(rng, 1)[0]
            qw, qx, qy, qz = q
            Rm = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
                           [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
                           [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])
            c = lo + 3.05 * R + rng.random(3) * (side - 6.1 * R)
            p = c + t.rel_xyz @ Rm.T
            if np.any(p - R < lo) or np.any(p + R > hi):
                continue
            if len(allp):
                d = np.linalg.norm(allp[None, :, :] - p[:, None, :], axis=-1)
                if np.min(d) < 2 * R - max_overlap * R:
                    continue
            xs.append(c); qs.append(q)
            allp = np.concatenate([allp, p])
            break
        else:
            raise RuntimeError("clump placement did not converge; lower fill")
    x = np.array(xs)
    q = np.array(qs)
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    wl = box_walls(lo + 0.05 * R, hi - 0.05 * R) if walls else []    # outer spheres touch the walls
    return Scene(lo, hi, Em, num, corm, mum, wl, tpls, kinds, None, x, q,
                 rng.normal(scale=vel_sigma, size=(n, 3)), rng.normal(scale=omega_sigma, size=(n, 3)), h,
                 np.array(g, np.float64), r_max=R, name=f"packed_clumps_n{n}_seed{seed}")


def drum_bed(n=150, R=1e-3, drum_radius=0.03, length=0.03, omega=3.0, e=0.5, mu=0.5, E=1e7, nu=0.3, seed=0,
             h=1e-6, vel_sigma=1.0) -> Scene:
    """Clumps (rods, tetrahedra) in the lower part of a drum about x spinning at omega,
    pushed radially outwards until the outermost sphere overlaps the drum by 0.02 R."""
    s = packed_clumps(n=n, R=R, seed=seed, e=e, mu=mu, E=E, nu=nu, h=h, walls=False, fill=0.1, vel_sigma=vel_sigma)
    c = s.x - np.mean(s.x, axis=0)
    c[:, 2] -= 0.45 * drum_radius
    # outermost radial extent of every clump's spheres about the x axis
    def extent(cc):
        out = 0.0
        for k in range(len(cc)):
            t = s.templates[int(s.owner_template[k])]
            qw, qx, qy, qz = s.q[k]
            Rm = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
                           [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
                           [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])
            p = cc[k] + t.rel_xyz @ Rm.T
            out = max(out, float(np.max(np.hypot(p[:, 1], p[:, 2]) + t.radii)))
        return out
    lo_f, hi_f = 0.1, 10.0
    target = drum_radius + 0.02 * R
    for _ in range(60):
        mid = 0.5 * (lo_f + hi_f)
        cc = c.copy()
        cc[:, 1:] *= mid
        if extent(cc) > target:
            hi_f = mid
        else:
            lo_f = mid
    c[:, 1:] *= hi_f
    s.x = c
    axis = np.array([1.0, 0.0, 0.0])
    half = max(length / 2, float(np.max(np.abs(c[:, 0]))) + 3.1 * R)
    s.walls = [dict(type=CYLINDER, mat=0, p=np.zeros(3), n=axis, r0=drum_radius, omega=omega * axis),
               dict(type=PLANE, mat=0, p=np.array([-half, 0, 0]), n=axis.copy(), omega=omega * axis),
               dict(type=PLANE, mat=0, p=np.array([half, 0, 0]), n=-axis, omega=omega * axis)]
    s.box_lo = np.array([-half, -drum_radius, -drum_radius])
    s.box_hi = np.array([half, drum_radius, drum_radius])
    s.name = f"drum_bed_n{n}_seed{seed}"
    return s


def cone_bed(n=300, R=1e-3, half_angle_deg=30.0, r_orifice=0.01, e=0.5, mu=0.4, E=1e7, nu=0.3, seed=0, h=1e-6,
             vel_sigma=0.2, sink_z=0.004) -> Scene:
    """Spheres resting against a conical hopper wall (overlap 0.02 R) at random heights
    and azimuths, plus a few falling through the orifice towards a sink plane."""
    rng = np.random.default_rng(seed)
    tan = math.tan(math.radians(half_angle_deg))
    cosw = math.cos(math.atan(tan))
    z_top = 0.06
    pts = []
    tries = 0
    while len(pts) < n - 5 and tries < 100 * n:
        tries += 1
        z = rng.uniform(0.004, z_top - 0.004)
        phi = rng.uniform(0, 2 * math.pi)
        rw = r_orifice + z * tan          # wall point (rw, z); inward normal (-cos, sin)
        d = R - 0.02 * R
        rho = rw - d * cosw
        p = np.array([rho * math.cos(phi), rho * math.sin(phi), z + d * math.sin(math.atan(tan))])
        if all(np.sum((p - qq) ** 2) > (1.9 * R) ** 2 for qq in pts):
            pts.append(p)
    for k in range(5):
        pts.append(np.array([0.002 * k - 0.004, 0.0, sink_z + 0.0006]))
    pts = np.array(pts)
    m = len(pts)
    v = rng.normal(scale=vel_sigma, size=(m, 3))
    v[-5:] = [0.0, 0.0, -1.0]
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    axis = np.array([0.0, 0.0, 1.0])
    r_top = r_orifice + z_top * tan
    walls = [dict(type=CONE, mat=0, p=np.zeros(3), n=axis, r0=r_orifice, z0=0.0, r1=r_top, z1=z_top)]
    return Scene(np.array([-r_top, -r_top, -0.01]), np.array([r_top, r_top, z_top]), Em, num, corm, mum, walls,
                 [sphere_template(R)], np.zeros(m, np.int64), None, pts, _identity_quats(m), v,
                 rng.normal(scale=50.0, size=(m, 3)), h, np.array([0.0, 0.0, -9.81]),
                 sink=(np.array([0.0, 0.0, sink_z]), axis.copy()), r_max=R, name=f"cone_bed_n{m}_seed{seed}")


# ----------------------------------------------------------------------------- meshes

def box_facets(lo, hi, n=(1, 1, 1)):
    """Triangles (k, 3, 3) of the surface of the axis-aligned box [lo, hi], each face split
    into a grid of quads (n[a] divisions along axis a), two triangles per quad."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    tris = []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for side in (lo[a], hi[a]):
            us = np.linspace(lo[b], hi[b], n[b] + 1)
            vs = np.linspace(lo[c], hi[c], n[c] + 1)
            for i in range(n[b]):
                for j in range(n[c]):
                    q = []
                    for u, v in ((us[i], vs[j]), (us[i + 1], vs[j]), (us[i + 1], vs[j + 1]), (us[i], vs[j + 1])):
                        p = np.empty(3)
                        p[a], p[b], p[c] = side, u, v
                        q.append(p)
                    tris.append([q[0], q[1], q[2]])
                    tris.append([q[0], q[2], q[3]])
    return np.array(tris)


def rotated_z(tris, angle):
    c, s = math.cos(angle), math.sin(angle)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return np.asarray(tris) @ Rz.T


def facet_walls(tris, mat=0, p=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0)):
    return [dict(type=TRIANGLE, mat=mat, p=np.asarray(p, np.float64), n=np.zeros(3),
                 omega=np.asarray(omega, np.float64), tri=np.asarray(t, np.float64).reshape(9)) for t in tris]


def mixer_mesh(r_in=0.05, r_out=0.45, z0=0.02, z1=0.12, thickness=0.02, hub_r=0.05, hub_h=0.15):
    """The bladed mixer: four blades (boxes from r_in to r_out, z0 to z1, each face split
    into quads: 716 facets a blade) around a heptagonal hub prism (28 facets), 2,892
    facets in all, about the z axis."""
    blade = box_facets([r_in, -thickness / 2, z0], [r_out, thickness / 2, z1], n=(29, 1, 5))
    tris = [rotated_z(blade, k * math.pi / 2) for k in range(4)]
    ang = np.linspace(0, 2 * math.pi, 8)[:7]
    ring = np.stack([hub_r * np.cos(ang), hub_r * np.sin(ang)], axis=1)
    hub = []
    for k in range(7):
        a, b = ring[k], ring[(k + 1) % 7]
        pa0, pb0 = [a[0], a[1], 0.0], [b[0], b[1], 0.0]
        pa1, pb1 = [a[0], a[1], hub_h], [b[0], b[1], hub_h]
        hub += [[pa0, pb0, pb1], [pa0, pb1, pa1], [[0, 0, hub_h], pa1, pb1], [[0, 0, 0.0], pb0, pa0]]
    return np.concatenate(tris + [np.array(hub)])


def paddle_bed(n=300, R=1e-3, omega=150.0, e=0.5, mu=0.4, E=1e7, nu=0.3, seed=0, h=1e-6, vel_sigma=0.02) -> Scene:
    """Layers of spheres in a walled box around a paddle mesh (a tessellated thin box, 20
    facets) turning about the vertical axis through the box centre, over a static facet
    floor (8 facets) lying on the box floor: the bottom layer starts overlapping the floor
    facets by 0.001 R and spheres inside the paddle's sweep are struck by its faces,
    edges and corners."""
    rng = np.random.default_rng(seed)
    side = 0.024
    lo = np.zeros(3)
    hi = np.array([side, side, 0.02])
    cx = side / 2
    pl = np.array([cx - 0.008, cx - 0.001, 0.0015])
    ph = np.array([cx + 0.008, cx + 0.001, 0.009])
    paddle = box_facets(pl, ph, n=(2, 1, 1))
    floor = box_facets([0.0005, 0.0005, 0.0], [side - 0.0005, side - 0.0005, 0.0005], n=(2, 2, 1))
    floor = floor[np.abs(floor[:, :, 2] - 0.0005).max(axis=1) < 1e-12]      # its top face only
    pts = []
    z = 0.0005 + R - 0.001 * R
    while len(pts) < n and z < 0.018:
        tries = 0
        layer = []
        while tries < 4000 and len(pts) + len(layer) < n:
            tries += 1
            p = np.array([rng.uniform(R + 1e-4, side - R - 1e-4), rng.uniform(R + 1e-4, side - R - 1e-4), z])
            if np.all(p[:2] > pl[:2] - R - 1e-4) and np.all(p[:2] < ph[:2] + R + 1e-4) and p[2] < ph[2] + R + 1e-4:
                continue                              # clear of the paddle at time 0
            if all(np.linalg.norm(p - q) > 2 * R + 1e-5 for q in layer):
                layer.append(p)
        pts += layer
        z += 2 * R + 1e-4
    x = np.array(pts[:n])
    m = len(x)
    Em, num, corm, mum = _single_material(E, nu, e, mu)
    walls = box_walls(lo, hi) + facet_walls(floor) + facet_walls(paddle, p=(cx, cx, 0.0), omega=(0.0, 0.0, omega))
    return Scene(lo, hi, Em, num, corm, mum, walls, [sphere_template(R)], np.zeros(m, np.int64), None, x,
                 _identity_quats(m), rng.normal(scale=vel_sigma, size=(m, 3)), np.zeros((m, 3)), h,
                 np.array([0.0, 0.0, -9.81]), r_max=R, name=f"paddle_bed_n{m}")


def six_template(R: float, mat: int = 0, rho: float = RHO) -> Template:
    """Six tangent spheres on the vertices of a regular octahedron (centres at +-a on each
    axis, neighbours 2R apart)."""
    m1 = rho * 4.0 / 3.0 * math.pi * R ** 3
    i1 = 0.4 * m1 * R * R
    a = 2 * R / math.sqrt(2)
    xs = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, a], [0, 0, -a]], np.float64)
    I = 6 * i1 + 4 * m1 * a * a      # four of the six centres lie at distance a from each axis
    return Template(xs, np.full(6, R), np.full(6, mat, np.int32), 6 * m1, np.array([I, I, I]))


def mixer(n=4_000_000, clump="sphere", omega=2 * math.pi, mu=0.5, seed=7, R=None, vel_sigma=0.0,
          start="above") -> Scene:
    """The mixer of Sec. 5: elements released at rest from a cylindrical region of radius
    0.5 m and height 1/3 m above a bladed mixer mesh (2,892 facets) that turns at
    omega = 2 pi rad/s inside a cylindrical container with a floor; material and step of
    Sec. 5's table (rho 2600, E 1e9, nu 0.3, CoR 0.2, dt 5e-7 s; mu is not printed:
    0.5).  clump: "sphere", "rod3" (three tangent spheres) or "six" (six on an
    octahedron); the element size follows from n (lattice of the region), as the paper
    sizes elements to set the count.  start="bed": the same lattice starts at the floor
    instead, leaving out the points within an element's reach of the blades (at their
    pose at t = 0) and of the hub, so that the turning blades meet the elements from the
    first step (a short run then times mixing, not the fall onto the blades)."""
    rng = np.random.default_rng(seed)
    Rc, h_mix, H = 0.5, 0.15, 1.0 / 3.0
    ext = {"sphere": 1.0, "rod3": 3.0, "six": 1.0 + math.sqrt(2)}[clump]
    vol = math.pi * (Rc - 0.01) ** 2 * H
    pitch = (vol / n) ** (1.0 / 3.0)
    if R is None:
        R = pitch / (2.0 * ext * 1.05)
    tpl = {"sphere": sphere_template, "rod3": rod_template, "six": six_template}[clump](R, rho=2600.0)
    span = ext * R * 1.05
    g = np.arange(-Rc + span, Rc - span + 1e-12, pitch)
    z0 = span if start == "bed" else h_mix + span
    zs = np.arange(z0, z0 + H + (h_mix if start == "bed" else 0.0) - 2 * span + 1e-12, pitch)
    X, Y, Z = np.meshgrid(g, g, zs, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    pts = pts[np.hypot(pts[:, 0], pts[:, 1]) < Rc - span]
    if start == "bed":
        # blades: boxes from r_in to r_out, |y| <= thickness / 2, z0 to z1, turned by k pi / 2
        # (mixer_mesh's defaults), grown by the element's reach; hub prism inside radius hub_r
        keep = np.hypot(pts[:, 0], pts[:, 1]) > 0.05 + span
        for k in range(4):
            c, sn = math.cos(-k * math.pi / 2), math.sin(-k * math.pi / 2)
            u = c * pts[:, 0] - sn * pts[:, 1]
            v = sn * pts[:, 0] + c * pts[:, 1]
            inside = ((u > 0.05 - span) & (u < 0.45 + span) & (np.abs(v) < 0.01 + span)
                      & (pts[:, 2] > 0.02 - span) & (pts[:, 2] < 0.12 + span))
            keep &= ~inside
        keep &= ~((pts[:, 2] > 0.15 - span) & (np.hypot(pts[:, 0], pts[:, 1]) < 0.05 + span))
        pts = pts[keep]
    pts = pts[np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2]))][:n]
    m = len(pts)
    q = _identity_quats(m) if clump == "sphere" else _random_quats(rng, m)
    Em, num, corm, mum = _single_material(1e9, 0.3, 0.2, mu)
    lo = np.array([-Rc - 0.02, -Rc - 0.02, -0.01])
    hi = np.array([Rc + 0.02, Rc + 0.02, h_mix + H + 0.05])
    walls = [dict(type=PLANE, mat=0, p=np.array([0.0, 0.0, 0.0]), n=np.array([0.0, 0.0, 1.0])),
             dict(type=CYLINDER, mat=0, p=np.zeros(3), n=np.array([0.0, 0.0, 1.0]), r0=Rc)]
    walls += facet_walls(mixer_mesh(), p=(0.0, 0.0, 0.0), omega=(0.0, 0.0, omega))
    return Scene(lo, hi, Em, num, corm, mum, walls, [tpl], np.zeros(m, np.int64), None, pts, q,
                 rng.normal(scale=vel_sigma, size=(m, 3)), np.zeros((m, 3)), 5e-7, np.array([0.0, 0.0, -9.81]),
                 r_max=R, name=f"mixer_{clump}_{start}_n{m}", meta=dict(element_radius=R, facets=2892, start=start))
