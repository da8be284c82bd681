"""FP64 CPU oracle of the DEM contact pipeline (arXiv 2311.04648, Chrono DEM-Engine).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with the
CUDA library in ``paper_2311_04648_gb300`` and never imports it.

The arithmetic lives in ``dem_oracle.c`` (plain C, double precision, no fused
multiply-add); this module only compiles it with gcc and marshals numpy arrays.

Every function of the C oracle cites the passage of the paper it follows.  Parity pins
(tests/test_oracle_*.py) tie it to closed forms: brute force on tiny inputs, the Hertz
head-on collision, momentum and energy balances, static settling of a stack, the
incline rolling threshold, torque-free rigid-body motion and wall distance functions.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_HDR = os.path.join(_HERE, "dem_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdem_oracle.so")
_LOCK = threading.Lock()
_LIB = None

WALL_PLANE, WALL_CYLINDER, WALL_CONE, WALL_TRIANGLE = 0, 1, 2, 3
ERR_CAPACITY, ERR_DIVERGED = -2, -3


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libdem_oracle.so (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        # OpenMP where the toolchain has it (the parallel loops give the serial results)
        r = subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Wall(C.Structure):
    _fields_ = [("type", C.c_int32), ("mat", C.c_int32), ("p", C.c_double * 3), ("n", C.c_double * 3),
                ("r0", C.c_double), ("z0", C.c_double), ("r1", C.c_double), ("z1", C.c_double),
                ("omega", C.c_double * 3), ("tri", C.c_double * 9)]


class _World(C.Structure):
    _fields_ = [("n_owner", C.c_int64), ("n_sphere", C.c_int64), ("n_mat", C.c_int32), ("n_wall", C.c_int32),
                ("E", C.c_void_p), ("nu", C.c_void_p), ("cor", C.c_void_p), ("mu", C.c_void_p),
                ("walls", C.c_void_p),
                ("x", C.c_void_p), ("v", C.c_void_p), ("wb", C.c_void_p), ("q", C.c_void_p),
                ("mass", C.c_void_p), ("moi", C.c_void_p), ("active", C.c_void_p),
                ("owner", C.c_void_p), ("rloc", C.c_void_p), ("rad", C.c_void_p), ("mat", C.c_void_p),
                ("h", C.c_double), ("g", C.c_double * 3), ("gyroscopic", C.c_int32), ("has_sink", C.c_int32),
                ("sink_p", C.c_double * 3), ("sink_n", C.c_double * 3), ("v_err", C.c_double),
                ("hist", C.c_void_p), ("cell_list", C.c_int32), ("n_threads", C.c_int32), ("crr", C.c_void_p),
                ("family", C.c_void_p), ("contact_mask", C.c_void_p), ("motion", C.c_void_p),
                ("model", C.c_int32), ("model_params", C.c_void_p), ("step", C.c_int64)]

MODEL_HERTZ_MINDLIN, MODEL_BONDED_BREAKAGE = 0, 1
BREAKAGE_PARAMS = ("tension", "cohesion", "eta", "damping")


class FamilyMotion(C.Structure):
    _fields_ = [("fix_v", C.c_int32), ("fix_w", C.c_int32), ("v", C.c_double * 3), ("w", C.c_double * 3)]


class Contact(C.Structure):
    _fields_ = [("i", C.c_int64), ("j", C.c_int64), ("force", C.c_double * 3), ("point", C.c_double * 3),
                ("normal", C.c_double * 3), ("overlap", C.c_double), ("ut", C.c_double * 3), ("age", C.c_double),
                ("torque_force", C.c_double * 3), ("wc", C.c_double * 4)]


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = C.CDLL(build())
            L = _LIB
            P = C.c_void_p
            L.orc_history_new.restype = P
            L.orc_history_free.argtypes = [P]
            L.orc_history_size.restype = C.c_int64
            L.orc_history_size.argtypes = [P]
            L.orc_history_set.argtypes = [P, C.c_int64, P, P, P, P]
            L.orc_history_get.argtypes = [P, C.c_int64, P, P, P, P, P]
            L.orc_sphere_positions.argtypes = [P, P]
            L.orc_listed_pairs_f64.argtypes = [C.c_int64, P, P, P, P, C.c_double, C.c_int64, P, P, P]
            L.orc_listed_pairs_voxel_f32.argtypes = [C.c_int64, P, P, C.c_float, P, P, P, C.c_float,
                                                     C.c_int64, P, P, P]
            L.orc_listed_wall_pairs.argtypes = [P, P, C.c_double, C.c_int64, P, P, P]
            L.orc_eval.argtypes = [P, P, P, C.c_int64, P, P]
            L.orc_step.argtypes = [P, C.c_int64]
            L.orc_diagnostics.argtypes = [P, P, P, P, P, P]
            L.orc_effective_moduli.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, P, P]
            L.orc_history_set_wildcards.argtypes = [P, C.c_int64, P, P, P]
            L.orc_history_get_wildcards.argtypes = [P, C.c_int64, P, P]
            L.orc_max_threads.restype = C.c_int
            L.orc_max_threads.argtypes = []
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def max_threads() -> int:
    """Threads the oracle's parallel loops can use (1 without OpenMP)."""
    return int(lib().orc_max_threads())


def effective_moduli(E_a, nu_a, E_b, nu_b):
    es, gs = C.c_double(), C.c_double()
    lib().orc_effective_moduli(E_a, nu_a, E_b, nu_b, C.byref(es), C.byref(gs))
    return es.value, gs.value


def listed_pairs_f64(p, rad, owner, beta, sphere_active=None):
    """Sorted (i, j) pairs with ((dx^2+dy^2)+dz^2) < ((Ri+Rj)+2beta)^2, brute force."""
    p = np.ascontiguousarray(p, np.float64)
    rad = np.ascontiguousarray(rad, np.float64)
    owner = np.ascontiguousarray(owner, np.int64)
    act = None if sphere_active is None else np.ascontiguousarray(sphere_active, np.uint8)
    n = len(rad)
    cap = max(16, 8 * n)
    while True:
        pi = np.empty(cap, np.int64)
        pj = np.empty(cap, np.int64)
        cnt = C.c_int64()
        rc = lib().orc_listed_pairs_f64(n, _ptr(p), _ptr(rad), _ptr(owner), _ptr(act), beta, cap,
                                        C.byref(cnt), _ptr(pi), _ptr(pj))
        if rc == ERR_CAPACITY:
            cap = cnt.value
            continue
        assert rc == 0
        return pi[:cnt.value].copy(), pj[:cnt.value].copy()


def listed_pairs_voxel_f32(cell, off, L, rad, owner, beta, sphere_active=None):
    """The same set with positions encoded as int cell + float32 offset (single precision)."""
    cell = np.ascontiguousarray(cell, np.int32)
    off = np.ascontiguousarray(off, np.float32)
    rad = np.ascontiguousarray(rad, np.float32)
    owner = np.ascontiguousarray(owner, np.int64)
    act = None if sphere_active is None else np.ascontiguousarray(sphere_active, np.uint8)
    n = len(rad)
    cap = max(16, 8 * n)
    while True:
        pi = np.empty(cap, np.int64)
        pj = np.empty(cap, np.int64)
        cnt = C.c_int64()
        rc = lib().orc_listed_pairs_voxel_f32(n, _ptr(cell), _ptr(off), C.c_float(L), _ptr(rad), _ptr(owner),
                                              _ptr(act), C.c_float(beta), cap, C.byref(cnt), _ptr(pi), _ptr(pj))
        if rc == ERR_CAPACITY:
            cap = cnt.value
            continue
        assert rc == 0
        return pi[:cnt.value].copy(), pj[:cnt.value].copy()


class OracleWorld:
    """A world for the oracle, built from a scene description (duck-typed; see
    paper_2311_04648_gb300.workloads.Scene for the fields read here)."""

    def __init__(self, scene, cell_list: bool = False, threads: int = 1):
        s = scene
        self.n_mat = len(s.E)
        self.E = np.ascontiguousarray(s.E, np.float64)
        self.nu = np.ascontiguousarray(s.nu, np.float64)
        self.cor = np.ascontiguousarray(s.cor, np.float64).reshape(self.n_mat, self.n_mat)
        self.mu = np.ascontiguousarray(s.mu, np.float64).reshape(self.n_mat, self.n_mat)
        crr = getattr(s, "crr", None)
        self.crr = (np.zeros((self.n_mat, self.n_mat)) if crr is None
                    else np.ascontiguousarray(crr, np.float64).reshape(self.n_mat, self.n_mat))
        walls = list(s.walls)
        self.walls = (Wall * max(1, len(walls)))()
        for k, wd in enumerate(walls):
            W = self.walls[k]
            W.type = int(wd["type"]); W.mat = int(wd["mat"])
            for a in range(3):
                W.p[a] = float(wd["p"][a]); W.n[a] = float(wd["n"][a]); W.omega[a] = float(wd.get("omega", (0, 0, 0))[a])
            W.r0 = float(wd.get("r0", 0.0)); W.z0 = float(wd.get("z0", 0.0))
            W.r1 = float(wd.get("r1", 0.0)); W.z1 = float(wd.get("z1", 0.0))
            if "tri" in wd:
                for a in range(9):
                    W.tri[a] = float(np.asarray(wd["tri"], np.float64).reshape(9)[a])
        self.n_wall = len(walls)
        # expand templates x instances into per-owner and per-sphere arrays
        M = len(s.owner_template)
        scale = np.ones(M) if s.owner_scale is None else np.asarray(s.owner_scale, np.float64)
        owner, rloc, rad, mat = [], [], [], []
        mass = np.empty(M)
        moi = np.empty((M, 3))
        for o in range(M):
            t = s.templates[int(s.owner_template[o])]
            sc = scale[o]
            mass[o] = t.mass * sc * sc * sc
            moi[o] = np.asarray(t.moi, np.float64) * (sc * sc * sc * sc * sc)
            for k in range(len(t.radii)):
                owner.append(o)
                rloc.append(np.asarray(t.rel_xyz[k], np.float64) * sc)
                rad.append(t.radii[k] * sc)
                mat.append(t.mats[k])
        self.owner = np.ascontiguousarray(owner, np.int64)
        self.rloc = np.ascontiguousarray(np.reshape(rloc, (-1, 3)), np.float64)
        self.rad = np.ascontiguousarray(rad, np.float64)
        self.mat = np.ascontiguousarray(mat, np.int32)
        self.mass = mass
        self.moi = np.ascontiguousarray(moi)
        self.x = np.ascontiguousarray(s.x, np.float64).reshape(M, 3).copy()
        self.v = np.ascontiguousarray(s.v, np.float64).reshape(M, 3).copy()
        self.wb = np.ascontiguousarray(s.wb, np.float64).reshape(M, 3).copy()
        self.q = np.ascontiguousarray(s.q, np.float64).reshape(M, 4).copy()
        self.active = np.ones(M, np.int32)
        self._w = _World()
        w = self._w
        w.n_owner = M; w.n_sphere = len(self.rad); w.n_mat = self.n_mat; w.n_wall = self.n_wall
        w.E = _ptr(self.E); w.nu = _ptr(self.nu); w.cor = _ptr(self.cor); w.mu = _ptr(self.mu)
        w.crr = _ptr(self.crr)
        w.walls = C.cast(self.walls, C.c_void_p)
        w.x = _ptr(self.x); w.v = _ptr(self.v); w.wb = _ptr(self.wb); w.q = _ptr(self.q)
        w.mass = _ptr(self.mass); w.moi = _ptr(self.moi); w.active = _ptr(self.active)
        w.owner = _ptr(self.owner); w.rloc = _ptr(self.rloc); w.rad = _ptr(self.rad); w.mat = _ptr(self.mat)
        w.h = float(s.h)
        for a in range(3):
            w.g[a] = float(s.g[a])
        w.gyroscopic = 1 if getattr(s, "gyroscopic", True) else 0
        sink = getattr(s, "sink", None)
        if sink is not None:
            w.has_sink = 1
            for a in range(3):
                w.sink_p[a] = float(sink[0][a]); w.sink_n[a] = float(sink[1][a])
        w.v_err = float(getattr(s, "v_err", 0.0) or 0.0)
        # family tags: per-owner family, contact mask between families, prescribed motion
        fam = getattr(s, "family", None)
        self.family = None if fam is None else np.ascontiguousarray(fam, np.uint8).reshape(M)
        masked = getattr(s, "family_masked", None)
        self.contact_mask = None
        if masked:
            self.contact_mask = np.ones((256, 256), np.uint8)
            for a, b in masked:
                self.contact_mask[a, b] = 0
                self.contact_mask[b, a] = 0
        motion = getattr(s, "family_motion", None)
        self.motion = None
        if motion:
            self.motion = (FamilyMotion * 256)()
            for f, (vel, om) in motion.items():
                fm = self.motion[int(f)]
                if vel is not None:
                    fm.fix_v = 1
                    for a in range(3):
                        fm.v[a] = float(vel[a])
                if om is not None:
                    fm.fix_w = 1
                    for a in range(3):
                        fm.w[a] = float(om[a])
        model = getattr(s, "force_model", None)
        self.model_params = None
        if model == "bonded_breakage":
            w.model = MODEL_BONDED_BREAKAGE
            par = s.model_params
            self.model_params = np.array([float(par[k]) for k in BREAKAGE_PARAMS], np.float64)
            w.model_params = _ptr(self.model_params)
        elif model not in (None, "hertz_mindlin"):
            raise ValueError(f"unknown force model {model!r}")
        w.family = _ptr(self.family)
        w.contact_mask = _ptr(self.contact_mask)
        w.motion = C.cast(self.motion, C.c_void_p) if self.motion is not None else None
        w.hist = lib().orc_history_new()
        w.cell_list = 1 if cell_list else 0
        w.n_threads = int(threads)

    def __del__(self):
        try:
            if self._w.hist:
                lib().orc_history_free(self._w.hist)
                self._w.hist = None
        except Exception:
            pass

    @property
    def n_owner(self):
        return self._w.n_owner

    @property
    def n_sphere(self):
        return self._w.n_sphere

    def _wp(self):
        return C.cast(C.pointer(self._w), C.c_void_p)

    def step(self, n: int = 1) -> int:
        return lib().orc_step(self._wp(), int(n))

    def sphere_positions(self):
        p = np.empty((self.n_sphere, 3))
        lib().orc_sphere_positions(self._wp(), _ptr(p))
        return p

    def sphere_active(self):
        return self.active[self.owner].astype(np.uint8)

    def listed_wall_pairs(self, p, beta):
        p = np.ascontiguousarray(p, np.float64)
        cap = max(16, 4 * self.n_sphere)
        while True:
            si = np.empty(cap, np.int64)
            wi = np.empty(cap, np.int64)
            cnt = C.c_int64()
            rc = lib().orc_listed_wall_pairs(self._wp(), _ptr(p), beta, cap, C.byref(cnt), _ptr(si), _ptr(wi))
            if rc == ERR_CAPACITY:
                cap = cnt.value
                continue
            assert rc == 0
            return si[:cnt.value].copy(), wi[:cnt.value].copy()

    def eval(self):
        """Per-owner force (gravity included) and torque plus all contacts, at the
        current state, without advancing it."""
        M = self.n_owner
        F = np.empty((M, 3))
        T = np.empty((M, 3))
        cap = max(64, 8 * self.n_sphere)
        while True:
            buf = (Contact * cap)()
            cnt = C.c_int64()
            rc = lib().orc_eval(self._wp(), _ptr(F), _ptr(T), cap, C.byref(cnt), C.cast(buf, C.c_void_p))
            if rc == ERR_CAPACITY:
                cap = cnt.value
                continue
            assert rc == 0
            n = cnt.value
            arr = np.ctypeslib.as_array(buf)[:n].copy() if n else np.zeros(0, dtype=np.ctypeslib.as_array(buf).dtype)
            return F, T, arr

    def history(self, with_age=False):
        """Stored tangential history (i, j, ut[n, 3]) and, with_age, the contacts' ages."""
        h = self._w.hist
        n = lib().orc_history_size(h)
        i = np.empty(max(n, 1), np.int64)
        j = np.empty(max(n, 1), np.int64)
        ut = np.empty((max(n, 1), 3))
        age = np.empty(max(n, 1))
        cnt = C.c_int64()
        rc = lib().orc_history_get(h, max(n, 1), C.byref(cnt), _ptr(i), _ptr(j), _ptr(ut), _ptr(age))
        assert rc == 0
        if with_age:
            return i[:n].copy(), j[:n].copy(), ut[:n].copy(), age[:n].copy()
        return i[:n].copy(), j[:n].copy(), ut[:n].copy()

    def set_history(self, i, j, ut, age=None):
        i = np.ascontiguousarray(i, np.int64)
        j = np.ascontiguousarray(j, np.int64)
        ut = np.ascontiguousarray(ut, np.float64).reshape(-1, 3)
        age = None if age is None else np.ascontiguousarray(age, np.float64).reshape(-1)
        rc = lib().orc_history_set(self._w.hist, len(i), _ptr(i), _ptr(j), _ptr(ut), _ptr(age))
        assert rc == 0

    def set_wildcards(self, i, j, wc):
        """Model wildcards wc[n, 4] of the contacts (i, j) (bonded breakage: bond state,
        bond length); entries not in the history are added with zero history."""
        i = np.ascontiguousarray(i, np.int64)
        j = np.ascontiguousarray(j, np.int64)
        wc = np.ascontiguousarray(wc, np.float64).reshape(-1, 4)
        assert lib().orc_history_set_wildcards(self._w.hist, len(i), _ptr(i), _ptr(j), _ptr(wc)) == 0

    def wildcards(self):
        n = lib().orc_history_size(self._w.hist)
        wc = np.empty((max(n, 1), 4))
        cnt = C.c_int64()
        assert lib().orc_history_get_wildcards(self._w.hist, max(n, 1), C.byref(cnt), _ptr(wc)) == 0
        return wc[:n].copy()

    def diagnostics(self):
        ke, pe, el = C.c_double(), C.c_double(), C.c_double()
        mom = np.empty(3)
        L = np.empty(3)
        lib().orc_diagnostics(self._wp(), C.byref(ke), C.byref(pe), C.byref(el), _ptr(mom), _ptr(L))
        return {"ke": ke.value, "pe": pe.value, "elastic": el.value, "momentum": mom, "angmom": L}
