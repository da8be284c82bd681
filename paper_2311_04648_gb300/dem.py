"""Thin ctypes binding of libdem_gb300.so (include/dem.h).

Every ``dem_*`` function of the C ABI is available under the same name on the object
returned by :func:`load`, with argument types set; :class:`World` and :class:`Batch`
only marshal numpy arrays into those calls.  All computation happens in the CUDA
library; if it cannot be loaded this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdem_gb300.so")
_LOCK = threading.Lock()
_LIB = None

OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_CAPACITY, ERR_DIVERGED, ERR_TIMEOUT, ERR_OVERFLOW, ERR_NOMEM, ERR_UNSUPPORTED = range(10)
PRECISION = {"fp64": 0, "voxel_fp32": 1}
SCHEDULE = {"every_step": 0, "velocity_bound": 1, "learned": 2}
PROP_COR, PROP_MU, PROP_CRR = 0, 1, 2
MODEL = {"default": 0, "hertz_mindlin": 1, "bonded_breakage": 2}
BREAKAGE_PARAMS = ("tension", "cohesion", "eta", "damping")
WALL_PLANE, WALL_CYLINDER, WALL_CONE, WALL_TRIANGLE = 0, 1, 2, 3


class DemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dem status {status}: {msg}")
        self.status = status


class WorldDesc(C.Structure):
    _fields_ = [("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("precision", C.c_int32),
                ("schedule", C.c_int32), ("device", C.c_int32), ("gyroscopic", C.c_int32),
                ("max_spheres", C.c_int64), ("margin_max", C.c_double), ("stream", C.c_void_p),
                ("detect_stream", C.c_void_p), ("alloc", C.c_void_p), ("free", C.c_void_p),
                ("alloc_ctx", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rebuilds", C.c_int64), ("audit_fallbacks", C.c_int64),
                ("overflow_regrows", C.c_int64), ("listed_pairs", C.c_int64), ("wall_pairs", C.c_int64),
                ("active_contacts", C.c_int64), ("list_capacity", C.c_int32), ("list_max_row", C.c_int32),
                ("margin", C.c_double), ("displacement_bound", C.c_double), ("max_speed", C.c_double),
                ("mean_steps_per_build", C.c_double), ("cell_size", C.c_double), ("n_cells", C.c_int64),
                ("ms_detect", C.c_double), ("ms_force", C.c_double), ("ms_hash", C.c_double),
                ("ms_link", C.c_double), ("n_detect", C.c_int64), ("n_force", C.c_int64), ("ms_total", C.c_double),
                ("last_cycle", C.c_int64), ("schedule_samples", C.c_int64), ("ms_integrate", C.c_double),
                ("n_integrate", C.c_int64), ("spheres_with_entries", C.c_int64),
                ("pair_steps", C.c_int64), ("busy_steps", C.c_int64), ("derived_constants", C.c_int32),
                ("counting_sort", C.c_int32), ("ms_contact_eval", C.c_double), ("n_contact_eval", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("contact_block", C.c_int32), ("integrate_block", C.c_int32), ("narrow_block", C.c_int32),
                ("detect_inline", C.c_int32), ("step_ms", C.c_double), ("cell_factor", C.c_double),
                ("integrate_staged", C.c_int32), ("contact_lean", C.c_int32), ("fused_block", C.c_int32),
                ("margin", C.c_double), ("contact_integrates", C.c_int32), ("binning", C.c_int32),
                ("narrow_staged", C.c_int32),
                ("contact_screen", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Diagnostics(C.Structure):
    _fields_ = [("kinetic", C.c_double), ("potential", C.c_double), ("elastic", C.c_double),
                ("momentum", C.c_double * 3), ("angular_momentum", C.c_double * 3)]


def _sigs(L):
    P, I32, I64, D, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "dem_world_create": [P, P], "dem_world_destroy": [P], "dem_add_material": [P, D, D, D, D, D, P],
        "dem_set_material_pair": [P, I32, I32, I32, D], "dem_add_box_walls": [P, I32, P],
        "dem_add_plane": [P, P, P, I32, P], "dem_add_cylinder": [P, P, P, D, I32, D, P],
        "dem_add_cone_segment": [P, P, P, D, D, D, D, I32, P], "dem_set_wall_spin": [P, I32, P],
        "dem_add_clump_template": [P, I32, P, P, P, D, P, P], "dem_add_clumps": [P, I32, I64, P, P, P, P, P, P],
        "dem_add_clumps_mixed": [P, I64, P, P, P, P, P, P, P],
        "dem_set_timestep": [P, D], "dem_set_gravity": [P, P], "dem_set_error_velocity": [P, D],
        "dem_set_margin": [P, D], "dem_set_sink": [P, P, P], "dem_load_schedule_model": [P, P, SZ],
        "dem_initialize": [P], "dem_step": [P, I64], "dem_sync": [P], "dem_get_stream": [P, P],
        "dem_set_profiling": [P, I32], "dem_set_tuning": [P, P], "dem_get_tuning": [P, P],
        "dem_autotune": [P, I32, C.c_char_p, P], "dem_set_graphs": [P, I32],
        "dem_get_owner_state": [P, I64, I64, P, P, P, P], "dem_set_owner_state": [P, I64, I64, P, P, P, P],
        "dem_get_sphere_positions": [P, I64, I64, P, P], "dem_get_sphere_voxels": [P, I64, I64, P, P, P],
        "dem_get_contacts": [P, I64, P, P, P, P, P, P, P], "dem_get_listed_pairs": [P, I64, P, P, P],
        "dem_get_listed_wall_pairs": [P, I64, P, P, P], "dem_get_owner_forces": [P, I64, I64, P, P],
        "dem_set_history": [P, I64, P, P, P], "dem_set_history_age": [P, I64, P, P, P, P],
        "dem_get_contact_rolling": [P, I64, P, P, P],
        "dem_add_mesh": [P, I64, P, I32, P, P, P],
        "dem_set_force_model": [P, I32, P, I32], "dem_set_contact_wildcards": [P, I64, P, P, P],
        "dem_get_contact_wildcards": [P, I64, P, P],
        "dem_set_family": [P, I64, I64, P], "dem_set_family_motion": [P, I32, P, P],
        "dem_set_family_contacts": [P, I32, I32, I32], "dem_set_active_box": [P, P, P, I32, I32], "dem_get_stats": [P, P], "dem_get_diagnostics": [P, P],
        "dem_save_state": [P, P, SZ, P], "dem_load_state": [P, P, SZ],
        "dem_batch_create": [I32, P, P], "dem_batch_world": [P, I32, P], "dem_batch_initialize": [P],
        "dem_batch_step": [P, I64], "dem_batch_destroy": [P],
        "dem_schedule_collect": [P, I32], "dem_schedule_train": [P, I32, C.c_float, C.c_uint64, P],
        "dem_schedule_export": [P, P, SZ, P],
        "dem_util_radix_sort_u32": [I64, P, P, I32, P, P],
        "dem_util_mlp_forward": [P, I32, P, P], "dem_util_mlp_loss_grad": [P, I32, P, P, P, P],
        "dem_util_radix_sort_u32_noalloc": [I64, P, P, I32, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.dem_last_error.argtypes = [P]
    L.dem_last_error.restype = C.c_char_p
    L.dem_util_noalloc_error.argtypes = []
    L.dem_util_noalloc_error.restype = C.c_char_p


def load(path: str | None = None):
    """Load the CUDA library (building it first if it is absent and nvcc exists)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                from . import build as _b
                _b.build()
            if not os.path.exists(p):
                raise DemError(ERR_UNSUPPORTED, f"CUDA library {p} is missing; build it with "
                                                "python -m paper_2311_04648_gb300.build")
            _LIB = C.CDLL(p)
            _sigs(_LIB)
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _check(status, handle=None):
    if status != OK:
        L = load()
        msg = L.dem_last_error(handle).decode() if L.dem_last_error(handle) else ""
        raise DemError(status, msg)


def radix_sort_u32(keys, vals, bits=32):
    keys = np.ascontiguousarray(keys, np.uint32)
    vals = np.ascontiguousarray(vals, np.uint32)
    ko = np.empty_like(keys)
    vo = np.empty_like(vals)
    _check(load().dem_util_radix_sort_u32(len(keys), _p(keys), _p(vals), bits, _p(ko), _p(vo)))
    return ko, vo


MLP_NPARAM = 64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2


def mlp_forward(params, X):
    params = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32).reshape(-1, 16)
    out = np.empty((len(X), 2), np.float32)
    _check(load().dem_util_mlp_forward(_p(params), len(X), _p(X), _p(out)))
    return out


def mlp_loss_grad(params, X, Y):
    params = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32).reshape(-1, 16)
    Y = np.ascontiguousarray(Y, np.float32).reshape(-1, 2)
    loss = C.c_float()
    grad = np.empty(MLP_NPARAM, np.float32)
    _check(load().dem_util_mlp_loss_grad(_p(params), len(X), _p(X), _p(Y), C.byref(loss), _p(grad)))
    return loss.value, grad


# device allocator callbacks of dem_world_desc: void *alloc(size_t, void *ctx), void free(void *, void *ctx)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class World:
    """One simulated world (or, with ``_handle``, one scene of a :class:`Batch`).

    ``stream`` / ``detect_stream``: cudaStream_t handles (ints) the library runs on
    instead of its own.  ``alloc(nbytes) -> device pointer`` and ``free(pointer)``: a
    device allocator the library takes all its memory from (both or neither); they must
    stay callable until the world is closed."""

    def __init__(self, box_lo=(0, 0, 0), box_hi=(1, 1, 1), precision="fp64", schedule="every_step", device=0,
                 gyroscopic=True, margin_max=0.0, stream=None, detect_stream=None, alloc=None, free=None,
                 _handle=None, _batch=None):
        self.L = load()
        self._batch = _batch
        self._callbacks = None
        if _handle is not None:
            self.h = _handle
            return
        d = WorldDesc()
        for a in range(3):
            d.box_lo[a] = float(box_lo[a])
            d.box_hi[a] = float(box_hi[a])
        d.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        d.schedule = SCHEDULE[schedule] if isinstance(schedule, str) else int(schedule)
        d.device = device
        d.gyroscopic = 1 if gyroscopic else 0
        d.margin_max = margin_max
        d.stream = stream
        d.detect_stream = detect_stream
        if (alloc is None) != (free is None):
            raise ValueError("alloc and free go together")
        if alloc is not None:
            cb_a = ALLOC_FN(lambda nbytes, ctx: alloc(int(nbytes)) or None)
            cb_f = FREE_FN(lambda ptr, ctx: free(ptr))
            self._callbacks = (cb_a, cb_f)            # alive until the world is destroyed
            d.alloc = C.cast(cb_a, C.c_void_p)
            d.free = C.cast(cb_f, C.c_void_p)
        h = C.c_void_p()
        _check(self.L.dem_world_create(C.byref(d), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self._batch is None:
            self.L.dem_world_destroy(self.h)
        self.h = None
        self._callbacks = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        _check(st, self.h)

    # ---- set-up
    def add_material(self, E, nu, cor, mu, crr=0.0):
        i = C.c_int32()
        self._c(self.L.dem_add_material(self.h, E, nu, cor, mu, crr, C.byref(i)))
        return i.value

    def set_material_pair(self, prop, a, b, value):
        self._c(self.L.dem_set_material_pair(self.h, prop, a, b, value))

    def add_box_walls(self, mat):
        i = C.c_int32()
        self._c(self.L.dem_add_box_walls(self.h, mat, C.byref(i)))
        return i.value

    def add_plane(self, p, n, mat):
        i = C.c_int32()
        self._c(self.L.dem_add_plane(self.h, _p(_f64(p)), _p(_f64(n)), mat, C.byref(i)))
        return i.value

    def add_cylinder(self, c, axis, radius, mat, omega=0.0):
        i = C.c_int32()
        self._c(self.L.dem_add_cylinder(self.h, _p(_f64(c)), _p(_f64(axis)), radius, mat, omega, C.byref(i)))
        return i.value

    def add_mesh(self, vertices, mat, axis_point=(0, 0, 0), omega=(0, 0, 0)):
        """A rigid triangle mesh (facets vertices[n, 3, 3]) turning with omega about
        axis_point; returns the first facet's wall id."""
        v = _f64(vertices).reshape(-1, 9)
        i = C.c_int32()
        self._c(self.L.dem_add_mesh(self.h, len(v), _p(v), int(mat), _p(_f64(axis_point)), _p(_f64(omega)),
                                    C.byref(i)))
        return i.value

    def add_cone_segment(self, p, axis, r0, z0, r1, z1, mat):
        i = C.c_int32()
        self._c(self.L.dem_add_cone_segment(self.h, _p(_f64(p)), _p(_f64(axis)), r0, z0, r1, z1, mat, C.byref(i)))
        return i.value

    def set_wall_spin(self, wall, omega):
        self._c(self.L.dem_set_wall_spin(self.h, wall, _p(_f64(omega))))

    def add_clump_template(self, rel_xyz, radii, mats, mass, moi):
        rel = _f64(rel_xyz).reshape(-1, 3)
        rad = _f64(radii)
        mt = np.ascontiguousarray(mats, np.int32)
        i = C.c_int32()
        self._c(self.L.dem_add_clump_template(self.h, len(rad), _p(rel), _p(rad), _p(mt), mass, _p(_f64(moi)),
                                              C.byref(i)))
        return i.value

    def add_clumps(self, tid, xyz, quat=None, vel=None, omega=None, scale=None):
        x = _f64(xyz).reshape(-1, 3)
        n = len(x)
        f = C.c_int64()
        q = None if quat is None else _f64(quat).reshape(n, 4)
        v = None if vel is None else _f64(vel).reshape(n, 3)
        w = None if omega is None else _f64(omega).reshape(n, 3)
        s = None if scale is None else _f64(scale).reshape(n)
        if np.isscalar(tid) or np.ndim(tid) == 0:
            self._c(self.L.dem_add_clumps(self.h, int(tid), n, _p(x), _p(q), _p(v), _p(w), _p(s), C.byref(f)))
        else:
            t = np.ascontiguousarray(tid, np.int32).reshape(n)
            self._c(self.L.dem_add_clumps_mixed(self.h, n, _p(t), _p(x), _p(q), _p(v), _p(w), _p(s), C.byref(f)))
        return f.value

    def set_timestep(self, h):
        self._c(self.L.dem_set_timestep(self.h, h))

    def set_gravity(self, g):
        self._c(self.L.dem_set_gravity(self.h, _p(_f64(g))))

    def set_error_velocity(self, v):
        self._c(self.L.dem_set_error_velocity(self.h, v))

    def set_margin(self, beta):
        self._c(self.L.dem_set_margin(self.h, beta))

    def set_sink(self, p, n):
        self._c(self.L.dem_set_sink(self.h, _p(_f64(p)), _p(_f64(n))))

    def initialize(self):
        self._c(self.L.dem_initialize(self.h))

    # ---- stepping
    def step(self, n=1):
        self._c(self.L.dem_step(self.h, int(n)))

    def sync(self):
        self._c(self.L.dem_sync(self.h))

    def schedule_collect(self, on=True):
        self._c(self.L.dem_schedule_collect(self.h, 1 if on else 0))

    def schedule_train(self, epochs=30, lr=1e-3, seed=0):
        loss = C.c_float()
        self._c(self.L.dem_schedule_train(self.h, epochs, lr, seed, C.byref(loss)))
        return loss.value

    def schedule_export(self):
        used = C.c_size_t()
        self.L.dem_schedule_export(self.h, None, 0, C.byref(used))
        buf = (C.c_uint8 * used.value)()
        self._c(self.L.dem_schedule_export(self.h, C.cast(buf, C.c_void_p), used.value, C.byref(used)))
        return bytes(buf)

    def load_schedule_model(self, blob: bytes):
        buf = (C.c_uint8 * len(blob)).from_buffer_copy(blob)
        self._c(self.L.dem_load_schedule_model(self.h, C.cast(buf, C.c_void_p), len(blob)))

    def autotune(self, steps=50, cache_path=None):
        t = Tuning()
        cp = cache_path.encode() if cache_path else None
        self._c(self.L.dem_autotune(self.h, steps, cp, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        self._c(self.L.dem_get_tuning(self.h, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        self._c(self.L.dem_set_tuning(self.h, C.byref(t)))

    def tuning(self):
        t = Tuning()
        self._c(self.L.dem_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    def set_graphs(self, on=True):
        self._c(self.L.dem_set_graphs(self.h, 1 if on else 0))

    def set_profiling(self, on=True):
        self._c(self.L.dem_set_profiling(self.h, 1 if on else 0))

    def stream(self):
        s = C.c_void_p()
        self._c(self.L.dem_get_stream(self.h, C.byref(s)))
        return s.value

    # ---- read back
    def owner_state(self, first=0, n=None, out=None):
        """Positions, orientations, velocities and body-frame angular velocities of owners
        first..first+n-1 as four float64 arrays; ``out``: four C-contiguous float64 arrays
        of shapes (n, 3), (n, 4), (n, 3), (n, 3) to fill instead (pinned host memory is
        written by the device directly)."""
        if n is None:
            n = self.n_owner
        if out is not None:
            x, q, v, w = out
            for a, c in zip(out, (3, 4, 3, 3)):
                if a.dtype != np.float64 or a.shape != (n, c) or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be C-contiguous float64 of shapes (n,3),(n,4),(n,3),(n,3)")
        else:
            x = np.empty((n, 3)); q = np.empty((n, 4)); v = np.empty((n, 3)); w = np.empty((n, 3))
        self._c(self.L.dem_get_owner_state(self.h, first, n, _p(x), _p(q), _p(v), _p(w)))
        return x, q, v, w

    def set_owner_state(self, first, xyz=None, quat=None, vel=None, omega=None):
        arrs = [a for a in (xyz, quat, vel, omega) if a is not None]
        n = len(np.asarray(arrs[0]).reshape(len(arrs[0]), -1))
        self._c(self.L.dem_set_owner_state(self.h, first, n, _p(_f64(xyz)), _p(_f64(quat)), _p(_f64(vel)),
                                           _p(_f64(omega))))

    def sphere_positions(self, first=0, n=None):
        if n is None:
            n = self.n_sphere
        x = np.empty((n, 3)); r = np.empty(n)
        self._c(self.L.dem_get_sphere_positions(self.h, first, n, _p(x), _p(r)))
        return x, r

    def sphere_voxels(self, first=0, n=None):
        if n is None:
            n = self.n_sphere
        c = np.empty((n, 3), np.int32); o = np.empty((n, 3), np.float32); e = C.c_double()
        self._c(self.L.dem_get_sphere_voxels(self.h, first, n, _p(c), _p(o), C.byref(e)))
        return c, o, e.value

    def contacts(self):
        cnt = C.c_int64()
        st = self.L.dem_get_contacts(self.h, 0, C.byref(cnt), None, None, None, None, None, None)
        if st not in (OK, ERR_CAPACITY):
            self._c(st)
        n = cnt.value
        i = np.empty(n, np.int64); j = np.empty(n, np.int64); f = np.empty((n, 3)); p = np.empty((n, 3))
        o = np.empty(n); h = np.empty((n, 3))
        self._c(self.L.dem_get_contacts(self.h, n, C.byref(cnt), _p(i), _p(j), _p(f), _p(p), _p(o), _p(h)))
        return dict(i=i, j=j, force=f, point=p, overlap=o, history=h)

    def listed_pairs(self):
        cnt = C.c_int64()
        st = self.L.dem_get_listed_pairs(self.h, 0, C.byref(cnt), None, None)
        if st not in (OK, ERR_CAPACITY):
            self._c(st)
        n = cnt.value
        i = np.empty(n, np.int64); j = np.empty(n, np.int64)
        self._c(self.L.dem_get_listed_pairs(self.h, n, C.byref(cnt), _p(i), _p(j)))
        return i, j

    def listed_wall_pairs(self):
        cnt = C.c_int64()
        st = self.L.dem_get_listed_wall_pairs(self.h, 0, C.byref(cnt), None, None)
        if st not in (OK, ERR_CAPACITY):
            self._c(st)
        n = cnt.value
        s = np.empty(n, np.int64); w = np.empty(n, np.int64)
        self._c(self.L.dem_get_listed_wall_pairs(self.h, n, C.byref(cnt), _p(s), _p(w)))
        return s, w

    def owner_forces(self, first=0, n=None):
        if n is None:
            n = self.n_owner
        F = np.empty((n, 3)); T = np.empty((n, 3))
        self._c(self.L.dem_get_owner_forces(self.h, first, n, _p(F), _p(T)))
        return F, T

    def set_history(self, i, j, ut, age=None):
        i = np.ascontiguousarray(i, np.int64); j = np.ascontiguousarray(j, np.int64)
        ut = _f64(ut).reshape(-1, 3)
        if age is None:
            self._c(self.L.dem_set_history(self.h, len(i), _p(i), _p(j), _p(ut)))
        else:
            self._c(self.L.dem_set_history_age(self.h, len(i), _p(i), _p(j), _p(ut), _p(_f64(age))))

    # ---- contact force models
    def set_force_model(self, model, params=None):
        """model: "default", "hertz_mindlin" (the default through the functor path) or
        "bonded_breakage" with params {tension, cohesion, eta, damping}."""
        par = None
        if model == "bonded_breakage":
            par = np.array([float(params[k]) for k in BREAKAGE_PARAMS], np.float64)
        self._c(self.L.dem_set_force_model(self.h, MODEL[model], _p(par) if par is not None else None,
                                           0 if par is None else len(par)))

    def set_contact_wildcards(self, i, j, wc):
        i = np.ascontiguousarray(i, np.int64); j = np.ascontiguousarray(j, np.int64)
        wc = _f64(wc).reshape(-1, 4)
        self._c(self.L.dem_set_contact_wildcards(self.h, len(i), _p(i), _p(j), _p(wc)))

    def contact_wildcards(self):
        cnt = C.c_int64()
        st = self.L.dem_get_contact_wildcards(self.h, 0, C.byref(cnt), None)
        if st not in (OK, ERR_CAPACITY):
            self._c(st)
        wc = np.empty((cnt.value, 8))
        self._c(self.L.dem_get_contact_wildcards(self.h, cnt.value, C.byref(cnt), _p(wc)))
        return wc

    # ---- family tags
    def set_family(self, first, family):
        f = np.ascontiguousarray(family, np.uint8)
        self._c(self.L.dem_set_family(self.h, int(first), len(f), _p(f)))

    def set_family_motion(self, family, v=None, omega=None):
        self._c(self.L.dem_set_family_motion(self.h, int(family), _p(_f64(v)) if v is not None else None,
                                             _p(_f64(omega)) if omega is not None else None))

    def set_family_contacts(self, fa, fb, on):
        self._c(self.L.dem_set_family_contacts(self.h, int(fa), int(fb), 1 if on else 0))

    def set_active_box(self, lo, hi, family_inside, family_outside):
        self._c(self.L.dem_set_active_box(self.h, _p(_f64(lo)), _p(_f64(hi)), int(family_inside),
                                          int(family_outside)))

    def contact_rolling(self):
        """Per contact (dem_get_contacts order): its age and the rolling-resistance force on i."""
        cnt = C.c_int64()
        st = self.L.dem_get_contact_rolling(self.h, 0, C.byref(cnt), None, None)
        if st not in (OK, ERR_CAPACITY):
            self._c(st)
        n = cnt.value
        age = np.empty(n); trf = np.empty((n, 3))
        self._c(self.L.dem_get_contact_rolling(self.h, n, C.byref(cnt), _p(age), _p(trf)))
        return age, trf

    def stats(self):
        s = Stats()
        self._c(self.L.dem_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def diagnostics(self):
        d = Diagnostics()
        self._c(self.L.dem_get_diagnostics(self.h, C.byref(d)))
        return {"ke": d.kinetic, "pe": d.potential, "elastic": d.elastic, "momentum": np.array(d.momentum),
                "angmom": np.array(d.angular_momentum)}

    def save_state(self):
        used = C.c_size_t()
        self.L.dem_save_state(self.h, None, 0, C.byref(used))
        buf = (C.c_uint8 * used.value)()
        self._c(self.L.dem_save_state(self.h, C.cast(buf, C.c_void_p), used.value, C.byref(used)))
        return bytes(buf)

    def load_state(self, blob: bytes):
        buf = (C.c_uint8 * len(blob)).from_buffer_copy(blob)
        self._c(self.L.dem_load_state(self.h, C.cast(buf, C.c_void_p), len(blob)))

    # ---- convenience: a whole scene description
    def setup_scene(self, scene, margin=None):
        """Issue the set-up calls for a workloads.Scene (materials, walls, templates,
        clumps, parameters)."""
        nm = len(scene.E)
        cor = np.asarray(scene.cor).reshape(nm, nm)
        mu = np.asarray(scene.mu).reshape(nm, nm)
        crr = (np.zeros((nm, nm)) if getattr(scene, "crr", None) is None
               else np.asarray(scene.crr, np.float64).reshape(nm, nm))
        for a in range(nm):
            self.add_material(float(scene.E[a]), float(scene.nu[a]), float(cor[a, a]), float(mu[a, a]),
                              float(crr[a, a]))
        for a in range(nm):
            for b in range(a + 1, nm):
                self.set_material_pair(PROP_COR, a, b, float(cor[a, b]))
                self.set_material_pair(PROP_MU, a, b, float(mu[a, b]))
                self.set_material_pair(PROP_CRR, a, b, float(crr[a, b]))
        walls = list(scene.walls)
        k = 0
        while k < len(walls):
            wd = walls[k]
            t = int(wd["type"])
            om = np.asarray(wd.get("omega", (0.0, 0.0, 0.0)), np.float64)
            if t == WALL_TRIANGLE:
                # consecutive facets of one material, axis point and spin form one mesh
                run = [wd]
                while (k + len(run) < len(walls) and int(walls[k + len(run)]["type"]) == WALL_TRIANGLE
                       and int(walls[k + len(run)]["mat"]) == int(wd["mat"])
                       and np.array_equal(walls[k + len(run)]["p"], wd["p"])
                       and np.array_equal(walls[k + len(run)].get("omega", om), om)):
                    run.append(walls[k + len(run)])
                self.add_mesh(np.array([r["tri"] for r in run]), int(wd["mat"]), wd["p"], om)
                k += len(run)
                continue
            k += 1
            if t == WALL_PLANE:
                wid = self.add_plane(wd["p"], wd["n"], int(wd["mat"]))
            elif t == WALL_CYLINDER:
                wid = self.add_cylinder(wd["p"], wd["n"], float(wd["r0"]), int(wd["mat"]), 0.0)
            else:
                wid = self.add_cone_segment(wd["p"], wd["n"], float(wd["r0"]), float(wd["z0"]), float(wd["r1"]),
                                            float(wd["z1"]), int(wd["mat"]))
            if np.any(om != 0):
                self.set_wall_spin(wid, om)
        for t in scene.templates:
            self.add_clump_template(t.rel_xyz, t.radii, t.mats, float(t.mass), t.moi)
        if getattr(scene, "force_model", None) not in (None, "default"):
            self.set_force_model(scene.force_model, getattr(scene, "model_params", None))
        fm = getattr(scene, "family_motion", None) or {}
        for f, (vel, om) in fm.items():
            self.set_family_motion(f, vel, om)
        for fa, fb in getattr(scene, "family_masked", None) or []:
            self.set_family_contacts(fa, fb, False)
        ot = np.asarray(scene.owner_template)
        tid = int(ot[0]) if len(ot) and np.all(ot == ot[0]) else ot
        if len(ot):
            self.add_clumps(tid, scene.x, scene.q, scene.v, scene.wb, scene.owner_scale)
        self.set_timestep(float(scene.h))
        self.set_gravity(scene.g)
        if getattr(scene, "v_err", 0.0):
            self.set_error_velocity(float(scene.v_err))
        if getattr(scene, "sink", None) is not None:
            self.set_sink(scene.sink[0], scene.sink[1])
        if margin is not None:
            self.set_margin(margin)
        if getattr(scene, "family", None) is not None:
            self.set_family(0, scene.family)
        self.n_owner = len(ot)
        self.n_sphere = scene.n_sphere
        return self

    @classmethod
    def from_scene(cls, scene, precision="fp64", schedule="every_step", margin=None, margin_max=0.0, device=0,
                   gyroscopic=None, initialize=True, **hooks):
        g = scene.gyroscopic if gyroscopic is None else gyroscopic
        w = cls(scene.box_lo, scene.box_hi, precision=precision, schedule=schedule, device=device, gyroscopic=g,
                margin_max=margin_max, **hooks)
        w.setup_scene(scene, margin=margin)
        if initialize:
            w.initialize()
        return w


class Batch:
    """Independent scenes stepped together (dem_batch_*)."""

    def __init__(self, scenes, precision="voxel_fp32", schedule="every_step", margin=None, margin_max=0.0, device=0):
        self.L = load()
        n = len(scenes)
        descs = (WorldDesc * n)()
        for k, s in enumerate(scenes):
            d = descs[k]
            for a in range(3):
                d.box_lo[a] = float(s.box_lo[a]); d.box_hi[a] = float(s.box_hi[a])
            d.precision = PRECISION[precision]
            d.schedule = SCHEDULE[schedule]
            d.device = device
            d.gyroscopic = 1
            d.margin_max = margin_max
        h = C.c_void_p()
        _check(self.L.dem_batch_create(n, descs, C.byref(h)))
        self.h = h
        self.worlds = []
        for k, s in enumerate(scenes):
            wh = C.c_void_p()
            _check(self.L.dem_batch_world(self.h, k, C.byref(wh)))
            w = World(_handle=wh, _batch=self)
            w.setup_scene(s, margin=margin)
            self.worlds.append(w)

    def initialize(self):
        _check(self.L.dem_batch_initialize(self.h))

    def step(self, n=1):
        _check(self.L.dem_batch_step(self.h, int(n)))

    def close(self):
        if getattr(self, "h", None) is not None:
            self.L.dem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
