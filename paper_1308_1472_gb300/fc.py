"""Thin ctypes binding of ``include/fc.h`` (libfc.so), with the same names.

Only argument marshalling happens here; every step of the method runs in the
library's CUDA kernels.  Importing this module never falls back to anything:
if the library cannot be built or loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

FC_OK = 0
FC_ERR_INVALID_ARG, FC_ERR_CAPACITY, FC_ERR_UNBALANCED, FC_ERR_DRY_STATE = -1, -2, -3, -4
FC_ERR_CFL_VIOLATION, FC_ERR_NONFINITE, FC_ERR_TIMEOUT, FC_ERR_CUDA, FC_ERR_UNIMPLEMENTED = -5, -6, -7, -8, -9
FC_CONN_SQUARE, FC_CONN_PERIODIC, FC_CONN_SPHERE, FC_CONN_PILLOW, FC_CONN_TABLE = 0, 1, 2, 3, 4
FC_MAX_TREES = 16
FC_EQ_SWE, FC_EQ_ADV = 0, 1
FC_FP64, FC_FP32 = 0, 1
FC_TAG_GRAD, FC_TAG_MAXMIN = 0, 1
FC_TAGGER_PLAIN, FC_TAGGER_LEARNED = 0, 1
FC_INIT_DAMBREAK, FC_INIT_HUMPS, FC_INIT_ADV_BOX, FC_INIT_ADV_SINE, FC_INIT_HILL, FC_INIT_HALF = 0, 1, 2, 3, 4, 5
FC_NB_NONE, FC_NB_SAME, FC_NB_COARSER, FC_NB_FINER = 0, 1, 2, 3
FC_UPDATE_VARIANTS = 7
FC_MAX_STEP_STREAMS = 4
FC_VEL_CONSTANT, FC_VEL_SWIRL = 0, 1
CNN_NPARAM = 3058


class fc_params(C.Structure):
    _fields_ = [
        ("conn", C.c_int32), ("m", C.c_int32), ("min_level", C.c_int32), ("max_level", C.c_int32),
        ("equation", C.c_int32), ("precision", C.c_int32), ("subcycle", C.c_int32),
        ("tag_crit", C.c_int32), ("refluxing", C.c_int32), ("device", C.c_int32),
        ("g", C.c_double), ("cfl", C.c_double), ("tag_threshold", C.c_double),
        ("adv_u", C.c_double), ("adv_v", C.c_double), ("stream", C.c_void_p),
        ("omega", C.c_double), ("omega_axis_tilt", C.c_double),
        ("transverse", C.c_int32), ("entropy_fix", C.c_int32), ("velocity", C.c_int32),
    ]


class fc_stats_t(C.Structure):
    _fields_ = [
        ("num_leaves", C.c_int64), ("leaves_per_level", C.c_int64 * 16), ("cell_updates", C.c_int64),
        ("steps", C.c_int64), ("retries", C.c_int64), ("regrids", C.c_int64), ("time", C.c_double),
        ("last_dt", C.c_double), ("last_courant", C.c_double), ("next_dt", C.c_double),
    ]


# name -> (restype, argtypes); the exported set equals the declarations of fc.h
_P = C.c_void_p
_i32p = C.POINTER(C.c_int32)
_i8p = C.POINTER(C.c_int8)
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
SIGNATURES = {
    "fc_create": (C.c_int, [C.POINTER(fc_params), C.POINTER(_P)]),
    "fc_destroy": (None, [_P]),
    "fc_last_error": (C.c_char_p, []),
    "fc_forest_uniform": (C.c_int, [_P, C.c_int]),
    "fc_set_connectivity": (C.c_int, [_P, C.c_int, _P]),
    "fc_forest_set_leaves": (C.c_int, [_P, C.c_int64, _i32p, _i32p, _i32p, _i32p]),
    "fc_forest_num_leaves": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "fc_forest_get_leaves": (C.c_int, [_P, _i32p, _i32p, _i32p, _i32p, C.c_int64]),
    "fc_forest_get_neighbors": (C.c_int, [_P, _i32p, C.c_int64]),
    "fc_forest_balance": (C.c_int, [_P]),
    "fc_set_initial": (C.c_int, [_P, C.c_int, _dp, C.c_int]),
    "fc_init_refine": (C.c_int, [_P, C.c_int, _dp, C.c_int]),
    "fc_num_fields": (C.c_int, [_P]),
    "fc_read_fields": (C.c_int, [_P, C.c_int, _P, C.c_int64, C.c_int]),
    "fc_write_fields": (C.c_int, [_P, _P, C.c_int64, C.c_int]),
    "fc_read_fields_async": (C.c_int, [_P, C.c_int, _P, C.c_int64, C.c_int]),
    "fc_write_fields_async": (C.c_int, [_P, _P, C.c_int64, C.c_int]),
    "fc_conservation_sums": (C.c_int, [_P, _dp]),
    "fc_conservation_sums_noalloc": (C.c_int, [_P, _P, C.c_int64, C.c_int, C.c_int, C.c_int, _P, _P]),
    "fc_tag": (C.c_int, [_P, _i8p, C.c_int]),
    "fc_regrid": (C.c_int, [_P, _i8p]),
    "fc_advance": (C.c_int, [_P, C.c_double, C.c_int, _dp, _dp]),
    "fc_advance_async": (C.c_int, [_P, C.c_double, C.c_int]),
    "fc_sync": (C.c_int, [_P]),
    "fc_stats": (C.c_int, [_P, C.POINTER(fc_stats_t)]),
    "fc_autotune": (C.c_int, [_P, C.POINTER(C.c_int), _dp]),
    "fc_set_variant": (C.c_int, [_P, C.c_int]),
    "fc_set_step_streams": (C.c_int, [_P, C.c_int]),
    "fc_step_schedule": (C.c_int, [_P, _i32p, _i32p, _i32p]),
    "fc_profile_steps": (C.c_int, [_P, C.c_double, C.c_int, _dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "fc_save": (C.c_int, [_P, C.c_char_p]),
    "fc_load": (C.c_int, [_P, C.c_char_p]),
    "fc_cnn_forward": (C.c_int, [C.c_int, C.c_int, _P, _P, _P, C.c_int, _P]),
    "fc_cnn_loss_grad": (C.c_int, [C.c_int, C.c_int, _P, _P, _P, _P, _fp, C.c_int, _P]),
    "fc_cnn_adam": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_float, _P]),
    "fc_cnn_set_wait_limit": (C.c_int, [C.c_longlong]),
    "fc_cnn_input_stats": (C.c_int, [C.c_int, C.c_int, _P, _dp, _P]),
    "fc_cnn_normalize": (C.c_int, [C.c_int, C.c_int, _P, _dp, _P]),
    "fc_export_tiles": (C.c_int, [_P, _P, C.c_int64, _dp, C.c_int]),
    "fc_set_tagger": (C.c_int, [_P, _fp, _dp, C.c_int]),
}

_lib = None


def lib():
    """Load (building first if needed) libfc.so; raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not _build.up_to_date():
        _build.build()
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class FCError(RuntimeError):
    def __init__(self, rc: int, where: str):
        msg = lib().fc_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({rc}): {msg}")
        self.rc = rc


def check(rc: int, where: str):
    if rc != FC_OK:
        raise FCError(rc, where)


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Context:
    """One library context (forest + device state).  Methods map one to one on
    the C entry points."""

    def __init__(self, conn=FC_CONN_SQUARE, m=16, min_level=2, max_level=2, equation=FC_EQ_SWE,
                 precision=FC_FP64, subcycle=0, tag_crit=FC_TAG_GRAD, refluxing=1, device=-1, g=1.0,
                 cfl=0.9, tag_threshold=0.05, adv_u=1.0, adv_v=0.0, stream=None, omega=0.0, omega_axis_tilt=0.0,
                 transverse=1, entropy_fix=0, velocity=0):
        self.L = lib()
        p = fc_params(conn, m, min_level, max_level, equation, precision, subcycle, tag_crit, refluxing,
                      device, g, cfl, tag_threshold, adv_u, adv_v, stream, omega, omega_axis_tilt, transverse,
                      entropy_fix, velocity)
        h = C.c_void_p()
        check(self.L.fc_create(C.byref(p), C.byref(h)), "fc_create")
        self.h = h
        self.params = p
        self.m = m
        self.F = self.L.fc_num_fields(h)
        self.dtype = np.float64 if precision == FC_FP64 else np.float32

    def close(self):
        if getattr(self, "h", None):
            self.L.fc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # forest
    def forest_uniform(self, level):
        check(self.L.fc_forest_uniform(self.h, level), "fc_forest_uniform")

    def set_connectivity(self, table):
        """table [ntrees][4][3] of a FC_CONN_TABLE context (see fc_set_connectivity)"""
        t = np.ascontiguousarray(table, dtype=np.int32)
        check(self.L.fc_set_connectivity(self.h, t.shape[0], t.ctypes.data), "fc_set_connectivity")

    def forest_set_leaves(self, tree, level, x, y):
        a = [_arr(v, np.int32) for v in (tree, level, x, y)]
        ptrs = [v.ctypes.data_as(_i32p) for v in a]
        check(self.L.fc_forest_set_leaves(self.h, len(a[0]), *ptrs), "fc_forest_set_leaves")

    @property
    def n(self) -> int:
        v = C.c_int64()
        check(self.L.fc_forest_num_leaves(self.h, C.byref(v)), "fc_forest_num_leaves")
        return v.value

    def forest_get_leaves(self):
        n = self.n
        out = [np.zeros(n, np.int32) for _ in range(4)]
        check(self.L.fc_forest_get_leaves(self.h, *[o.ctypes.data_as(_i32p) for o in out], n),
              "fc_forest_get_leaves")
        return tuple(out)

    def forest_get_neighbors(self):
        n = self.n
        t = np.zeros((n, 8, 4), np.int32)
        check(self.L.fc_forest_get_neighbors(self.h, t.ctypes.data_as(_i32p), t.size), "fc_forest_get_neighbors")
        return t

    def forest_balance(self):
        check(self.L.fc_forest_balance(self.h), "fc_forest_balance")

    # fields
    def set_initial(self, kind, params):
        a = _arr(params, np.float64)
        check(self.L.fc_set_initial(self.h, kind, a.ctypes.data_as(_dp), len(a)), "fc_set_initial")

    def init_refine(self, kind, params):
        a = _arr(params, np.float64)
        check(self.L.fc_init_refine(self.h, kind, a.ctypes.data_as(_dp), len(a)), "fc_init_refine")

    def read_fields(self, field=-1) -> np.ndarray:
        n, m = self.n, self.m
        shape = (n, self.F, m, m) if field < 0 else (n, m, m)
        out = np.zeros(shape, self.dtype)
        check(self.L.fc_read_fields(self.h, field, out.ctypes.data, out.nbytes, 0), "fc_read_fields")
        return out

    def read_fields_device(self, dst_ptr: int, nbytes: int, field=-1):
        check(self.L.fc_read_fields(self.h, field, dst_ptr, nbytes, 1), "fc_read_fields")

    def write_fields(self, q):
        a = _arr(q, self.dtype)
        check(self.L.fc_write_fields(self.h, a.ctypes.data, a.nbytes, 0), "fc_write_fields")

    def read_fields_async(self, dst_ptr: int, nbytes: int, field=-1, dst_is_device=False):
        """enqueue a read of the state into a page-locked host (or device) buffer"""
        check(self.L.fc_read_fields_async(self.h, field, dst_ptr, nbytes, int(dst_is_device)), "fc_read_fields_async")

    def write_fields_async(self, src_ptr: int, nbytes: int, src_is_device=False):
        """enqueue a write of the state from a page-locked host (or device) buffer"""
        check(self.L.fc_write_fields_async(self.h, src_ptr, nbytes, int(src_is_device)), "fc_write_fields_async")

    def write_fields_device(self, src_ptr: int, nbytes: int):
        check(self.L.fc_write_fields(self.h, src_ptr, nbytes, 1), "fc_write_fields")

    def conservation_sums(self) -> np.ndarray:
        out = np.zeros(self.F)
        check(self.L.fc_conservation_sums(self.h, out.ctypes.data_as(_dp)), "fc_conservation_sums")
        return out

    # tagging / regrid
    def tag(self, tagger=FC_TAGGER_PLAIN) -> np.ndarray:
        f = np.zeros(self.n, np.int8)
        check(self.L.fc_tag(self.h, f.ctypes.data_as(_i8p), tagger), "fc_tag")
        return f

    def regrid(self, flags):
        f = _arr(flags, np.int8)
        check(self.L.fc_regrid(self.h, f.ctypes.data_as(_i8p)), "fc_regrid")

    # stepping
    def advance(self, nsteps, dt=0.0):
        t = C.c_double()
        d = C.c_double()
        check(self.L.fc_advance(self.h, dt, nsteps, C.byref(t), C.byref(d)), "fc_advance")
        return t.value, d.value

    def advance_async(self, nsteps, dt=0.0):
        check(self.L.fc_advance_async(self.h, dt, nsteps), "fc_advance_async")

    def sync(self):
        check(self.L.fc_sync(self.h), "fc_sync")

    def stats(self) -> dict:
        s = fc_stats_t()
        check(self.L.fc_stats(self.h, C.byref(s)), "fc_stats")
        d = {k: getattr(s, k) for k, _ in fc_stats_t._fields_}
        d["leaves_per_level"] = list(s.leaves_per_level)
        return d

    def autotune(self):
        v = C.c_int()
        ms = np.zeros(FC_UPDATE_VARIANTS)
        check(self.L.fc_autotune(self.h, C.byref(v), ms.ctypes.data_as(_dp)), "fc_autotune")
        return v.value, ms

    def set_variant(self, variant):
        check(self.L.fc_set_variant(self.h, variant), "fc_set_variant")

    def set_step_streams(self, nstreams):
        check(self.L.fc_set_step_streams(self.h, nstreams), "fc_set_step_streams")

    def step_schedule(self):
        """(launches per step, streams used, launches on the longest dependence chain)"""
        v = [C.c_int32() for _ in range(3)]
        check(self.L.fc_step_schedule(self.h, *[C.byref(x) for x in v]), "fc_step_schedule")
        return tuple(x.value for x in v)

    def profile_steps(self, nsteps, dt=0.0):
        ms = np.zeros(4)
        cnt = np.zeros(4, np.int64)
        cells = np.zeros(4, np.int64)
        check(self.L.fc_profile_steps(self.h, dt, nsteps, ms.ctypes.data_as(_dp),
                                      cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                      cells.ctypes.data_as(C.POINTER(C.c_int64))), "fc_profile_steps")
        return ms, cnt, cells

    def export_tiles_device(self, dst_ptr: int, cap_floats: int, xform):
        x = _arr(xform, np.float64)
        check(self.L.fc_export_tiles(self.h, dst_ptr, cap_floats, x.ctypes.data_as(_dp), 1), "fc_export_tiles")

    def export_tiles(self, xform) -> np.ndarray:
        n, S = self.n, self.m + 4
        out = np.zeros((n, 3, S, S), np.float32)
        x = _arr(xform, np.float64)
        check(self.L.fc_export_tiles(self.h, out.ctypes.data, out.size, x.ctypes.data_as(_dp), 0), "fc_export_tiles")
        return out

    def set_tagger(self, w, xform, bf16=1):
        wa = _arr(w, np.float32)
        x = _arr(xform, np.float64)
        assert wa.size == CNN_NPARAM
        check(self.L.fc_set_tagger(self.h, wa.ctypes.data_as(_fp), x.ctypes.data_as(_dp), bf16), "fc_set_tagger")

    def save(self, path):
        check(self.L.fc_save(self.h, os.fsencode(path)), "fc_save")

    def load(self, path):
        check(self.L.fc_load(self.h, os.fsencode(path)), "fc_load")
