"""Thin ctypes binding of the three-dimensional C ABI (include/fc3.h):
argument marshalling only; every step runs in libfc.so's kernels.

An octree of m^3 patches on the periodic unit cube, scalar advection with a
constant velocity (arXiv:1308.1472, the method of Sec. 2-4 for d = 3).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import fc

FC3_INIT_BOX, FC3_INIT_SINE, FC3_INIT_GAUSS = 0, 1, 2


class fc3_params(C.Structure):
    _fields_ = [
        ("m", C.c_int32), ("min_level", C.c_int32), ("max_level", C.c_int32), ("precision", C.c_int32),
        ("limiter", C.c_int32), ("transverse", C.c_int32), ("refluxing", C.c_int32), ("subcycle", C.c_int32),
        ("device", C.c_int32),
        ("cfl", C.c_double), ("u", C.c_double), ("v", C.c_double), ("w", C.c_double),
        ("tag_threshold", C.c_double), ("stream", C.c_void_p),
    ]


_bound = False
_VP, _I8, _I32, _D = C.c_void_p, C.POINTER(C.c_int8), C.POINTER(C.c_int32), C.POINTER(C.c_double)
SIGNATURES = {
    "fc3_create": (C.c_int, [C.POINTER(fc3_params), C.POINTER(C.c_void_p)]),
    "fc3_destroy": (None, [_VP]),
    "fc3_forest_uniform": (C.c_int, [_VP, C.c_int]),
    "fc3_forest_set_leaves": (C.c_int, [_VP, C.c_int64, _I8, _I32, _I32, _I32]),
    "fc3_forest_num_leaves": (C.c_int, [_VP, C.POINTER(C.c_int64)]),
    "fc3_forest_get_leaves": (C.c_int, [_VP, _I8, _I32, _I32, _I32, C.c_int64]),
    "fc3_write_fields": (C.c_int, [_VP, _VP, C.c_int64]),
    "fc3_read_fields": (C.c_int, [_VP, _VP, C.c_int64]),
    "fc3_set_initial": (C.c_int, [_VP, C.c_int, _D, C.c_int]),
    "fc3_init_refine": (C.c_int, [_VP, C.c_int, _D, C.c_int]),
    "fc3_tag": (C.c_int, [_VP, _I8]),
    "fc3_regrid": (C.c_int, [_VP, _I8]),
    "fc3_advance": (C.c_int, [_VP, C.c_int, C.c_double, _D, _D]),
    "fc3_conservation_sum": (C.c_int, [_VP, _D]),
    "fc3_stats": (C.c_int, [_VP, _D, _D, _D]),
    "fc3_sync": (C.c_int, [_VP]),
}


def lib():
    global _bound
    L = fc.lib()
    if not _bound:
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class Context3:
    """One three-dimensional solver context on one GPU."""

    def __init__(self, m=8, min_level=1, max_level=1, precision=fc.FC_FP64, limiter=1, transverse=2, refluxing=1,
                 subcycle=0, device=-1, cfl=0.9, u=1.0, v=0.0, w=0.0, tag_threshold=0.05, stream=None):
        self.L = lib()
        self.m = m
        self.dtype = np.float64 if precision == fc.FC_FP64 else np.float32
        p = fc3_params(m=m, min_level=min_level, max_level=max_level, precision=precision, limiter=limiter,
                       transverse=transverse, refluxing=refluxing, subcycle=subcycle, device=device, cfl=cfl, u=u,
                       v=v, w=w, tag_threshold=tag_threshold, stream=stream)
        h = C.c_void_p()
        fc.check(self.L.fc3_create(C.byref(p), C.byref(h)), "fc3_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.fc3_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def n(self):
        n = C.c_int64()
        fc.check(self.L.fc3_forest_num_leaves(self.h, C.byref(n)), "fc3_forest_num_leaves")
        return n.value

    def forest_uniform(self, level):
        fc.check(self.L.fc3_forest_uniform(self.h, level), "fc3_forest_uniform")

    def forest_set_leaves(self, level, x, y, z):
        lv = np.ascontiguousarray(level, np.int8)
        x, y, z = (np.ascontiguousarray(a, np.int32) for a in (x, y, z))
        fc.check(self.L.fc3_forest_set_leaves(self.h, len(lv), _p(lv, C.c_int8), _p(x, C.c_int32), _p(y, C.c_int32),
                                              _p(z, C.c_int32)), "fc3_forest_set_leaves")

    def forest_get_leaves(self):
        n = self.n
        lv = np.zeros(n, np.int8)
        x, y, z = (np.zeros(n, np.int32) for _ in range(3))
        fc.check(self.L.fc3_forest_get_leaves(self.h, _p(lv, C.c_int8), _p(x, C.c_int32), _p(y, C.c_int32),
                                              _p(z, C.c_int32), n), "fc3_forest_get_leaves")
        return lv, x, y, z

    def write_fields(self, q):
        q = np.ascontiguousarray(q, self.dtype)
        fc.check(self.L.fc3_write_fields(self.h, q.ctypes.data, q.size), "fc3_write_fields")

    def read_fields(self):
        q = np.empty((self.n, self.m, self.m, self.m), self.dtype)
        fc.check(self.L.fc3_read_fields(self.h, q.ctypes.data, q.size), "fc3_read_fields")
        return q

    def set_initial(self, kind, prm):
        a = np.ascontiguousarray(prm, np.float64)
        fc.check(self.L.fc3_set_initial(self.h, kind, _p(a, C.c_double), len(a)), "fc3_set_initial")

    def init_refine(self, kind, prm):
        a = np.ascontiguousarray(prm, np.float64)
        fc.check(self.L.fc3_init_refine(self.h, kind, _p(a, C.c_double), len(a)), "fc3_init_refine")

    def tag(self):
        f = np.zeros(self.n, np.int8)
        fc.check(self.L.fc3_tag(self.h, _p(f, C.c_int8)), "fc3_tag")
        return f

    def regrid(self, flags):
        f = np.ascontiguousarray(flags, np.int8)
        if len(f) != self.n:
            raise ValueError("one flag per leaf")
        fc.check(self.L.fc3_regrid(self.h, _p(f, C.c_int8)), "fc3_regrid")

    def advance(self, nsteps, dt=0.0):
        t, d = C.c_double(), C.c_double()
        fc.check(self.L.fc3_advance(self.h, nsteps, dt, C.byref(t), C.byref(d)), "fc3_advance")
        return t.value, d.value

    def conservation_sum(self):
        s = C.c_double()
        fc.check(self.L.fc3_conservation_sum(self.h, C.byref(s)), "fc3_conservation_sum")
        return s.value

    def stats(self):
        t, nd, cu = C.c_double(), C.c_double(), C.c_double()
        fc.check(self.L.fc3_stats(self.h, C.byref(t), C.byref(nd), C.byref(cu)), "fc3_stats")
        return {"time": t.value, "next_dt": nd.value, "cell_updates": cu.value}

    def sync(self):
        fc.check(self.L.fc3_sync(self.h), "fc3_sync")
