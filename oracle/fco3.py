"""ctypes wrapper of the three-dimensional FP64 oracle (oracle/fco3.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and
the CPU-baseline legs of the benchmark; never by the product path.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from .fco import build_oracle

INIT_BOX, INIT_SINE, INIT_GAUSS = 0, 1, 2
ERR_ARG, ERR_UNBALANCED, ERR_CFL = -1, -3, -5

_lib = None


class _Params(C.Structure):
    _fields_ = [
        ("m", C.c_int32), ("min_level", C.c_int32), ("max_level", C.c_int32), ("limiter", C.c_int32),
        ("transverse", C.c_int32), ("refluxing", C.c_int32), ("subcycle", C.c_int32), ("cfl", C.c_double),
        ("u", C.c_double),
        ("v", C.c_double), ("w", C.c_double), ("tag_threshold", C.c_double),
    ]


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build_oracle())
    vp, ip, dp, bp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int8)
    L.fco3_last_error.restype = C.c_char_p
    L.fco3_create.restype = vp
    L.fco3_create.argtypes = [C.POINTER(_Params)]
    L.fco3_destroy.argtypes = [vp]
    L.fco3_num_leaves.argtypes = [vp]
    L.fco3_forest_uniform.argtypes = [vp, C.c_int]
    L.fco3_set_leaves.argtypes = [vp, C.c_int, bp, ip, ip, ip]
    L.fco3_get_leaves.argtypes = [vp, bp, ip, ip, ip]
    L.fco3_balance.argtypes = [vp]
    L.fco3_is_balanced.argtypes = [vp]
    L.fco3_set_fields.argtypes = [vp, dp]
    L.fco3_get_fields.argtypes = [vp, dp]
    L.fco3_init.argtypes = [vp, C.c_int, dp, C.c_int]
    L.fco3_init_refine.argtypes = [vp, C.c_int, dp, C.c_int]
    L.fco3_fill_tiles.argtypes = [vp, dp]
    L.fco3_tag.argtypes = [vp, bp]
    L.fco3_regrid.argtypes = [vp, bp]
    L.fco3_advance.argtypes = [vp, C.c_int, C.c_double, dp, dp]
    L.fco3_next_dt.restype = C.c_double
    L.fco3_next_dt.argtypes = [vp]
    L.fco3_time.restype = C.c_double
    L.fco3_time.argtypes = [vp]
    L.fco3_sum.argtypes = [vp, dp]
    _lib = L
    return L


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class Oracle3Error(RuntimeError):
    def __init__(self, rc, where):
        super().__init__(f"oracle3 {where} failed rc={rc}: {lib().fco3_last_error().decode()}")
        self.rc = rc


@dataclass
class Oracle3Params:
    m: int = 8
    min_level: int = 1
    max_level: int = 1
    limiter: int = 1
    transverse: int = 2
    refluxing: int = 1
    subcycle: int = 0
    cfl: float = 0.9
    u: float = 1.0
    v: float = 0.0
    w: float = 0.0
    tag_threshold: float = 0.05


class Oracle3:
    def __init__(self, params: Oracle3Params):
        self.L = lib()
        self.params = params
        self.m = params.m
        self.h = self.L.fco3_create(C.byref(_Params(**params.__dict__)))
        if not self.h:
            raise RuntimeError("fco3_create: " + self.L.fco3_last_error().decode())

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.fco3_destroy(h)
            self.h = None

    def _chk(self, rc, where):
        if rc != 0:
            raise Oracle3Error(rc, where)

    @property
    def n(self):
        return self.L.fco3_num_leaves(self.h)

    def uniform(self, level):
        self._chk(self.L.fco3_forest_uniform(self.h, level), "uniform")

    def set_leaves(self, lv, x, y, z):
        lv = np.ascontiguousarray(lv, np.int8)
        x, y, z = (np.ascontiguousarray(a, np.int32) for a in (x, y, z))
        self._chk(self.L.fco3_set_leaves(self.h, len(lv), _p(lv, C.c_int8), _p(x, C.c_int32), _p(y, C.c_int32),
                                         _p(z, C.c_int32)), "set_leaves")

    def leaves(self):
        n = self.n
        lv = np.zeros(n, np.int8)
        x, y, z = (np.zeros(n, np.int32) for _ in range(3))
        self.L.fco3_get_leaves(self.h, _p(lv, C.c_int8), _p(x, C.c_int32), _p(y, C.c_int32), _p(z, C.c_int32))
        return lv, x, y, z

    def balance(self):
        self._chk(self.L.fco3_balance(self.h), "balance")

    def is_balanced(self):
        return bool(self.L.fco3_is_balanced(self.h))

    def fields(self):
        q = np.zeros((self.n, self.m, self.m, self.m))
        self.L.fco3_get_fields(self.h, _p(q, C.c_double))
        return q

    def set_fields(self, q):
        q = np.ascontiguousarray(q, np.float64)
        assert q.shape == (self.n, self.m, self.m, self.m)
        self.L.fco3_set_fields(self.h, _p(q, C.c_double))

    def init(self, kind, prm):
        a = np.ascontiguousarray(prm, np.float64)
        self._chk(self.L.fco3_init(self.h, kind, _p(a, C.c_double), len(a)), "init")

    def init_refine(self, kind, prm):
        a = np.ascontiguousarray(prm, np.float64)
        self._chk(self.L.fco3_init_refine(self.h, kind, _p(a, C.c_double), len(a)), "init_refine")

    def tiles(self):
        P = self.m + 4
        t = np.zeros((self.n, P, P, P))
        self._chk(self.L.fco3_fill_tiles(self.h, _p(t, C.c_double)), "fill_tiles")
        return t

    def tag(self):
        f = np.zeros(self.n, np.int8)
        self._chk(self.L.fco3_tag(self.h, _p(f, C.c_int8)), "tag")
        return f

    def regrid(self, flags):
        f = np.ascontiguousarray(flags, np.int8)
        assert len(f) == self.n
        self._chk(self.L.fco3_regrid(self.h, _p(f, C.c_int8)), "regrid")

    def advance(self, nsteps, dt=0.0):
        t, d = C.c_double(), C.c_double()
        self._chk(self.L.fco3_advance(self.h, nsteps, dt, C.byref(t), C.byref(d)), "advance")
        return t.value, d.value

    @property
    def next_dt(self):
        return self.L.fco3_next_dt(self.h)

    @property
    def time(self):
        return self.L.fco3_time(self.h)

    def sum(self):
        s = C.c_double()
        self.L.fco3_sum(self.h, C.byref(s))
        return s.value

    def grid(self, level=None):
        """fields on one uniform grid of the given level (finest by default):
        coarse cells repeated, finer cells averaged"""
        lv, x, y, z = self.leaves()
        L = int(lv.max()) if level is None else level
        m, q = self.m, self.fields()
        N = (1 << L) * m
        G = np.zeros((N, N, N))
        for k in range(len(lv)):
            r = L - int(lv[k])
            if r >= 0:
                b = q[k]
                for ax in range(3):
                    b = np.repeat(b, 1 << r, axis=ax)
                s = m << r
                G[z[k] * s:(z[k] + 1) * s, y[k] * s:(y[k] + 1) * s, x[k] * s:(x[k] + 1) * s] = b
            else:
                f = 1 << (-r)
                b = q[k].reshape(m // f, f, m // f, f, m // f, f).mean(axis=(1, 3, 5))
                s = m // f
                G[z[k] * s:(z[k] + 1) * s, y[k] * s:(y[k] + 1) * s, x[k] * s:(x[k] + 1) * s] = b
        return G
