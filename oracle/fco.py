"""ctypes binding of the C oracle (TEST INFRASTRUCTURE, see package docstring).

``build_oracle()`` compiles ``oracle/*.c`` with gcc into ``oracle/libfco.so``
(contraction of a*b+c into fused multiply-adds is switched off so that the
arithmetic is the one written in the source on every host).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["fco_forest.c", "fco_riemann.c", "fco_sim.c", "fco_sphere.c", "fco_pillow.c", "fco_cnn.c", "fco3.c"]
_LIB_PATH = os.path.join(_HERE, "libfco.so")
_lib = None
# fco_substep_hook: (ctx, level, q, qold, n) -> 0 to go on
_HOOK = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int)

CONN_SQUARE, CONN_PERIODIC, CONN_SPHERE, CONN_PILLOW, CONN_TABLE = 0, 1, 2, 3, 4
EQ_SWE, EQ_ADV = 0, 1
TAG_GRAD, TAG_MAXMIN = 0, 1
INIT_DAMBREAK, INIT_HUMPS, INIT_ADV_BOX, INIT_ADV_SINE, INIT_HILL, INIT_HALF = 0, 1, 2, 3, 4, 5
VEL_CONSTANT, VEL_SWIRL = 0, 1
NB_NONE, NB_SAME, NB_COARSER, NB_FINER = 0, 1, 2, 3
CNN_NPARAM = 3058


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than a source."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdrs = [os.path.join(_HERE, h) for h in ("fco.h", "fco_internal.h", "fco3.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(p) <= t for p in srcs + hdrs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *srcs, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_oracle_variant(outdir: str, edits) -> str:
    """Compile a copy of the oracle with textual edits applied, for tests that
    plant a mistake in the oracle and check that a pin catches it.  `edits` is
    a list of (file name, old text, new text); each old text must occur exactly
    once in its file.  Returns the path of the shared library in `outdir`."""
    import shutil
    os.makedirs(outdir, exist_ok=True)
    for name in _SOURCES + ["fco.h", "fco_internal.h", "fco3.h"]:
        shutil.copy(os.path.join(_HERE, name), os.path.join(outdir, name))
    for name, old, new in edits:
        path = os.path.join(outdir, name)
        text = open(path).read()
        if text.count(old) != 1:
            raise ValueError(f"edit of {name}: the text to replace occurs {text.count(old)} times")
        open(path, "w").write(text.replace(old, new))
    lib = os.path.join(outdir, "libfco_variant.so")
    cmd = ["gcc", "-std=gnu99", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           *[os.path.join(outdir, s) for s in _SOURCES], "-o", lib, "-lm"]
    subprocess.run(cmd, check=True)
    return lib


class _Params(C.Structure):
    _fields_ = [
        ("conn", C.c_int32), ("m", C.c_int32), ("min_level", C.c_int32), ("max_level", C.c_int32),
        ("equation", C.c_int32), ("subcycle", C.c_int32), ("tag_crit", C.c_int32),
        ("refluxing", C.c_int32), ("g", C.c_double), ("cfl", C.c_double),
        ("tag_threshold", C.c_double), ("adv_u", C.c_double), ("adv_v", C.c_double),
        ("omega_axis_tilt", C.c_double), ("omega", C.c_double),
        ("transverse", C.c_int32), ("entropy_fix", C.c_int32), ("velocity", C.c_int32),
    ]


def oracle_lib():
    global _lib
    if _lib is not None:
        return _lib
    _lib = load_oracle_lib(build_oracle())
    return _lib


def load_oracle_lib(path: str):
    """Load an oracle shared library from `path` and declare its signatures.
    ``oracle_lib()`` uses it for the in-tree build; a test may load a copy
    built from modified sources (a planted mistake) beside it."""
    lib = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    bp = C.POINTER(C.c_int8)
    sig = {
        "fco_create": (P, [C.POINTER(_Params)]),
        "fco_destroy": (None, [P]),
        "fco_last_error": (C.c_char_p, []),
        "fco_forest_uniform": (C.c_int, [P, C.c_int]),
        "fco_set_connectivity": (C.c_int, [P, C.c_int, ip]),
        "fco_forest_set_leaves": (C.c_int, [P, C.c_int, ip, ip, ip, ip]),
        "fco_num_leaves": (C.c_int, [P]),
        "fco_get_leaves": (C.c_int, [P, ip, ip, ip, ip]),
        "fco_get_neighbors": (C.c_int, [P, ip]),
        "fco_is_balanced": (C.c_int, [P]),
        "fco_balance": (C.c_int, [P]),
        "fco_adapt_topology": (C.c_int, [P, bp]),
        "fco_num_fields": (C.c_int, [P]),
        "fco_init_fields": (C.c_int, [P, C.c_int, dp, C.c_int]),
        "fco_init_refine": (C.c_int, [P, C.c_int, dp, C.c_int]),
        "fco_get_fields": (C.c_int, [P, dp]),
        "fco_set_fields": (C.c_int, [P, dp]),
        "fco_conservation_sums": (C.c_int, [P, dp]),
        "fco_fill_ghosts": (C.c_int, [P, dp]),
        "fco_tag": (C.c_int, [P, bp]),
        "fco_regrid": (C.c_int, [P, bp]),
        "fco_advance": (C.c_int, [P, C.c_double, C.c_int, dp, dp]),
        "fco_set_substep_hook": (None, [P, _HOOK, P]),
        "fco_table_map_point": (C.c_int, [ip, C.c_int, C.c_longlong, C.c_longlong, C.POINTER(C.c_longlong),
                                          C.POINTER(C.c_longlong)]),
        "fco_map_point": (C.c_int, [C.c_int, C.c_int, C.c_longlong, C.c_longlong, C.POINTER(C.c_longlong),
                                    C.POINTER(C.c_longlong)]),
        "fco_time": (C.c_double, [P]),
        "fco_next_dt": (C.c_double, [P]),
        "fco_last_courant": (C.c_double, [P]),
        "fco_cell_updates": (C.c_int64, [P]),
        "fco_roe_x": (C.c_int, [dp, dp, C.c_double, dp, dp, dp, dp]),
        "fco_roe_transverse_x": (C.c_int, [dp, dp, C.c_double, dp, dp, dp]),
        "fco_mc": (C.c_double, [C.c_double]),
        "fco_patch_step": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double, dp, dp, dp]),
        "fco_swe1d": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, dp, dp]),
        "fco_swe1d_efix": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, dp, dp]),
        "fco_roe_x_efix": (C.c_int, [dp, dp, C.c_double, dp, dp]),
        "fco_swe_exact": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int, dp, dp, dp]),
        "fco_tag_patch_f32": (C.c_int, [C.c_int, C.c_int, C.c_float, C.POINTER(C.c_float)]),
        "fco_cnn_forward": (C.c_int, [C.c_int, C.c_int, dp, dp, dp]),
        "fco_cnn_loss_grad": (C.c_double, [C.c_int, C.c_int, dp, dp, dp, dp]),
        "fco_sphere_fold": (C.c_int, [C.c_int, C.c_longlong, C.c_longlong, C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_longlong)]),
        "fco_sphere_point": (C.c_int, [C.c_int, C.c_longlong, C.c_longlong, dp]),
        "fco_sphere_cell_area": (C.c_double, [C.c_int, C.c_longlong, C.c_longlong, C.c_longlong,
                                              C.c_longlong]),
        "fco_pillow_fold": (C.c_int, [C.c_int, C.c_longlong, C.c_longlong, C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_longlong)]),
        "fco_pillow_point": (C.c_int, [C.c_int, C.c_longlong, C.c_longlong, dp]),
        "fco_pillow_cell_area": (C.c_double, [C.c_int, C.c_longlong, C.c_longlong, C.c_longlong,
                                              C.c_longlong]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _bp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int8))


class OracleError(RuntimeError):
    def __init__(self, rc: int, where: str):
        msg = oracle_lib().fco_last_error().decode()
        super().__init__(f"oracle {where} failed rc={rc}: {msg}")
        self.rc = rc


@dataclass
class OracleParams:
    conn: int = CONN_SQUARE
    m: int = 8
    min_level: int = 2
    max_level: int = 2
    equation: int = EQ_SWE
    subcycle: int = 0
    tag_crit: int = TAG_GRAD
    refluxing: int = 1
    g: float = 1.0
    cfl: float = 0.9
    tag_threshold: float = 0.05
    adv_u: float = 1.0
    adv_v: float = 0.0
    omega_axis_tilt: float = 0.0
    omega: float = 0.0
    transverse: int = 1
    entropy_fix: int = 0
    velocity: int = 0


class Oracle:
    """One oracle simulation: forest + FP64 fields."""

    def __init__(self, params: OracleParams, lib=None):
        self.lib = lib if lib is not None else oracle_lib()
        self.params = params
        p = _Params(**params.__dict__)
        self.h = self.lib.fco_create(C.byref(p))
        if not self.h:
            raise RuntimeError("fco_create: " + self.lib.fco_last_error().decode())
        self.m = params.m
        self.F = self.lib.fco_num_fields(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.fco_destroy(h)
            self.h = None

    def _chk(self, rc, where):
        if rc:
            raise OracleError(rc, where)

    # forest ---------------------------------------------------------------
    def uniform(self, level: int):
        self._chk(self.lib.fco_forest_uniform(self.h, level), "uniform")

    def set_connectivity(self, table):
        """table [ntrees][4][3] of a CONN_TABLE oracle (see fco_set_connectivity)"""
        t = np.ascontiguousarray(table, dtype=np.int32)
        self._chk(self.lib.fco_set_connectivity(self.h, t.shape[0], _ip(t)), "set_connectivity")

    def set_leaves(self, tree, level, x, y):
        arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (tree, level, x, y)]
        self._chk(self.lib.fco_forest_set_leaves(self.h, len(arrs[0]), *[_ip(a) for a in arrs]), "set_leaves")

    @property
    def n(self) -> int:
        return self.lib.fco_num_leaves(self.h)

    def leaves(self):
        n = self.n
        out = [np.zeros(n, np.int32) for _ in range(4)]
        self.lib.fco_get_leaves(self.h, *[_ip(a) for a in out])
        return tuple(out)

    def neighbors(self) -> np.ndarray:
        t = np.zeros((self.n, 8, 4), np.int32)
        self._chk(self.lib.fco_get_neighbors(self.h, _ip(t)), "neighbors")
        return t

    def is_balanced(self) -> bool:
        return bool(self.lib.fco_is_balanced(self.h))

    def balance(self):
        self._chk(self.lib.fco_balance(self.h), "balance")

    def adapt_topology(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.int8)
        self._chk(self.lib.fco_adapt_topology(self.h, _bp(f)), "adapt_topology")

    # fields ---------------------------------------------------------------
    def init_fields(self, kind: int, p):
        a = np.ascontiguousarray(p, dtype=np.float64)
        self._chk(self.lib.fco_init_fields(self.h, kind, _dp(a), len(a)), "init_fields")

    def init_refine(self, kind: int, p):
        a = np.ascontiguousarray(p, dtype=np.float64)
        self._chk(self.lib.fco_init_refine(self.h, kind, _dp(a), len(a)), "init_refine")

    def fields(self) -> np.ndarray:
        out = np.zeros((self.n, self.F, self.m, self.m))
        self.lib.fco_get_fields(self.h, _dp(out))
        return out

    def set_fields(self, q):
        a = np.ascontiguousarray(q, dtype=np.float64)
        assert a.shape == (self.n, self.F, self.m, self.m)
        self.lib.fco_set_fields(self.h, _dp(a))

    def sums(self) -> np.ndarray:
        out = np.zeros(self.F)
        self.lib.fco_conservation_sums(self.h, _dp(out))
        return out

    def fill_ghosts(self) -> np.ndarray:
        out = np.zeros((self.n, self.F, self.m + 4, self.m + 4))
        self._chk(self.lib.fco_fill_ghosts(self.h, _dp(out)), "fill_ghosts")
        return out

    # tagging / regrid -----------------------------------------------------
    def tag(self) -> np.ndarray:
        f = np.zeros(self.n, np.int8)
        self._chk(self.lib.fco_tag(self.h, _bp(f)), "tag")
        return f

    def regrid(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.int8)
        assert f.shape == (self.n,)
        self._chk(self.lib.fco_regrid(self.h, _bp(f)), "regrid")

    # stepping -------------------------------------------------------------
    def set_substep_hook(self, fn):
        """fn(level, q, qold) before the ghost fill of every (sub)step: level
        -1 with a global dt, q and qold writable [n][F][m][m] views of the
        current state and of each level's substep start state (the same
        array with a global dt); None removes the hook"""
        if fn is None:
            self._hook = None
            self.lib.fco_set_substep_hook(self.h, _HOOK(), None)
            return
        shape = (self.F, self.m, self.m)

        def call(_ctx, level, q, qold, n):
            try:
                fn(level, np.ctypeslib.as_array(q, (n,) + shape), np.ctypeslib.as_array(qold, (n,) + shape))
                return 0
            except Exception:            # noqa: BLE001 -- reported to the caller as a failed step
                return 1

        self._hook = _HOOK(call)         # kept alive as long as the oracle
        self.lib.fco_set_substep_hook(self.h, self._hook, None)

    def advance(self, nsteps: int, dt: float = 0.0):
        t = C.c_double(0.0)
        d = C.c_double(0.0)
        rc = self.lib.fco_advance(self.h, dt, nsteps, C.byref(t), C.byref(d))
        self._chk(rc, "advance")
        return t.value, d.value

    @property
    def time(self) -> float:
        return self.lib.fco_time(self.h)

    @property
    def next_dt(self) -> float:
        return self.lib.fco_next_dt(self.h)

    @property
    def last_courant(self) -> float:
        return self.lib.fco_last_courant(self.h)

    @property
    def cell_updates(self) -> int:
        return self.lib.fco_cell_updates(self.h)


# single-edge / single-patch helpers used by pins -----------------------------
def roe_x(qL, qR, g=1.0):
    L = oracle_lib()
    qL = np.ascontiguousarray(qL, np.float64)
    qR = np.ascontiguousarray(qR, np.float64)
    W = np.zeros(9)
    s = np.zeros(3)
    am = np.zeros(3)
    ap = np.zeros(3)
    rc = L.fco_roe_x(_dp(qL), _dp(qR), g, _dp(W), _dp(s), _dp(am), _dp(ap))
    if rc:
        raise OracleError(rc, "roe_x")
    return W.reshape(3, 3), s, am, ap


def roe_transverse_x(qL, qR, asdq, g=1.0):
    L = oracle_lib()
    qL = np.ascontiguousarray(qL, np.float64)
    qR = np.ascontiguousarray(qR, np.float64)
    d = np.ascontiguousarray(asdq, np.float64)
    bm = np.zeros(3)
    bpv = np.zeros(3)
    rc = L.fco_roe_transverse_x(_dp(qL), _dp(qR), g, _dp(d), _dp(bm), _dp(bpv))
    if rc:
        raise OracleError(rc, "roe_transverse_x")
    return bm, bpv


def mc(theta: float) -> float:
    return oracle_lib().fco_mc(theta)


def patch_step(equation, qpad, dx, dy, dt, g=1.0, adv_u=0.0, adv_v=0.0):
    L = oracle_lib()
    qpad = np.ascontiguousarray(qpad, np.float64)
    F, P, _ = qpad.shape
    m = P - 4
    out = np.zeros((F, m, m))
    smax = C.c_double(0.0)
    rc = L.fco_patch_step(equation, m, g, dx, dy, dt, adv_u, adv_v, _dp(qpad), _dp(out), C.byref(smax))
    if rc:
        raise OracleError(rc, "patch_step")
    return out, smax.value


def swe1d(h, hu, dx, dt, nsteps, g=1.0, efix=0):
    """1D wave propagation (Roe waves, MC-limited corrections, transmissive
    ends); efix = 1 applies the Harten-Hyman entropy fix"""
    L = oracle_lib()
    h = np.array(h, np.float64)
    hu = np.array(hu, np.float64)
    rc = L.fco_swe1d_efix(len(h), dx, dt, nsteps, g, int(efix), _dp(h), _dp(hu))
    if rc:
        raise OracleError(rc, "swe1d")
    return h, hu


def roe_x_efix(qL, qR, g=1.0):
    """entropy-fixed fluctuations (A-dQ, A+dQ) of an x-edge"""
    L = oracle_lib()
    qL = np.ascontiguousarray(qL, np.float64)
    qR = np.ascontiguousarray(qR, np.float64)
    am, ap = np.zeros(3), np.zeros(3)
    rc = L.fco_roe_x_efix(_dp(qL), _dp(qR), g, _dp(am), _dp(ap))
    if rc:
        raise OracleError(rc, "roe_x_efix")
    return am, ap


def swe_exact(hL, uL, hR, uR, xi, g=1.0):
    L = oracle_lib()
    xi = np.ascontiguousarray(xi, np.float64)
    h = np.zeros_like(xi)
    u = np.zeros_like(xi)
    rc = L.fco_swe_exact(hL, uL, hR, uR, g, len(xi), _dp(xi), _dp(h), _dp(u))
    if rc:
        raise OracleError(rc, "swe_exact")
    return h, u


def tag_patch_f32(crit, hpad, threshold):
    L = oracle_lib()
    a = np.ascontiguousarray(hpad, np.float32)
    m = a.shape[0] - 4
    return L.fco_tag_patch_f32(crit, m, np.float32(threshold), a.ctypes.data_as(C.POINTER(C.c_float)))


def cnn_forward(w, x):
    L = oracle_lib()
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    N, _, S, _ = x.shape
    out = np.zeros((N, 2))
    rc = L.fco_cnn_forward(N, S, _dp(w), _dp(x), _dp(out))
    if rc:
        raise OracleError(rc, "cnn_forward")
    return out


def cnn_loss_grad(w, x, targets):
    L = oracle_lib()
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(targets, np.float64)
    N, _, S, _ = x.shape
    g = np.zeros(CNN_NPARAM)
    loss = L.fco_cnn_loss_grad(N, S, _dp(w), _dp(x), _dp(t), _dp(g))
    return loss, g


# cubed-sphere geometry (doubled centred coordinates, N = 2^30) ---------------
SPHERE_N = 1 << 30


def sphere_fold(t, U, V):
    """(tree, U, V) holding a point given in tree t's coordinates, or None
    beyond a cube corner"""
    uo, vo = C.c_longlong(0), C.c_longlong(0)
    t2 = oracle_lib().fco_sphere_fold(t, U, V, C.byref(uo), C.byref(vo))
    return None if t2 < 0 else (t2, uo.value, vo.value)


def sphere_point(t, U, V):
    p = np.zeros(3)
    oracle_lib().fco_sphere_point(t, U, V, _dp(p))
    return p


def sphere_cell_area(t, U0, U1, V0, V1):
    return oracle_lib().fco_sphere_cell_area(t, U0, U1, V0, V1)


def pillow_fold(t, U, V):
    """(tree, U, V) holding a point given in tree t's coordinates (two-tree sphere)"""
    uo, vo = C.c_longlong(0), C.c_longlong(0)
    t2 = oracle_lib().fco_pillow_fold(t, U, V, C.byref(uo), C.byref(vo))
    return (t2, uo.value, vo.value)


def pillow_point(t, U, V):
    p = np.zeros(3)
    oracle_lib().fco_pillow_point(t, U, V, _dp(p))
    return p


def pillow_cell_area(t, U0, U1, V0, V1):
    return oracle_lib().fco_pillow_cell_area(t, U0, U1, V0, V1)
