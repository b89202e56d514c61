"""The C-ABI library builds for sm_103a, loads on a host without a GPU, and
exports exactly the entry points that include/fc.h declares.  No compute
call is made here."""
import ctypes
import os
import re
import subprocess

from paper_1308_1472_gb300 import _build, fc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fc_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = _build.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_exports_match_header_and_binding():
    names = declared_functions()
    assert len(names) >= 25
    assert set(names) == set(fc.SIGNATURES), set(names) ^ set(fc.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fc_[a-z0-9_]+)\b", out))
    assert set(names) <= exported


def test_build_targets_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_rejects_bad_params_without_gpu():
    L = fc.lib()
    p = fc.fc_params(0, 12, 0, 0, 0, 0, 0, 0, 1, -1, 1.0, 0.9, 0.05, 1.0, 0.0, None)   # m = 12 invalid
    h = ctypes.c_void_p()
    assert L.fc_create(ctypes.byref(p), ctypes.byref(h)) == fc.FC_ERR_INVALID_ARG
    assert b"invalid" in L.fc_last_error()


def declared_functions_3d():
    src = open(os.path.join(ROOT, "include", "fc3.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fc3_[a-z0-9_]+)\s*\(", src)))


def test_3d_exports_match_header_and_binding():
    from paper_1308_1472_gb300 import fc3
    names = declared_functions_3d()
    assert len(names) >= 15
    assert set(names) == set(fc3.SIGNATURES), set(names) ^ set(fc3.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fc3_[a-z0-9_]+)\b", out))
    assert set(names) <= exported


def test_3d_binding_rejects_bad_params_without_gpu():
    from paper_1308_1472_gb300 import fc3
    L = fc3.lib()
    h = ctypes.c_void_p()
    for bad in (dict(m=6), dict(cfl=1.5), dict(transverse=3), dict(max_level=11), dict(subcycle=2)):
        kw = dict(m=8, min_level=1, max_level=2, precision=0, limiter=1, transverse=2, refluxing=1, subcycle=0, device=-1,
                  cfl=0.9, u=1.0, v=0.0, w=0.0, tag_threshold=0.05, stream=None)
        kw.update(bad)
        p = fc3.fc3_params(**kw)
        assert L.fc3_create(ctypes.byref(p), ctypes.byref(h)) == fc.FC_ERR_INVALID_ARG, bad
        assert b"invalid" in L.fc_last_error()
