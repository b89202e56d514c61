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
