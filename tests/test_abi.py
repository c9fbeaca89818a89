"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/gsm.h; the Python binding declares the same set."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gsm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1501_04438_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gsm_[a-z_0-9]+)", out))
    assert set(names) <= exported


def test_binding_declares_the_same_functions(libpath):
    from paper_1501_04438_gb300 import _abi
    assert sorted(_abi.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(libpath):
    from paper_1501_04438_gb300 import _abi
    lib = _abi.load(libpath)
    assert lib.gsm_status_string(0) == b"ok"
    assert lib.gsm_status_string(7) == b"bad plan handle"
    # invalid handles are rejected on the host, before any CUDA call
    assert lib.gsm_apply(None, None, None, None) == 7
    assert lib.gsm_plan_destroy(None) == 7
    opt = _abi.Options()
    lib.gsm_default_options(ctypes.byref(opt))
    assert opt.delta == 1e-3 and opt.precision == 0 and opt.dip_n[2] == 1.0
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(7, 7, 7)
    assert lib.gsm_plan(ctypes.byref(h), 0, 3, 1.0, n, 0.0, None, None) == 2   # odd n
    n = (ctypes.c_int * 3)(16, 16, 16)
    assert lib.gsm_plan(ctypes.byref(h), 0, 2, 1.0, n, 0.0, None, None) == 1   # wrong d
    assert lib.gsm_plan(ctypes.byref(h), 0, 3, -1.0, n, 0.0, None, None) == 1  # L <= 0
    assert b"L" in lib.gsm_last_error()


def test_missing_library_fails_loudly(tmp_path):
    from paper_1501_04438_gb300 import _abi
    saved = _abi._lib
    _abi._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _abi.load(str(tmp_path / "nope.so"))
    finally:
        _abi._lib = saved
