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
    # batches: an empty one is a no-op; a negative count, NULL arrays or a bad
    # handle are refused on the host before any CUDA call
    assert lib.gsm_apply_batched(0, None, None, None, None) == 0
    assert lib.gsm_apply_batched(-1, None, None, None, None) == 1
    assert lib.gsm_apply_batched(2, None, None, None, None) == 1
    plans = (ctypes.c_void_p * 1)(None)
    arrs = (ctypes.c_void_p * 1)(None)
    assert lib.gsm_apply_batched(1, plans, arrs, arrs, None) == 7


def test_box_and_saved_plan_errors_without_gpu(libpath):
    """Box validation and the checks of a saved plan run on the host, before
    any CUDA call: a bad box, a short buffer, a wrong magic, a size that does
    not match the header, a corrupted checksum."""
    import struct
    from paper_1501_04438_gb300 import _abi
    lib = _abi.load(libpath)
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(16, 16, 16)
    opt = _abi.Options()
    lib.gsm_default_options(ctypes.byref(opt))
    opt.box[0], opt.box[1], opt.box[2] = 4.0, -1.0, 2.0
    assert lib.gsm_plan(ctypes.byref(h), 0, 3, 1.0, n, 0.0, ctypes.byref(opt), None) == 1
    opt.box[1] = 4.0
    opt.box[2] = 0.002          # eta = 5e-4 < delta = 1e-3
    assert lib.gsm_plan(ctypes.byref(h), 0, 3, 1.0, n, 0.0, ctypes.byref(opt), None) == 1
    assert b"delta" in lib.gsm_last_error()

    size = ctypes.c_size_t()
    assert lib.gsm_plan_save(None, None, 0, ctypes.byref(size)) == 7
    assert lib.gsm_plan_load(ctypes.byref(h), b"short", 5, -1, None) == 1
    # a header of the saved layout: magic, version, header bytes, 20 int32, 16 doubles, u64,
    # then the forward and inverse radices of three axes (12 bytes each)
    nterms = 4
    ints = [0, 3, 8, 8, 8, 0, 3, nterms, 5] + [1] * 5 + [8] * 5 + [0]
    dbl = [1.0, 1.0, 1.0, 1.0, 2e-15, 1e-3, 0, 0, 1, 0, 0, 1, 0.0, 0.0, 0.0, 1.0]
    radices = bytes([8, 2] + [0] * 10) * 6
    hdr = struct.pack("<QII20i16dQ", 0x47534D5341564531, 3, 304, *ints, *dbl, 9 ** 3) + radices
    assert len(hdr) == 304
    body = hdr + b"\0" * (8 * (2 * nterms + 9 ** 3))
    bad = body + struct.pack("<Q", 12345)
    assert lib.gsm_plan_load(ctypes.byref(h), bad, len(bad), -1, None) == 1
    assert b"checksum" in lib.gsm_last_error()
    assert lib.gsm_plan_load(ctypes.byref(h), bad[:-8], len(bad) - 8, -1, None) == 1
    assert b"size" in lib.gsm_last_error()
    wrong = struct.pack("<Q", 7) + bad[8:]
    assert lib.gsm_plan_load(ctypes.byref(h), wrong, len(wrong), -1, None) == 1
    assert b"format" in lib.gsm_last_error()
    assert h.value is None


def test_missing_library_fails_loudly(tmp_path):
    from paper_1501_04438_gb300 import _abi
    saved = _abi._lib
    _abi._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _abi.load(str(tmp_path / "nope.so"))
    finally:
        _abi._lib = saved


def _build_c_client(libpath, out):
    """Compile and link tests/c/gsm_c_client.c (C99) against include/gsm.h and
    libgsm.so; returns the gcc result."""
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.dirname(libpath)
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-O1", os.path.join(ROOT, "tests", "c", "gsm_c_client.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), "-o", out,
           "-L", libdir, "-lgsm", "-Wl,-rpath," + libdir, "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def test_c_client_builds_against_header_and_library(libpath, tmp_path):
    """The header is valid C99 and a C program links against the library
    (no GPU needed to build)."""
    r = _build_c_client(libpath, str(tmp_path / "client"))
    assert r.returncode == 0, r.stderr
