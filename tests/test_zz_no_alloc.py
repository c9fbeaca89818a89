"""gsm_fft_lines_noalloc: the batched line FFT for callers that cannot
allocate device memory (their memory belongs to another allocator, or the call
sits on a path that must not allocate).  It keeps its tables in the library's
fixed device scratch instead of allocating them per call.

Checked through the C interface against gsm_fft_lines, the entry point that
allocates: the same tables and the same arithmetic, so the same bits, on calls
in a row that reuse the shared scratch with different lengths (including the
largest, whose FP64 tables fill most of the scratch); and against the oracle's
FFT with the FFT-engine tolerance of the other GPU tests.  This file is
collected last so that a run stopping at the first failure has run every other
test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _call(fn, M, x, sign, prec):
    import torch
    from paper_1501_04438_gb300 import _abi
    out = torch.empty_like(x)
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    st = fn(M, x.shape[0], sign, _abi.PRECISIONS[prec], ctypes.c_void_p(x.data_ptr()),
            ctypes.c_void_p(out.data_ptr()), stream)
    _abi.check(st)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32"])
def test_noalloc_fft_matches_allocating_fft(precision):
    import torch
    from paper_1501_04438_gb300 import _abi
    lib = _abi.load()
    rng = np.random.default_rng(2024)
    bound = {"fp64": 1e-15, "fp32x2": 2e-14, "fp32": 3e-7}[precision]
    # calls in a row through the shared scratch: different lengths and signs
    for M, sign in ((512, -1), (96, +1), (8192, -1), (320, +1)):
        x = rng.standard_normal((5, M)) + 1j * rng.standard_normal((5, M))
        xt = torch.tensor(x, dtype=torch.complex128, device="cuda")
        got = _call(lib.gsm_fft_lines_noalloc, M, xt, sign, precision)
        ref = _call(lib.gsm_fft_lines, M, xt, sign, precision)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (M, precision)
        g = got.cpu().numpy()
        o = np.stack([oracle.fftn(x[i], sign) for i in range(x.shape[0])])
        err = np.max(np.abs(g - o)) / np.max(np.abs(o))
        assert err <= bound * np.log2(M) * 4, (M, precision, err)


def test_noalloc_fft_rejects_bad_sizes():
    import torch
    from paper_1501_04438_gb300 import _abi
    lib = _abi.load()
    x = torch.zeros((1, 16384), dtype=torch.complex128, device="cuda")
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    st = lib.gsm_fft_lines_noalloc(16384, 1, -1, 0, ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(x.data_ptr()), stream)
    assert st == 2    # GSM_ERR_UNSUPPORTED_SIZE
    assert b"8192" in lib.gsm_last_error()


def test_noalloc_fft_makes_no_library_allocation():
    """With the next device allocation of the library set to fail, the no-alloc
    entry point still succeeds and the library's live allocations do not
    change; the allocating entry point, given the same armed failure, reports
    out-of-memory."""
    import torch
    from paper_1501_04438_gb300 import _abi
    lib = _abi.load()
    x = torch.tensor(np.random.default_rng(7).standard_normal((3, 256)) + 0j, dtype=torch.complex128,
                     device="cuda")
    ref = _call(lib.gsm_fft_lines, 256, x, -1, "fp64")
    torch.cuda.synchronize()
    c0, b0 = ctypes.c_size_t(), ctypes.c_size_t()
    c1, b1 = ctypes.c_size_t(), ctypes.c_size_t()
    lib.gsm_debug_alloc_stats(ctypes.byref(c0), ctypes.byref(b0))
    try:
        lib.gsm_debug_fail_alloc(0)
        got = _call(lib.gsm_fft_lines_noalloc, 256, x, -1, "fp64")
        torch.cuda.synchronize()
        lib.gsm_debug_alloc_stats(ctypes.byref(c1), ctypes.byref(b1))
        assert (c1.value, b1.value) == (c0.value, b0.value)
        assert torch.equal(got, ref)
        out = torch.empty_like(x)
        stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
        st = lib.gsm_fft_lines(256, 3, -1, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 3    # GSM_ERR_OOM: the armed failure was still pending
    finally:
        lib.gsm_debug_fail_alloc(-1)
