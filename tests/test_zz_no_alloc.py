"""gsm_fft_lines_noalloc: the batched line FFT for callers that cannot
allocate device memory (their memory belongs to another allocator, or the call
sits on a path that must not allocate).  It keeps its twiddle table in the
library's fixed device scratch instead of allocating one per call.

Checked through the C interface against gsm_fft_lines, the entry point that
allocates, with the FFT-engine tolerance of the other GPU tests, on two calls
in a row that reuse the shared scratch with different lengths.  This file is
collected last so that a run stopping at the first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

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
    # two calls in a row through the shared scratch, different lengths and signs
    for M, sign in ((512, -1), (96, +1)):
        x = rng.standard_normal((5, M)) + 1j * rng.standard_normal((5, M))
        xt = torch.tensor(x, dtype=torch.complex128, device="cuda")
        got = _call(lib.gsm_fft_lines_noalloc, M, xt, sign, precision)
        ref = _call(lib.gsm_fft_lines, M, xt, sign, precision)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        err = np.max(np.abs(g - r)) / np.max(np.abs(r))
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
