"""The tensor-core DFT stage (gsm_dft32_tc): length-32 DFTs on tcgen05 with the
operands split into 8-bit digit planes, against the oracle's FFT.

Bound: each input is rounded to 48 bits of its vector's largest value (2^-47
relative to it), the DFT matrix likewise, and the dropped digit-plane products
are below 2^-48; a 32-term sum of such errors stays below 64 * 2^-47 ~ 5e-13 of
the vector's largest input, about 1e-13 of its largest output for the
vectors below.  The test asks for 2e-13 of each vector's largest output."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sign", [-1, 1])
def test_tc_dft32_against_oracle(sign):
    import torch
    import paper_1501_04438_gb300 as gsm
    rng = np.random.default_rng(2026 + sign)
    nvec = 1000                                   # not a multiple of the 128 vectors of a CTA
    x = rng.standard_normal((nvec, 32)) + 1j * rng.standard_normal((nvec, 32))
    x *= 10.0 ** rng.uniform(-4, 4, size=(nvec, 1))   # block scales over eight decades
    x[5] = 0.0                                    # an all-zero vector
    x[6, :] = 0.0
    x[6, 3] = 1e-300                              # a tiny one (subnormal-range products)
    got = gsm.dft32_tc(torch.tensor(x, device="cuda"), sign).cpu().numpy()
    ref = np.stack([oracle.fftn(x[i], sign) for i in range(nvec)])
    scale = np.maximum(np.max(np.abs(ref), axis=1), 1e-300)
    err = np.max(np.abs(got - ref), axis=1) / scale
    assert np.all(got[5] == 0)
    assert np.max(err) < 2e-13, (np.max(err), int(np.argmax(err)))


def test_tc_dft32_rejects_bad_arguments():
    import torch
    import paper_1501_04438_gb300 as gsm
    with pytest.raises(ValueError):
        gsm.dft32_tc(torch.zeros((4, 16), dtype=torch.complex128, device="cuda"))
    from paper_1501_04438_gb300 import _abi
    lib = _abi.load()
    assert lib.gsm_dft32_tc(4, 3, None, None, None) == 1
