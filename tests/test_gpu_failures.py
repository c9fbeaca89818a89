"""Failure handling on the GPU path, with every failure made on the host.

Out-of-memory: gsm_debug_fail_alloc makes the k-th device allocation of the
library fail, for every k along a call, and gsm_debug_alloc_stats shows that
each failing call returns GSM_ERR_OOM and leaves the library's live
allocations as they were (nothing leaks), and that the call succeeds once k
is past its last allocation.  Stale handles: a destroyed plan or batch handle
is rejected with GSM_ERR_BAD_PLAN.  Bounded waits: the batch queue
kernel, told by a test hook that one instance's first pass never completes,
reports GSM_ERR_TIMEOUT after the bound with every CTA returned, and the next
batch on the same context gives the right bits.  No test here makes a GPU
fault, trap or hang, and nothing is left waiting after a call returns.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1501_04438_gb300 import _abi
    return _abi.load()


def _stats():
    c, b = ctypes.c_size_t(), ctypes.c_size_t()
    assert _lib().gsm_debug_alloc_stats(ctypes.byref(c), ctypes.byref(b)) == 0
    return c.value, b.value


def _sweep(call, max_k=64):
    """Run call() with the k-th allocation failing for k = 0, 1, ...: each run
    must fail with GSM_ERR_OOM without changing the live allocations, until a
    run succeeds.  Returns the number of allocations the call made."""
    lib = _lib()
    try:
        for k in range(max_k):
            before = _stats()
            lib.gsm_debug_fail_alloc(k)
            status, cleanup = call()
            lib.gsm_debug_fail_alloc(-1)
            if status == 0:
                cleanup()
                assert _stats() == before
                return k
            assert status == 3, (k, status, lib.gsm_last_error())
            assert _stats() == before, (k, before, _stats())
        raise AssertionError("call still failing after max_k allocations")
    finally:
        lib.gsm_debug_fail_alloc(-1)


@pytest.mark.parametrize("kernel,d,prec,dip", [
    (0, 3, 0, None), (0, 3, 1, None), (0, 3, 2, None), (2, 2, 0, None),
    (3, 3, 0, ((0.6, 0.0, 0.8), (0.0, 0.8, 0.6))),     # general dipolar: half-spectrum table
])
def test_plan_creation_out_of_memory_leaks_nothing(kernel, d, prec, dip):
    from paper_1501_04438_gb300 import _abi
    lib = _lib()
    opt = _abi.Options()
    lib.gsm_default_options(ctypes.byref(opt))
    opt.precision = prec
    if dip:
        for i in range(3):
            opt.dip_n[i], opt.dip_m[i] = dip[0][i], dip[1][i]
    n = (ctypes.c_int * 3)(16, 20, 24)

    def call():
        h = ctypes.c_void_p()
        st = lib.gsm_plan(ctypes.byref(h), kernel, d, 3.0, n, 0.0, ctypes.byref(opt), None)
        if st != 0:
            assert not h.value
        return st, (lambda: lib.gsm_plan_destroy(h))

    allocs = _sweep(call)
    assert allocs >= 8


def test_apply_host_hartree_autotune_out_of_memory_leaks_nothing():
    """The staging buffers of the host apply (pageable arrays), the scratch of
    the energy and the temporaries of the tuner: each failure point returns
    GSM_ERR_OOM, releases what the call took and leaves the plan usable."""
    import torch
    import paper_1501_04438_gb300 as gsm
    lib = _lib()
    plan = gsm.Plan("coulomb3d", 3.0, (16, 12, 20))
    rho = np.random.default_rng(3).standard_normal(plan.shape)
    ref = plan.apply(torch.tensor(rho, device="cuda")).cpu().numpy()
    out = np.empty_like(rho)

    def host_apply():
        st = lib.gsm_apply_host(plan.handle, ctypes.c_void_p(rho.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                                None)
        return st, (lambda: None)

    # the staging buffers stay with the plan once made, so compare after destroy
    before = _stats()
    lib.gsm_debug_fail_alloc(0)
    assert host_apply()[0] == 3
    lib.gsm_debug_fail_alloc(1)
    assert host_apply()[0] == 3
    lib.gsm_debug_fail_alloc(-1)
    assert _stats() == before
    assert host_apply()[0] == 0
    assert np.array_equal(out, ref)

    psi = torch.tensor(np.random.default_rng(4).standard_normal(plan.shape + (2,)), device="cuda")
    psi = torch.view_as_complex(psi).contiguous()
    lib.gsm_debug_fail_alloc(0)
    with pytest.raises(gsm.GSMError, match="OOM"):
        plan.hartree(psi)
    lib.gsm_debug_fail_alloc(-1)
    e1, _, _ = plan.hartree(psi)

    plan.destroy()

    # the tuner: a failure part-way puts the plan's schedules back (same bits
    # as before); a success may change the plan's tables, so leaks are checked
    # against the state before the plan was made
    base = _stats()
    for k in range(64):
        p2 = gsm.Plan("coulomb3d", 3.0, (16, 12, 20))
        info0 = p2.info()
        lib.gsm_debug_fail_alloc(k)
        st = lib.gsm_plan_autotune(p2.handle, None, None, 0)
        lib.gsm_debug_fail_alloc(-1)
        if st == 0:
            p2.destroy()
            assert _stats() == base
            break
        assert st == 3, (k, st)
        info1 = p2.info()
        assert info1["radix_fwd"] == info0["radix_fwd"] and info1["radix_inv"] == info0["radix_inv"]
        assert np.array_equal(p2.apply(torch.tensor(rho, device="cuda")).cpu().numpy(), ref)
        p2.destroy()
        assert _stats() == base, (k, base, _stats())
    else:
        raise AssertionError("the tuner still failed after 64 allocations")


def test_destroyed_handles_are_rejected():
    import torch
    import paper_1501_04438_gb300 as gsm
    lib = _lib()
    plan = gsm.Plan("coulomb3d", 3.0, 16)
    h = ctypes.c_void_p(plan.handle.value)
    rho = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    batch = gsm.Batch([plan], [rho])
    hb = ctypes.c_void_p(batch._h.value)
    batch.destroy()
    assert lib.gsm_batch_launch(hb, None) == 7
    assert lib.gsm_batch_destroy(hb) == 7
    plan.destroy()
    u = torch.empty_like(rho)
    assert lib.gsm_apply(h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr()), None) == 7
    assert lib.gsm_plan_destroy(h) == 7
    info = gsm._abi.PlanInfo()
    assert lib.gsm_plan_info(h, ctypes.byref(info)) == 7


def test_batch_wait_runs_out_reported_and_recoverable():
    import torch
    import paper_1501_04438_gb300 as gsm
    lib = _lib()
    plans = [gsm.Plan("coulomb3d", 4.0, n) for n in (16, 20, 24)]
    rhos = [torch.tensor(np.random.default_rng(n).standard_normal((n, n, n)), device="cuda") for n in (16, 20, 24)]
    singles = [p.apply(r).clone() for p, r in zip(plans, rhos)]
    before = _stats()
    lib.gsm_debug_batch_wait(20_000_000, 1)     # 20 ms; instance 1's first pass never completes
    try:
        with pytest.raises(gsm.GSMError) as ei:
            gsm.apply_batched(plans, rhos)
        assert ei.value.status == 6
        with pytest.raises(gsm.GSMError) as ei:   # creation runs the batch to time it
            gsm.Batch(plans, rhos)
        assert ei.value.status == 6
    finally:
        lib.gsm_debug_batch_wait(0, -1)
    torch.cuda.synchronize()
    assert _stats() == before
    outs = gsm.apply_batched(plans, rhos)
    for o, s1 in zip(outs, singles):
        assert torch.equal(o, s1)
    batch = gsm.Batch(plans, rhos)
    batch.launch()
    for o, s1 in zip(batch.wait(), singles):
        assert torch.equal(o, s1)
    batch.destroy()
