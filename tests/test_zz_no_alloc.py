"""fmm_morton_order_noalloc (no device allocation) against fmm_morton_order.

The no-allocation entry point serves callers that must not allocate device
memory while they call the library (allocator callbacks, fixed-arena
runtimes, latency-critical loops); its scratch is a fixed device array.  Two
calls in a row must each reproduce the allocating entry point bit for bit
(keys and permutation are integer results), also when the second call is
smaller than the first and the array still holds the first call's data.
"""
import ctypes

import numpy as np
import pytest

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu


def _call_noalloc(fmm, pos_d, keys, perm):
    import torch
    return fmm.noalloc_entry()(
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.c_void_p(pos_d.data_ptr()),
        ctypes.c_int64(pos_d.shape[0]), ctypes.c_void_p(keys.data_ptr()),
        ctypes.c_void_p(perm.data_ptr()))


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    from paper_2005_12351_gb300 import fmm
    cases = [synth.make_system(1_000_000, 0, "plummer", 901)[0],
             synth.make_system(300_001, 0, "uniform", 902)[0]]
    for pos in cases:
        pos_d = torch.from_numpy(pos).cuda()
        ref_keys, ref_perm = fmm.morton_order(pos_d)
        keys = torch.full_like(ref_keys, -1)
        perm = torch.full_like(ref_perm, -1)
        assert _call_noalloc(fmm, pos_d, keys, perm) == fmm.FMM_OK
        torch.cuda.synchronize()
        assert torch.equal(keys, ref_keys) and torch.equal(perm, ref_perm)


def test_noalloc_call_leaves_free_device_memory_unchanged():
    """After the per-device set-up (a call with n == 0 and NULL pointers), a call
    allocates nothing: the device's free memory is the same before and after
    it, and the result is the allocating entry point's."""
    import torch
    from paper_2005_12351_gb300 import fmm
    f = fmm.noalloc_entry()
    assert f(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), None, ctypes.c_int64(0),
             None, None) == fmm.FMM_OK
    pos_d = torch.from_numpy(synth.make_system(500_000, 0, "plummer", 903)[0]).cuda()
    ref_keys, ref_perm = fmm.morton_order(pos_d)
    keys = torch.full_like(ref_keys, -1)
    perm = torch.full_like(ref_perm, -1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _call_noalloc(fmm, pos_d, keys, perm) == fmm.FMM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(keys, ref_keys) and torch.equal(perm, ref_perm)


def test_noalloc_rejects_oversize_and_bad_input():
    import torch
    from paper_2005_12351_gb300 import fmm
    big = torch.zeros((fmm.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float64, device="cuda")
    k = torch.empty(1, dtype=torch.int64, device="cuda")
    p = torch.empty(1, dtype=torch.int32, device="cuda")
    assert _call_noalloc(fmm, big, k, p) == fmm.FMM_EBUDGET
    pos = synth.uniform_cube(1000, 3)
    pos[5, 2] = np.inf
    pos_d = torch.from_numpy(pos).cuda()
    k = torch.empty(1000, dtype=torch.int64, device="cuda")
    p = torch.empty(1000, dtype=torch.int32, device="cuda")
    assert _call_noalloc(fmm, pos_d, k, p) == fmm.FMM_EINVAL
