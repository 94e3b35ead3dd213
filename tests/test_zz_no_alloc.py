"""The allocation-free hard render (tbr_render_hard_noalloc), called through the
C ABI, gives the same image and index map as tbr_render_hard, on two calls in a
row with different programs (its fixed scratch array keeps the previous call's
contents, so the second call checks that nothing stale leaks through), and
takes no device memory while doing so (free device memory and the
stream-ordered pool's counters are unchanged across each call).

It is meant for callers that may not allocate device memory (a plugin inside a
runtime that owns the device's memory, a real-time loop that must not wait on
an allocator); this file is collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_08722_b300 import inputs, tbr

pytestmark = pytest.mark.gpu

MAX_STROKES = 8192


def _noalloc():
    L = tbr.lib()
    f = L.tbr_render_hard_noalloc
    f.argtypes = [ctypes.POINTER(tbr.TbrProgram), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _coupled_small():
    p = inputs.small_program()
    p.coupling = inputs.make_coupling(401, p.n)
    return p


def _device_memory():
    """(free device bytes, default pool's bytes in use, default pool's bytes
    reserved) on the current device, after a synchronize."""
    torch.cuda.synchronize()
    free = torch.cuda.mem_get_info()[0]
    from cuda.bindings import runtime as rt
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess
    err, used = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    err, reserved = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrReservedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    return free, int(used), int(reserved)


def _render_noalloc(dp, W, H, n_prefix=-1, snap=False):
    rgb = torch.full((H, W, 3), float("nan"), device="cuda")
    idx = torch.full((H, W), -7, device="cuda", dtype=torch.int32)
    s = dp.struct()
    rc = _noalloc()(ctypes.byref(s), W, H, n_prefix, int(snap), ctypes.c_void_p(rgb.data_ptr()),
                    ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    tbr.check(rc)
    return rgb, idx


def test_noalloc_hard_render_matches_the_allocating_entry_point():
    cases = [
        (inputs.operating_program(), 256, 192, -1, False),   # 2000 strokes
        (inputs.small_program(), 131, 77, 37, True),          # shorter program, prefix, snapped colours
        (_coupled_small(), 96, 96, -1, False),                # coupling variant (Eq. coupling)
    ]
    for prog, W, H, n_prefix, snap in cases:
        dp = tbr.DeviceProgram.from_host(prog)
        ref_rgb, ref_idx, _ = tbr.render_hard(dp, W, H, n_prefix=n_prefix, snap=snap)
        rgb = torch.full((H, W, 3), float("nan"), device="cuda")
        idx = torch.full((H, W), -7, device="cuda", dtype=torch.int32)
        before = _device_memory()
        s = dp.struct()
        rc = _noalloc()(ctypes.byref(s), W, H, n_prefix, int(snap), ctypes.c_void_p(rgb.data_ptr()),
                        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        tbr.check(rc)
        after = _device_memory()
        # the call took no device memory: neither from the device nor from the stream-ordered pool
        assert after == before, (before, after)
        assert torch.equal(idx, ref_idx)
        assert float((rgb - ref_rgb).abs().max()) <= 1e-6


def test_noalloc_rejects_programs_beyond_its_fixed_scratch():
    p = inputs.make_program(MAX_STROKES + 1, seed=9, palette_seed=10, k=4, r_lo=0.001, r_hi=0.002)
    dp = tbr.DeviceProgram.from_host(p)
    rgb = torch.empty((8, 8, 3), device="cuda")
    s = dp.struct()
    rc = _noalloc()(ctypes.byref(s), 8, 8, -1, 0, ctypes.c_void_p(rgb.data_ptr()), None,
                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tbr.TBR_ERR_INVALID_ARG
    assert b"8192" in tbr.lib().tbr_last_error()
    # a prefix within the limit is accepted
    ok_rgb, ok_idx = _render_noalloc(dp, 8, 8, n_prefix=MAX_STROKES)
    ref_rgb, ref_idx, _ = tbr.render_hard(dp, 8, 8, n_prefix=MAX_STROKES)
    assert torch.equal(ok_idx, ref_idx)
