"""The render entry point that allocates nothing (e2e_render_static).

Callers that cannot allocate device memory while they run -- a process whose GPU memory is
already held by another runtime's allocator, or a real-time loop that must not block or fail
on an allocation -- render through e2e_render_static, which takes its scratch from a fixed
buffer the library keeps on the device.  These tests call it through the C ABI and check:

- its frames are bitwise those of the ordinary e2e_render (same kernels, same exact box
  sums, same merge order), on two calls in a row: the second call finds the previous
  call's data still in the shared buffer;
- a blazed model, whose blazed spectra and second flux table also live in the buffer;
- nothing is taken from the device's stream-ordered pool (its high-water mark of used bytes
  does not move) and the device's free memory is the same before and after a call (the
  second: the first call in a process may load the library module that holds the buffer);
- a model too big for the buffer is refused with a clear error.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2008_05858_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8  # CUmemPool_attribute values of the driver API


class _DefaultPool:
    """Used-bytes counters of the device's default stream-ordered memory pool (driver API),
    the pool the library's ordinary renders allocate their scratch from."""

    def __init__(self, device=0):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _static(B, r, mid, sids, like, dtype, free_out=None):
    """One static render into a fresh NaN-filled frame; with free_out, also the device's free
    bytes just before and just after the call (the frame is allocated before)."""
    out = torch.full_like(like, float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    B.e2e_render_static(r.ctx, mid, sids, dtype, [out.data_ptr()], [out.stride(0)])
    torch.cuda.synchronize()
    if free_out is not None:
        free_out.append((free0, torch.cuda.mem_get_info()[0]))
    return out.cpu().numpy()


def _blazed(seed):
    w = W.small_config(seed=seed, n_lambda=400, n_slit=20)
    for s in w.model.slices:
        s.blaze_order = 110.0
        s.blaze_lambda = 0.5 * (s.lambda_lo + s.lambda_hi)
    return w


@pytest.mark.parametrize("case", ["plain", "blazed"])
def test_static_render_is_bitwise_the_render_twice(case):
    from paper_2008_05858_gb300 import binding as B

    r = B.Renderer(0)
    pool = _DefaultPool(0)
    try:
        w = W.small_config(seed=101, n_lambda=500, n_slit=24) if case == "plain" else _blazed(105)
        mid = r.load_model(w.model)
        sids = r.load_spectra(w)
        ref = r.render(mid, sids, "mixed", "f32")[0]
        torch.cuda.synchronize()
        ref_np = ref.cpu().numpy()
        assert np.abs(ref_np).max() > 0
        pool.reset_high()
        used0 = pool.get(_USED_MEM_CURRENT)
        for call in range(2):
            free = []
            got = _static(B, r, mid, sids, ref, B.E2E_F32, free)
            # the first call in a process may load the library module that holds the buffer
            assert call == 0 or free[0][0] == free[0][1], f"call {call}: the device's free memory changed"
            assert np.array_equal(got, ref_np), f"call {call}: frames differ from e2e_render"
        assert pool.get(_USED_MEM_HIGH) <= used0, "the static render took memory from the pool"
        # a second model through the same buffer, in FP64, then the first again
        w2 = W.small_config(seed=102, K=7, degree=3)
        mid2 = r.load_model(w2.model)
        sids2 = r.load_spectra(w2)
        ref2 = r.render(mid2, sids2, "mixed", "f64")[0]
        torch.cuda.synchronize()
        assert np.array_equal(_static(B, r, mid2, sids2, ref2, B.E2E_F64), ref2.cpu().numpy())
        assert np.array_equal(_static(B, r, mid, sids, ref, B.E2E_F32), ref_np)
    finally:
        r.close()


def test_static_render_refuses_models_beyond_the_buffer():
    from paper_2008_05858_gb300 import binding as B

    r = B.Renderer(0)
    try:
        w = W.config2(n_orders=24)
        mid = r.load_model(w.model)
        assert r.plan(mid)["scratch_bytes"] > B.E2E_STATIC_SCRATCH_BYTES
        sids = r.load_spectra(w)
        out = torch.empty(w.model.det_shape[0], dtype=torch.float32, device="cuda")
        with pytest.raises(B.E2EError) as e:
            B.e2e_render_static(r.ctx, mid, sids, B.E2E_F32, [out.data_ptr()])
        assert e.value.code == B.E2E_ETOOBIG and "fixed buffer" in str(e.value)
    finally:
        r.close()
