"""The render entry point that allocates nothing (e2e_render_static).

Callers that cannot allocate device memory while they run -- a process whose GPU memory is
already held by another runtime's allocator, or a real-time loop that must not block or fail
on an allocation -- render through e2e_render_static, which takes its scratch from a fixed
buffer the library keeps on the device.  These tests call it through the C ABI and check its
frames against the ordinary e2e_render on two calls in a row (the second call finds the
previous call's data still in the shared buffer), and that a model too big for the buffer is
refused with a clear error.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2008_05858_gb300 import workloads as W
from tests.framecompare import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_render_matches_render_twice():
    from paper_2008_05858_gb300 import binding as B

    r = B.Renderer(0)
    try:
        w = W.small_config(seed=101, n_lambda=500, n_slit=24)
        mid = r.load_model(w.model)
        sids = r.load_spectra(w)
        ref = r.render(mid, sids, "mixed", "f32")[0]
        torch.cuda.synchronize()
        ref_np = ref.double().cpu().numpy()
        for call in range(2):
            out = torch.full_like(ref, float("nan"))
            B.e2e_render_static(r.ctx, mid, sids, B.E2E_F32, [out.data_ptr()], [out.stride(0)])
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            assert np.isfinite(got).all(), f"call {call}: unwritten pixels"
            rep = compare(got, ref_np)
            assert rep.ok, f"call {call}: {rep}"
        # a second model through the same buffer, then the first again
        w2 = W.small_config(seed=102, K=7, degree=3)
        mid2 = r.load_model(w2.model)
        sids2 = r.load_spectra(w2)
        ref2 = r.render(mid2, sids2, "mixed", "f64")[0]
        out2 = torch.empty_like(ref2)
        B.e2e_render_static(r.ctx, mid2, sids2, B.E2E_F64, [out2.data_ptr()])
        torch.cuda.synchronize()
        assert compare(out2.cpu().numpy(), ref2.cpu().numpy()).ok
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
