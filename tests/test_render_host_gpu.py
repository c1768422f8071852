"""Rendering into host memory (e2e_render_host).

The mixed-precision frame is rendered band by band (whole merge tiles, the same fraction of
every detector's rows) on side streams, and each band is copied to the host as soon as it is
final.  The items, their order and the merge are those of e2e_render, so the host frame must
equal the device render bit for bit (the plain FP64 renderer, which adds with atomics, to
rounding); these tests check that for every PSF kind, several
detectors, ragged heights, frames with fewer tile rows than bands, pitched and pageable
destinations, and that device memory is refused.
"""
import numpy as np
import pytest

from paper_2008_05858_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def _unload(r, mid, sids):
    from paper_2008_05858_gb300.binding import e2e_unload_spectrum

    for s in sids:
        e2e_unload_spectrum(r.ctx, s)
    r.unload_model(mid)


def device_and_host(r, w, precision="mixed", dtype="f32", pad=0, pinned=True):
    """(device-render frames, host-render frames) as numpy arrays; with pad > 0 the host frames
    are views of wider buffers whose padding columns must stay untouched (checked here)."""
    mid = r.load_model(w.model)
    sids = r.load_spectra(w)
    try:
        dev = r.render(mid, sids, precision, dtype)
        torch.cuda.synchronize()
        dev = [t.cpu().numpy() for t in dev]
        td = torch.float32 if dtype == "f32" else torch.float64
        bufs = []
        for h, wd in w.model.det_shape:
            b = torch.full((h, wd + pad), -7.0, dtype=td)
            bufs.append(b.pin_memory() if pinned else b)
        views = [b[:, : b.shape[1] - pad] for b in bufs]
        r.render_host(mid, sids, precision, dtype, out=views)
        for b in bufs:
            if pad:
                assert torch.all(b[:, b.shape[1] - pad:] == -7.0), "padding columns were written"
        return dev, [v.numpy().copy() for v in views]
    finally:
        _unload(r, mid, sids)


def assert_same(dev, host):
    assert len(dev) == len(host)
    for a, b in zip(dev, host):
        assert a.shape == b.shape
        assert np.array_equal(a, b)


def test_full_frame_many_bands_matches_device_render(renderer):
    # 9216 rows = 288 merge-tile rows: 16 bands of 18 tile rows, traces crossing band edges
    w = W.config2(n_orders=12, n_lambda=2000, n_slit=32)
    dev, host = device_and_host(renderer, w)
    assert_same(dev, host)
    assert np.abs(dev[0]).max() > 0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_several_detectors_ragged_height(renderer, dtype):
    # 1000 rows: 32 tile rows (the last one partial) over 16 bands; detector 2 stays empty
    w = W.small_config(seed=61, n_detectors=3, height=1000, width=260, orders=12, trace_pitch=20.0)
    w.model.slices = [s for s in w.model.slices if s.detector != 2]
    dev, host = device_and_host(renderer, w, dtype=dtype)
    assert_same(dev, host)
    assert not host[2].any()


def test_fewer_tile_rows_than_bands(renderer):
    # 160 rows = 5 tile rows: 5 bands of one tile row
    w = W.small_config(seed=62)
    assert_same(*device_and_host(renderer, w))


def test_single_row_frame(renderer):
    w = W.small_config(seed=63, height=1, width=300, n_slit=3)
    for s in w.model.slices:
        s.cy[0] = 0.0
    assert_same(*device_and_host(renderer, w))


@pytest.mark.parametrize("psf", [W.PSF_ELLIPTICAL, W.PSF_TABLE], ids=["elliptical", "table"])
def test_other_psf_kinds(renderer, psf):
    w = W.small_config(seed=64, height=700, orders=6, trace_pitch=20.0,
                       psf=W.PSF_ELLIPTICAL if psf == W.PSF_ELLIPTICAL else W.PSF_SEPARABLE)
    if psf == W.PSF_TABLE:
        w = W.Workload(w.name, W.with_psf_maps(w.model), w.spectra, w.out_dtype, w.precision)
    assert_same(*device_and_host(renderer, w))


def test_fp64_precision(renderer):
    # the plain FP64 renderer adds with FP64 atomics, whose order (and so the last bits) varies
    # from run to run: the two renders agree to rounding, not bit for bit
    w = W.small_config(seed=65, height=400, orders=4, trace_pitch=20.0)
    dev, host = device_and_host(renderer, w, precision="fp64", dtype="f64")
    for a, b in zip(dev, host):
        assert np.all(np.abs(a - b) <= 1e-12 * np.abs(a) + 1e-15 * np.abs(a).max())


def test_pitched_and_pageable_destinations(renderer):
    w = W.small_config(seed=66, height=500, orders=5, trace_pitch=20.0)
    assert_same(*device_and_host(renderer, w, pad=37))
    assert_same(*device_and_host(renderer, w, pinned=False))
    assert_same(*device_and_host(renderer, w, pad=5, pinned=False))


def test_model_without_slices_gives_zero_frame(renderer):
    m = W.OpticalModel([(100, 70)], [])
    mid = renderer.load_model(m)
    try:
        out = renderer.render_host(mid, [], out=[torch.full((100, 70), 3.0).pin_memory()])
        assert not out[0].any().item()
    finally:
        renderer.unload_model(mid)


def test_device_destination_is_refused(renderer):
    from paper_2008_05858_gb300.binding import E2EError

    w = W.small_config(seed=67)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    try:
        with pytest.raises(E2EError):
            renderer.render_host(mid, sids, out=renderer.empty_frames(mid))
    finally:
        _unload(renderer, mid, sids)
