"""Band sharding on one GPU: each band of rows rendered as a model of its own (the way one rank
of a multi-GPU run renders its share of a large frame, halo stamps rendered by both
neighbours), the bands concatenated, and the result compared with the whole-frame render and
with the oracle."""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import shard
from paper_2008_05858_gb300 import workloads as W
from tests.framecompare import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def render(r, w, precision="mixed", dtype="f32"):
    from paper_2008_05858_gb300.binding import e2e_unload_spectrum

    mid = r.load_model(w.model)
    sids = r.load_spectra(w)
    try:
        out = r.render(mid, sids, precision, dtype)
        torch.cuda.synchronize()
        return [t.double().cpu().numpy() for t in out]
    finally:
        for s in sids:
            e2e_unload_spectrum(r.ctx, s)
        r.unload_model(mid)


def render_by_bands(r, w, world, **kw):
    bands, rows = [], []
    for rank in range(world):
        sub, rr = shard.shard_workload_by_band(w, rank, world)
        bands.append(render(r, sub, **kw))
        rows.append(rr)
    return shard.assemble_bands(bands, rows, w.model.det_shape)


@pytest.mark.parametrize("world", [2, 3, 8])
def test_bands_match_whole_frame_and_oracle(renderer, world):
    w = W.small_config(seed=403, n_detectors=2, height=200, n_lambda=150, n_slit=9, orders=4, trace_pitch=12.0)
    whole = render(renderer, w)
    banded = render_by_bands(renderer, w, world)
    ref = oracle.render_workload(w)
    for b, a, o in zip(banded, whole, ref):
        assert compare(b, o).ok
        assert compare(b, a).ok


def test_full_detector_frame_in_four_bands(renderer):
    w = W.config2(n_orders=8, n_lambda=1500, n_slit=32)
    whole = render(renderer, w)[0]
    banded = render_by_bands(renderer, w, 4)[0]
    rep = compare(banded, whole)
    assert rep.ok, str(rep)


def test_elliptical_bands(renderer):
    w = W.small_config(seed=404, height=240, orders=4, trace_pitch=12.0, psf=W.PSF_ELLIPTICAL)
    ref = oracle.render_workload(w)
    for b, o in zip(render_by_bands(renderer, w, 3), ref):
        assert compare(b, o).ok
