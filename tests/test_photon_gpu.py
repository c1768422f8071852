"""Photon Monte-Carlo renderer (e2e_render_photons) against the oracle: the same photons,
so the counts are compared bit for bit (every decision -- the bin's photon count, the slit
point, the pixel -- is taken in FP64 on both sides; the spectral-format polynomial is
evaluated in a different order, which moves a pixel decision only for a photon within
~1e-12 px of a pixel edge)."""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def scaled_workload(w, photons):
    tot = sum(float(np.sum(w.flux_for(s))) * (s.lambda_hi - s.lambda_lo) / s.n_lambda * float(np.sum(s.slit_weights))
              for s in w.model.slices)
    k = photons / tot
    for f in w.spectra.values():
        for o in f.flux:
            f.flux[o] = f.flux[o] * k
    return w


CASES = [dict(seed=301), dict(seed=302, K=7, n_lambda=257, n_slit=16, n_detectors=2),
         dict(seed=303, psf=W.PSF_ELLIPTICAL, n_lambda=200, n_slit=9), dict(seed=304, degree=0, n_slit=1)]


@pytest.mark.parametrize("kw", CASES, ids=[f"p{c['seed']}" for c in CASES])
@pytest.mark.parametrize("photons", [3e4, 1e6])
def test_photon_counts_bit_exact(renderer, kw, photons):
    w = scaled_workload(W.small_config(**kw), photons)
    ref, ref_total = oracle.render_photons(w.model, w.flux_for, seed=4242)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    out, total = renderer.render_photons(mid, sids, seed=4242)
    torch.cuda.synchronize()
    assert total == ref_total
    for g, o in zip(out, ref):
        got = g.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, o), int((got != o).sum())
    renderer.unload_model(mid)


@pytest.mark.parametrize("photons", [3e2, 3e6])
def test_sparse_spectrum_bit_exact(renderer, photons):
    """An emission-line spectrum: all but every 97th bin empty, so photons sit in a few heavy
    bins between long runs of empty ones (the bin search between two guide entries must skip
    the empty bins), with fewer photons than guide entries (3e2) and more (3e6)."""
    w = W.small_config(seed=306, n_lambda=1000, n_slit=7)
    for fib, sp in w.spectra.items():
        for o in sp.flux:
            x = np.zeros_like(np.asarray(sp.flux[o], dtype=np.float64))
            x[(o * 13 + fib * 5) % 97::97] = 1.0
            sp.flux[o] = x
    w = scaled_workload(w, photons)
    ref, ref_total = oracle.render_photons(w.model, w.flux_for, seed=77)
    mid = renderer.load_model(w.model)
    out, total = renderer.render_photons(mid, renderer.load_spectra(w), seed=77)
    torch.cuda.synchronize()
    assert total == ref_total and total > 0
    for g, o in zip(out, ref):
        got = g.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, o), int((got != o).sum())
    renderer.unload_model(mid)


def test_empty_model_and_zero_flux(renderer):
    m = W.OpticalModel([(20, 30)], [])
    mid = renderer.load_model(m)
    out, total = renderer.render_photons(mid, [], seed=1)
    torch.cuda.synchronize()
    assert total == 0 and not out[0].any().item()
    renderer.unload_model(mid)
    w = scaled_workload(W.small_config(seed=305), 1e4)
    for f in w.spectra.values():
        for o in f.flux:
            f.flux[o] = f.flux[o] * 0.0
    mid = renderer.load_model(w.model)
    out, total = renderer.render_photons(mid, renderer.load_spectra(w), seed=1)
    torch.cuda.synchronize()
    assert total == 0 and not out[0].any().item()
    renderer.unload_model(mid)


def test_blazed_photons_bit_exact(renderer):
    w = scaled_workload(W.small_config(seed=321, orders=2), 2e5)
    for s in w.model.slices:
        s.blaze_order = 110.0
        s.blaze_lambda = 0.5 * (s.lambda_lo + s.lambda_hi)
    ref, ref_total = oracle.render_photons(w.model, w.flux_for, seed=77)
    mid = renderer.load_model(w.model)
    out, total = renderer.render_photons(mid, renderer.load_spectra(w), seed=77)
    torch.cuda.synchronize()
    assert total == ref_total
    assert np.array_equal(out[0].cpu().numpy().view(np.uint32), ref[0])
    renderer.unload_model(mid)
