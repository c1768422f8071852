"""Two-dimensional fiber sub-apertures on the GPU (Sec. 2.2: each image is the fiber's
spatial profile convolved with the PSF): round fibers of n_slit x n_aper points against the
oracle, which renders the 2-D definition directly, for every renderer -- separable mixed and
FP64, elliptical, tabulated PSF, the adjoint (gradients of the caller's slices) and the photon
Monte-Carlo (bit-exact counts).  The library renders each aperture row as a one-dimensional
slice with its lt-terms moved, so these tests also pin that expansion."""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W
from tests.framecompare import compare, tie_boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def frames(r, w, precision, dtype):
    mid = r.load_model(w.model)
    out = r.render(mid, r.load_spectra(w), precision, dtype)
    torch.cuda.synchronize()
    res = [t.double().cpu().numpy() for t in out]
    r.unload_model(mid)
    return res


def fiber_workload(seed, psf=W.PSF_SEPARABLE, n_aper=7, n_slit=6, quad=False, **kw):
    w = W.small_config(seed=seed, psf=psf, **kw)
    m = W.with_round_fiber(w.model, n_aper=n_aper, n_slit=n_slit)
    if quad:  # a quadratic displacement term: rows of a degree-1 slice become degree-2 slices
        for s in m.slices:
            s.aper_x = np.array([3.0, 0.2, 0.15])
            s.aper_y = np.array([0.2, -0.05, 0.04])
    return W.Workload(w.name, m, w.spectra, "f32", "mixed")


CASES = [dict(seed=801), dict(seed=802, K=7, n_lambda=150, n_aper=5, n_slit=9),
         dict(seed=803, K=9, degree=1, n_lambda=120, quad=True), dict(seed=804, K=13, n_aper=2, n_slit=3)]


@pytest.mark.parametrize("kw", CASES, ids=[f"f{c['seed']}" for c in CASES])
def test_round_fiber_matches_oracle(renderer, kw):
    w = fiber_workload(**kw)
    ref = oracle.render_workload(w)
    ties = tie_boxes(w.model, w.flux_for)
    for d, (g, o) in enumerate(zip(frames(renderer, w, "mixed", "f32"), ref)):
        rep = compare(g, o, ties=ties[d])
        assert rep.ok, str(rep)
        assert np.abs(o).max() > 0
    for g, o in zip(frames(renderer, w, "fp64", "f64"), ref):
        assert np.all(np.abs(g - o) <= 5e-11 * np.abs(o) + 1e-15 * np.abs(o).max())


def test_round_fiber_elliptical_and_tabulated(renderer):
    w = fiber_workload(811, psf=W.PSF_ELLIPTICAL, n_lambda=120, n_aper=5, n_slit=5)
    ref = oracle.render_workload(w)
    for g, o in zip(frames(renderer, w, "mixed", "f32"), ref):
        assert compare(g, o).ok
    w2 = fiber_workload(812, n_lambda=90, n_aper=4, n_slit=4, K=9)
    w2 = W.Workload(w2.name, W.with_psf_maps(w2.model, oversample=6.0, half_px=6.0, coma=0.2), w2.spectra, "f32",
                    "mixed")
    ref2 = oracle.render_workload(w2)
    for g, o in zip(frames(renderer, w2, "mixed", "f32"), ref2):
        assert compare(g, o).ok


def test_round_fiber_adjoint_is_the_parent_gradient(renderer):
    from tests.test_adjoint_gpu import check_groups

    w = fiber_workload(821, K=9, degree=3, n_lambda=90, n_aper=5, n_slit=5)
    rng = np.random.default_rng(821)
    dldi = [rng.standard_normal((h, wd)) for h, wd in w.model.det_shape]
    ref = oracle.vjp(w.model, w.flux_for, dldi)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    got = renderer.adjoint(mid, sids, [torch.tensor(d, dtype=torch.float64, device="cuda") for d in dldi])
    torch.cuda.synchronize()
    assert got[0].numel() == sum(W.n_coeffs(s.degree) for s in w.model.slices)
    check_groups(got, ref)
    # an update in the caller's layout renders what a fresh load of the updated model renders
    cx, cy, sx, sy = renderer.params(mid)
    cx = cx + rng.uniform(-0.05, 0.05, cx.shape)
    renderer.update(mid, cx, cy, sx, sy)
    a = renderer.render(mid, sids, "mixed", "f32")[0].cpu().numpy()
    m2 = renderer.models[mid]
    mid2 = renderer.load_model(m2)
    b = renderer.render(mid2, sids, "mixed", "f32")[0].cpu().numpy()
    assert np.array_equal(a, b)
    renderer.unload_model(mid)
    renderer.unload_model(mid2)


def test_round_fiber_photons_bit_exact(renderer):
    from tests.test_photon_gpu import scaled_workload

    w = scaled_workload(fiber_workload(831, n_lambda=150, n_aper=5, n_slit=4), 2e5)
    ref, ref_total = oracle.render_photons(w.model, w.flux_for, seed=99)
    mid = renderer.load_model(w.model)
    out, total = renderer.render_photons(mid, renderer.load_spectra(w), seed=99)
    torch.cuda.synchronize()
    assert total == ref_total
    for g, o in zip(out, ref):
        assert np.array_equal(g.cpu().numpy().view(np.uint32), o)
    renderer.unload_model(mid)


def test_bad_apertures_are_rejected(renderer):
    from paper_2008_05858_gb300.binding import E2EError, E2E_EINVAL

    w = fiber_workload(841)
    m = w.model.copy()
    m.slices[0].n_aper = 65
    m.slices[0].slit_weights = np.ones(65 * m.slices[0].n_slit)
    with pytest.raises(E2EError) as e:
        renderer.load_model(m)
    assert e.value.code == E2E_EINVAL
    m = w.model.copy()
    m.slices[1].aper_x = np.array([np.nan, 0.0, 0.0])
    with pytest.raises(E2EError) as e:
        renderer.load_model(m)
    assert e.value.code == E2E_EINVAL
