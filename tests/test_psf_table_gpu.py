"""Tabulated-PSF renderers (E2E_PSF_TABLE) against the oracle, whose stamp is the pixel
integral of the field-blended maps' bilinear density at the stamp's exact sub-pixel centre
(Sec. 2.1 PSF maps per field point, Sec. 2.2 pixel integration).  The library evaluates the
same integral exactly through per-cell biquadratics in the phase, so the mixed renderer meets
the separable PSF's tolerance (1e-6 relative per pixel) and the FP64 renderer the separable FP64
renderer's 5e-11."""
import numpy as np
import pytest

import oracle
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


def frames(r, w, precision, dtype):
    mid = r.load_model(w.model)
    out = r.render(mid, r.load_spectra(w), precision, dtype)
    torch.cuda.synchronize()
    res = [t.double().cpu().numpy() for t in out]
    r.unload_model(mid)
    return res


# K = 11, 9, 13, 15 and 3: FP32 table rows of 121, 81, 169, 225 and 9 floats padded to 128, 96,
# 192, 256 and 32; q = 8, 5, 3, 1 and 12; maps of odd and even size (cells that start half a
# cell into the phase range)
CASES = [dict(seed=701, coma=0.0), dict(seed=702, coma=0.3, K=9, n_lambda=200, n_slit=12, q=5.0, even=True),
         dict(seed=703, coma=0.2, K=13, n_lambda=90, n_slit=20, q=3.0),
         dict(seed=704, coma=0.1, K=15, n_lambda=60, n_slit=9, q=1.0, even=True),
         dict(seed=705, coma=0.2, K=3, n_lambda=120, n_slit=6, q=12.0)]


@pytest.mark.parametrize("kw", CASES, ids=[f"t{c['seed']}" for c in CASES])
def test_table_psf_matches_oracle(renderer, kw):
    kw = dict(kw)
    coma, q, even = kw.pop("coma"), kw.pop("q", 8.0), kw.pop("even", False)
    w = W.small_config(orders=2, **kw)
    w = W.Workload(w.name, W.with_psf_maps(w.model, oversample=q, half_px=7.0, coma=coma, even_size=even),
                   w.spectra, "f32", "mixed")
    ref = oracle.render_workload(w)
    got = frames(renderer, w, "mixed", "f32")
    for g, o in zip(got, ref):
        rep = compare(g, o)
        assert rep.ok, str(rep)
    g64 = frames(renderer, w, "fp64", "f64")
    for g, o in zip(g64, ref):
        # the separable FP64 renderer's bound: the GPU (Horner) and the oracle (monomial sums)
        # place a centre ~1e-13 px apart, which tail pixels amplify by their log-slope
        err = np.abs(g - o)
        print(f"fp64 max rel {np.max(err[o > 0] / o[o > 0]) if (o > 0).any() else 0:.2e}")
        assert np.all(err <= 5e-11 * np.abs(o) + 1e-15 * np.abs(o).max())


def test_bad_maps_are_rejected(renderer):
    from paper_2008_05858_gb300.binding import E2EError, E2E_EINVAL

    w = W.small_config(seed=711)
    m = W.with_psf_maps(w.model)
    m.slices[0].psf_map.maps[0, 3, 3] = -1.0
    with pytest.raises(E2EError) as e:
        renderer.load_model(m)
    assert e.value.code == E2E_EINVAL
    m = W.with_psf_maps(w.model)
    m.slices[1].psf_map.field_lt[1] = m.slices[1].psf_map.field_lt[0]
    with pytest.raises(E2EError) as e:
        renderer.load_model(m)
    assert e.value.code == E2E_EINVAL
    for q in (2.5, 33.0, 0.0):  # the phase cells need an integer number of samples per pixel
        m = W.with_psf_maps(w.model)
        m.slices[0].psf_map.oversample = q
        with pytest.raises(E2EError) as e:
            renderer.load_model(m)
        assert e.value.code == E2E_EINVAL and "map_oversample" in str(e.value)
