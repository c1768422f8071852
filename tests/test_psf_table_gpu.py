"""Tabulated-PSF renderers (E2E_PSF_TABLE) against the oracle: the same definition (tables of
pixel integrals of the maps' bilinear density at (P + 1)^2 sub-pixel phases, interpolated in
phase and wavelength), so the mixed renderer meets the separable PSF's tolerance and the
FP64 renderer 5e-11."""
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
# 192, 256 and 32
CASES = [dict(seed=701, coma=0.0), dict(seed=702, coma=0.3, K=9, n_lambda=200, n_slit=12),
         dict(seed=703, coma=0.2, K=13, n_lambda=90, n_slit=20, phases=4),
         dict(seed=704, coma=0.1, K=15, n_lambda=60, n_slit=9, phases=2),
         dict(seed=705, coma=0.2, K=3, n_lambda=120, n_slit=6, phases=16)]


@pytest.mark.parametrize("kw", CASES, ids=[f"t{c['seed']}" for c in CASES])
def test_table_psf_matches_oracle(renderer, kw):
    kw = dict(kw)
    coma, phases = kw.pop("coma"), kw.pop("phases", 8)
    w = W.small_config(orders=2, **kw)
    w = W.Workload(w.name, W.with_psf_maps(w.model, oversample=8.0, half_px=7.0, coma=coma, phases=phases),
                   w.spectra, "f32", "mixed")
    ref = oracle.render_workload(w)
    got = frames(renderer, w, "mixed", "f32")
    for g, o in zip(got, ref):
        rep = compare(g, o)
        assert rep.ok, str(rep)
    g64 = frames(renderer, w, "fp64", "f64")
    for g, o in zip(g64, ref):
        assert np.all(np.abs(g - o) <= 5e-11 * np.abs(o) + 1e-15 * np.abs(o).max())


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
