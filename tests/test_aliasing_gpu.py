"""Flat-field aliasing (Sec. 2.2, Fig. 4) measured on frames from the GPU renderer: the ripple
of the extracted spectrum equals the oracle's and the Poisson-summation amplitude, and ~10
samples per resolution element keep it far below photon noise at ~40000 e-/px."""
import pytest

import oracle
from paper_2008_05858_gb300 import aliasing as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_renderer_ripple_matches_oracle_and_closed_form():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)

    def render(w):
        mid = r.load_model(w.model)
        out = r.render(mid, r.load_spectra(w), "mixed", "f64")[0].cpu().numpy()
        r.unload_model(mid)
        return out

    try:
        rows = A.study(render, samples=(0.75, 1.0, 1.25, 10.0))
    finally:
        r.close()
    for row in rows[:3]:
        assert row["ripple"] == pytest.approx(row["predicted"], rel=2e-3)
    for n in (0.75, 1.0, 1.25):
        w = A.flat_field(n)
        ref = A.measured_ripple(oracle.render_workload(w)[0], w)["ripple"]
        got = next(x for x in rows if x["samples_per_resel"] == n)["ripple"]
        assert got == pytest.approx(ref, rel=1e-4)
    assert rows[-1]["ripple"] < 1e-3 * rows[-1]["photon_noise_peak_pixel"]
