"""Pins of the oracle's tabulated-PSF path (PSF maps per field point, Sec. 2.1): the
effective-PSF pixel integrals of a sampled Gaussian equal the analytic pixel integrals (erf
differences, an independent formula) to the bilinear-sampling error, they integrate to the
map's unit mass, a centred symmetric map gives a symmetric table, and a model whose maps
are its own Gaussians renders like the analytic PSF up to the phase/field interpolation."""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W


def _slice(K=11, oversample=10.0, half_px=8.0):
    w = W.small_config(seed=601, K=K, n_lambda=80, n_slit=5, orders=1, fibers=1, slices=1)
    s = w.model.slices[0]
    s.psf_map = W.psf_maps(s, oversample=oversample, half_px=half_px)
    return w, s


def _sig(s, lt):
    return (s.sigma_x[0] + s.sigma_x[1] * lt + s.sigma_x[2] * lt * lt,
            s.sigma_y[0] + s.sigma_y[1] * lt + s.sigma_y[2] * lt * lt)


@pytest.mark.parametrize("ph", [(0.0, 0.0), (0.2, -0.1), (-0.5, 0.45)])
def test_epsf_of_a_sampled_gaussian_is_its_pixel_integral(ph):
    from scipy.special import ndtr

    w, s = _slice()
    sx, sy = _sig(s, s.psf_map.field_lt[0])
    H = s.K // 2
    err = 0.0
    for n in range(s.K):
        for m in range(s.K):
            got = oracle.epsf_pixel(s, 0, ph[0], ph[1], m, n)
            ax = ndtr((m - H + 0.5 - ph[0]) / sx) - ndtr((m - H - 0.5 - ph[0]) / sx)
            ay = ndtr((n - H + 0.5 - ph[1]) / sy) - ndtr((n - H - 0.5 - ph[1]) / sy)
            err = max(err, abs(got - ax * ay))
    assert err < 1e-4  # bilinear interpolation of samples 0.1 px apart


def test_epsf_table_has_unit_mass_and_symmetry():
    w, s = _slice(K=15, half_px=7.0)
    tot = sum(oracle.epsf_pixel(s, 2, 0.0, 0.0, m, n) for m in range(15) for n in range(15))
    assert tot == pytest.approx(1.0, abs=1e-12)  # the window covers the whole map
    for m in range(15):
        for n in range(15):
            a = oracle.epsf_pixel(s, 2, 0.0, 0.0, m, n)
            assert a == pytest.approx(oracle.epsf_pixel(s, 2, 0.0, 0.0, 14 - m, 14 - n), rel=1e-13, abs=1e-17)


def test_table_render_approximates_the_analytic_psf():
    w, _ = _slice()
    wt = W.Workload("t", W.with_psf_maps(w.model, oversample=10.0, half_px=8.0), w.spectra, "f64", "mixed")
    a = oracle.render_workload(wt)[0]
    b = oracle.render_workload(w)[0]
    # phase interpolation at P = 8 and linear interpolation of the width between 5 field nodes
    assert np.abs(a - b).max() < 5e-3 * np.abs(b).max()
    assert a.sum() == pytest.approx(b.sum(), rel=2e-3)
