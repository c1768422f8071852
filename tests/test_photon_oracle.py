"""Pins of the oracle's photon Monte-Carlo renderer (the alternative of Sec. 2.2): the photon
total is Poisson with the spectrum's expected count, and the counts are distributed as the
image model predicts: a chi-square test against the expected frame that the stamp oracle
computes (finely sampled so that the two models coincide to well below the shot noise)."""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W


def scaled(w, photons):
    tot = sum(float(np.sum(w.flux_for(s))) * (s.lambda_hi - s.lambda_lo) / s.n_lambda * float(np.sum(s.slit_weights))
              for s in w.model.slices)
    k = photons / tot
    return (lambda s: w.flux_for(s) * k), photons


def fine(psf, seed):
    # dense sampling (0.3-0.6 px per sample along x, 0.3 px per slit point) and K = 15
    return W.small_config(seed=seed, psf=psf, K=15, n_lambda=700, n_slit=24, orders=1, fibers=1, slices=2,
                          width=240, height=90)


@pytest.mark.parametrize("psf", [W.PSF_SEPARABLE, W.PSF_ELLIPTICAL], ids=["separable", "elliptical"])
def test_photon_counts_follow_the_image_model(psf):
    w = fine(psf, 11 + psf)
    flux, n = scaled(w, 4e5)
    frames, total = oracle.render_photons(w.model, flux, seed=99)
    assert abs(total - n) < 5 * np.sqrt(n)
    E = oracle.render(w.model, flux)[0] * (total / n)
    c = frames[0].astype(np.float64)
    sel = E >= 10
    chi2 = float(np.sum((c[sel] - E[sel]) ** 2 / E[sel]))
    dof = int(sel.sum())
    assert abs(chi2 / dof - 1.0) < 5 * np.sqrt(2.0 / dof) + 0.05, (chi2, dof)
    assert c.sum() <= total


def test_photon_frames_are_a_function_of_the_seed():
    w = W.small_config(seed=21, n_lambda=50, n_slit=4)
    flux, _ = scaled(w, 2e4)
    a, ta = oracle.render_photons(w.model, flux, seed=5)
    b, tb = oracle.render_photons(w.model, flux, seed=5)
    c, tc = oracle.render_photons(w.model, flux, seed=6)
    assert ta == tb and np.array_equal(a[0], b[0])
    assert not np.array_equal(a[0], c[0])
