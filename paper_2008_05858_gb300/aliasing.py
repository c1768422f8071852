"""Aliasing of the wavelength sampling: the flat-field study of Sec. 2.2 (Fig. 4).

The image model renders a spectrum from discrete wavelength samples, so a flat field (a
constant photon density along the dispersion) becomes a sum of pixel-integrated PSFs spaced
h px apart along the trace: flat only in the limit h -> 0.  By the Poisson summation formula
the extracted spectrum (each column summed over the trace) ripples with period h and a
relative amplitude, to first order,

    ripple(h) = 2 |P(1/h)| / P(0),   P(f) = exp(-2 pi^2 sigma^2 f^2) sinc(f),

the PSF's Fourier transform times the pixel box's (sinc(f) = sin(pi f) / (pi f)).  Photon
noise on the same column is 1/sqrt(N_e).  The paper samples ~10 times per resolution
element, which keeps aliasing just below photon noise at ~40000 e-/px (Fig. 4); here the
resolution element is the PSF's FWHM, 2 sqrt(2 ln 2) sigma px.

This module builds the flat-field model and measures the ripple of a rendered frame; the
rendering itself is the library's (any renderer of the image model can be passed in).
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Sequence

import numpy as np

from .workloads import OpticalModel, OrderSlice, Spectrum, Workload

FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


def flat_field(samples_per_resel: float, *, sigma: float = 1.5, width: int = 1024, height: int = 48, K: int = 15,
               peak_e: float = 40000.0) -> Workload:
    """One straight trace along x (x = x0 + D lt, y = height/2), a constant spectrum scaled so
    the brightest pixel collects ~peak_e electrons, sampled samples_per_resel times per FWHM."""
    x0, D = width / 2.0, 0.4 * width
    h = FWHM_PER_SIGMA * sigma / samples_per_resel  # px between wavelength samples
    n_lambda = max(2, int(round(2.0 * D / h)))
    lo, hi = 5000.0, 5100.0
    dlam = (hi - lo) / n_lambda
    h = 2.0 * D / n_lambda
    a0 = math.erf(0.5 / (math.sqrt(2.0) * sigma))  # centre pixel's share of the y-profile
    F = peak_e * h / (a0 * dlam)  # photons per Angstrom
    s = OrderSlice(detector=0, order=100, fiber=0, slice=0, degree=1, K=K, n_lambda=n_lambda, n_slit=1,
                   lambda_lo=lo, lambda_hi=hi, cx=np.array([x0, D, 0.0]), cy=np.array([height / 2.0, 0.0, 0.0]),
                   sigma_x=np.array([sigma, 0.0, 0.0]), sigma_y=np.array([sigma, 0.0, 0.0]), theta=0.0,
                   slit_weights=np.array([1.0]))
    model = OpticalModel([(height, width)], [s])
    spec = {0: Spectrum(0, {100: np.full(n_lambda, F)})}
    return Workload(f"flat-field-{samples_per_resel:g}-per-resel", model, spec, "f64", "mixed",
                    f"h = {h:.4f} px, sigma = {sigma} px")


def sample_spacing(w: Workload) -> float:
    s = w.model.slices[0]
    return 2.0 * s.cx[1] / s.n_lambda


def predicted_ripple(h: float, sigma: float) -> float:
    f = 1.0 / h
    return 2.0 * math.exp(-2.0 * math.pi ** 2 * sigma ** 2 * f * f) * abs(float(np.sinc(f)))


def measured_ripple(frame: np.ndarray, w: Workload) -> Dict[str, float]:
    """Half the peak-to-peak of the extracted spectrum over the trace's central 80 %, relative
    to its mean, and the photon-noise level of one extracted column and of the peak pixel."""
    s = w.model.slices[0]
    x0, D = s.cx[0], s.cx[1]
    lo, hi = int(math.ceil(x0 - 0.8 * D)), int(math.floor(x0 + 0.8 * D))
    E = np.asarray(frame, dtype=np.float64).sum(axis=0)[lo:hi]
    mean = float(E.mean())
    return {"ripple": float((E.max() - E.min()) / (2.0 * mean)), "column_electrons": mean,
            "photon_noise_column": 1.0 / math.sqrt(mean),
            "photon_noise_peak_pixel": 1.0 / math.sqrt(float(np.max(frame)))}


def study(render: Callable[[Workload], np.ndarray], samples: Sequence[float] = (0.75, 1.0, 1.25, 1.5, 2.0, 3.0, 5.0, 10.0),
          sigma: float = 1.5, peak_e: float = 40000.0) -> List[Dict[str, float]]:
    """Ripple vs samples per resolution element; render(w) returns the frame of w."""
    rows = []
    for n in samples:
        w = flat_field(n, sigma=sigma, peak_e=peak_e)
        h = sample_spacing(w)
        r = measured_ripple(render(w), w)
        r.update(samples_per_resel=n, spacing_px=h, predicted=predicted_ripple(h, sigma),
                 below_photon_noise=bool(r["ripple"] < r["photon_noise_peak_pixel"]))
        rows.append(r)
    return rows
