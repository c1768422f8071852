"""Seeded synthetic echelle workloads: optical models, slit profiles and spectra.

This module only *generates inputs*.  It holds none of the renderer's arithmetic
(no sample grid, no polynomial evaluation, no PSF integral): the CUDA renderer
and the CPU oracle each implement that themselves, and both consume the plain
arrays built here.

Every workload stands in for an instrument the paper simulates (ESPRESSO and
ELT-HIRES echellograms, Sec. 4): there are no optical design files, spectra or
frames on this machine, so the shapes below (detector size, orders x fibers x
slices, samples per order, slit points, PSF width, polynomial degree, stamp size)
are those of the named configurations, with seeded random geometry and spectra.

Conventions shared with the C ABI (the renderer's header documents them too):

* An *order-slice* is one trace on one detector: (detector, order, fiber, slice).
* Mapping coefficients ``cx``/``cy`` multiply monomials ``lt**a * s**b`` with
  ``a+b <= degree``; they are ordered by total degree ``t = a+b`` ascending and,
  within a degree, by ``a`` descending: index(a, b) = t(t+1)/2 + b.
* ``lt`` is the wavelength normalised to [-1, 1] over [lambda_lo, lambda_hi];
  ``s`` is the slit coordinate in [-1, 1].
* ``flux[j]`` is the photon flux density (photons per Angstrom) of sample ``j``
  of the order, sampled at the centre of the j-th of ``n_lambda`` equal bins
  spanning [lambda_lo, lambda_hi].
* ``slit_weights[k]`` is the normalised illumination of slit point ``k``
  (Sec. 2.1: a normalised per-fiber illumination profile).
* ``sigma_x``/``sigma_y`` are the quadratic coefficients (in ``lt``) of the PSF
  widths in pixels; for the elliptical PSF they are the widths along the PSF's
  own axes, which are rotated by ``theta`` (radians) from the detector axes.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

PSF_SEPARABLE = 0
PSF_ELLIPTICAL = 1
PSF_TABLE = 2

#: seed base: the arXiv identifier of the paper; config i uses SEED_BASE + i
SEED_BASE = 200805858

#: grating relation m * lambda_centre = const (Angstrom), used to lay out orders
GRATING_CONST_A = 6.0e5

C_KMS = 299792.458


def n_coeffs(degree: int) -> int:
    """Number of monomials lt**a s**b with a+b <= degree."""
    return (degree + 1) * (degree + 2) // 2


def coeff_index(a: int, b: int) -> int:
    """Position of the monomial lt**a s**b in a coefficient vector."""
    t = a + b
    return t * (t + 1) // 2 + b


@dataclass
class OrderSlice:
    detector: int
    order: int
    fiber: int
    slice: int
    degree: int
    K: int
    n_lambda: int
    n_slit: int
    lambda_lo: float
    lambda_hi: float
    cx: np.ndarray
    cy: np.ndarray
    sigma_x: np.ndarray
    sigma_y: np.ndarray
    theta: float
    slit_weights: np.ndarray
    blaze_order: float = 0.0   # echelle order of the blaze function (0: no blaze)
    blaze_lambda: float = 0.0  # its blaze wavelength (Angstrom)
    psf_map: "PsfMap | None" = None  # tabulated PSF (models with psf = PSF_TABLE)
    # two-dimensional fiber sub-aperture: n_aper rows t_l at the bin centres of [-1, 1]
    # (0 or 1: a one-dimensional pseudo-slit), slit_weights then n_slit per row (row-major), and
    # the image of row l moved by t_l (aper_x(lt), aper_y(lt)) px, quadratics in lt
    n_aper: int = 0
    aper_x: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    aper_y: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))

    def copy(self) -> "OrderSlice":
        return dataclasses.replace(
            self,
            psf_map=None if self.psf_map is None else self.psf_map.copy(),
            cx=self.cx.copy(),
            cy=self.cy.copy(),
            sigma_x=self.sigma_x.copy(),
            sigma_y=self.sigma_y.copy(),
            slit_weights=self.slit_weights.copy(),
            aper_x=np.array(self.aper_x, dtype=np.float64),
            aper_y=np.array(self.aper_y, dtype=np.float64),
        )

    @property
    def n_points(self) -> int:
        """Sub-aperture points: n_slit, or n_slit x n_aper for a 2-D fiber."""
        return self.n_slit * (self.n_aper if self.n_aper > 1 else 1)


@dataclass
class PsfMap:
    """Tabulated PSF of one order-slice: maps[f] samples the PSF density at offsets
    ((u - c)/oversample, (v - c)/oversample) px from the centre (c = (M - 1)/2) at the
    normalised wavelength field_lt[f]."""

    field_lt: np.ndarray
    maps: np.ndarray  # (n_field, M, M)
    oversample: float

    def copy(self) -> "PsfMap":
        return PsfMap(self.field_lt.copy(), self.maps.copy(), self.oversample)


def psf_maps(s: "OrderSlice", *, n_field: int = 5, oversample: float = 10.0, half_px: float = 8.0,
             coma: float = 0.0, even_size: bool = False) -> PsfMap:
    """Synthetic PSF maps (the optical design's maps are not available): at n_field
    wavelengths the slice's Gaussian (widths sigma_x, sigma_y at that wavelength), plus, when
    coma > 0, a fainter Gaussian displaced along x by 1.5 sigma_x (a comatic tail) carrying
    that fraction of the light.  The map has an odd number of samples per side (a sample at
    the centre) unless even_size, which centres the PSF between the two middle samples."""
    M = int(2 * round(half_px * oversample) + (0 if even_size else 1))
    c = (M - 1) / 2.0
    lt = np.linspace(-1.0, 1.0, n_field)
    x = (np.arange(M) - c) / oversample
    maps = np.empty((n_field, M, M))
    for f, l in enumerate(lt):
        sx = s.sigma_x[0] + s.sigma_x[1] * l + s.sigma_x[2] * l * l
        sy = s.sigma_y[0] + s.sigma_y[1] * l + s.sigma_y[2] * l * l
        gx = np.exp(-0.5 * (x / sx) ** 2) / sx
        gy = np.exp(-0.5 * (x / sy) ** 2) / sy
        img = np.outer(gy, gx)
        if coma > 0:
            gx2 = np.exp(-0.5 * ((x - 1.5 * sx) / (1.3 * sx)) ** 2) / (1.3 * sx)
            img = (1 - coma) * img + coma * np.outer(gy, gx2)
        maps[f] = img / (2 * np.pi)
    return PsfMap(lt, maps, oversample)


def with_round_fiber(model: "OpticalModel", n_aper: int = 8, n_slit: int = 8, extent_x: float = 3.6,
                     tilt_y: float = 0.3) -> "OpticalModel":
    """The model with every slice's fiber a round two-dimensional sub-aperture: an n_slit x n_aper
    grid of points at the bin centres of [-1, 1]^2 weighted by the unit disk (each slice keeping
    its total slit weight), the second axis imaged along the dispersion with half-extent
    extent_x px (slowly varying with wavelength) and a small cross-dispersion tilt tilt_y px."""
    m = model.copy()
    s_ = (2 * np.arange(n_slit) + 1 - n_slit) / n_slit
    t_ = (2 * np.arange(n_aper) + 1 - n_aper) / n_aper
    disk = ((t_[:, None] ** 2 + s_[None, :] ** 2) <= 1.0).astype(np.float64)
    for s in m.slices:
        tot = float(np.sum(s.slit_weights))
        s.n_slit = n_slit
        s.n_aper = n_aper
        s.slit_weights = (disk / disk.sum() * tot).ravel()
        s.aper_x = np.array([extent_x, 0.04 * extent_x, 0.0])
        s.aper_y = np.array([tilt_y, 0.0, 0.0])
    return m


def with_psf_maps(model: "OpticalModel", **kw) -> "OpticalModel":
    """The model with every slice's PSF replaced by synthetic tabulated maps (psf_maps)."""
    m = model.copy()
    for s in m.slices:
        s.psf_map = psf_maps(s, **kw)
    m.psf = PSF_TABLE
    return m


@dataclass
class OpticalModel:
    """Spectral format of one instrument: detectors and their order-slices."""

    det_shape: List[Tuple[int, int]]  # (height, width) per detector, pixels
    slices: List[OrderSlice]
    psf: int = PSF_SEPARABLE

    def copy(self) -> "OpticalModel":
        return OpticalModel(list(self.det_shape), [s.copy() for s in self.slices], self.psf)

    @property
    def n_stamps(self) -> int:
        return int(sum(s.n_lambda * s.n_points for s in self.slices))

    @property
    def n_deposits(self) -> int:
        return int(sum(s.n_lambda * s.n_points * s.K * s.K for s in self.slices))

    @property
    def fibers(self) -> List[int]:
        return sorted({s.fiber for s in self.slices})


@dataclass
class Spectrum:
    """Flux samples of one fiber for a set of orders (order -> flux[n_lambda])."""

    fiber: int
    flux: Dict[int, np.ndarray]


@dataclass
class Workload:
    name: str
    model: OpticalModel
    spectra: Dict[int, Spectrum]  # fiber -> spectrum
    out_dtype: str  # "f32" or "f64"
    precision: str  # "mixed" or "fp64"
    notes: str = ""

    def flux_for(self, s: OrderSlice) -> np.ndarray:
        return self.spectra[s.fiber].flux[s.order]


# --------------------------------------------------------------------------
# spectra
# --------------------------------------------------------------------------


def bin_centres(lambda_lo: float, lambda_hi: float, n: int) -> np.ndarray:
    """Wavelengths at which the flux samples of an order are given."""
    step = (lambda_hi - lambda_lo) / n
    return lambda_lo + (np.arange(n, dtype=np.float64) + 0.5) * step


def absorption_spectrum(
    lam: np.ndarray,
    continuum: float,
    centres: np.ndarray,
    depths: np.ndarray,
    widths: np.ndarray,
) -> np.ndarray:
    """Flat continuum times Gaussian absorption lines (``widths`` are Gaussian sigmas)."""
    f = np.full(lam.shape, continuum, dtype=np.float64)
    for c, d, w in zip(centres, depths, widths):
        near = np.abs(lam - c) < 8.0 * w
        if np.any(near):
            f[near] *= 1.0 - d * np.exp(-0.5 * ((lam[near] - c) / w) ** 2)
    return f


def fabry_perot_comb(lam: np.ndarray, continuum: float, lam0: float, dv_kms: float = 10.0) -> np.ndarray:
    """Airy transmission comb with lines equally spaced in velocity.

    Lines sit at lam0 * (1 + dv/c)**n; the coefficient of finesse is chosen so that a
    line's FWHM is about a tenth of the spacing.
    """
    step = np.log1p(dv_kms / C_KMS)
    coef = (20.0 / np.pi) ** 2  # FWHM/period = 2/(pi*sqrt(coef)) = 0.1
    phase = np.pi * np.log(lam / lam0) / step
    return continuum / (1.0 + coef * np.sin(phase) ** 2)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------


def _order_numbers(n_orders: int, first: int) -> List[int]:
    return [first + i for i in range(n_orders)]


def _make_slice(
    rng: np.random.Generator,
    *,
    detector: int,
    order: int,
    fiber: int,
    slc: int,
    width: int,
    y_centre: float,
    degree: int,
    K: int,
    n_lambda: int,
    n_slit: int,
    sigma: Tuple[float, float, float] | None,
    sigma_range: Tuple[float, float] | None,
    theta: float,
    slit_half_height: float = 4.0,
) -> OrderSlice:
    lam_c = GRATING_CONST_A / order
    half = 0.6 * lam_c / order
    nc = n_coeffs(degree)
    cx = np.zeros(nc)
    cy = np.zeros(nc)
    for t in range(2, degree + 1):
        for b in range(t + 1):
            a = t - b
            cx[coeff_index(a, b)] = rng.uniform(-1.0, 1.0) * 2.0 ** (-t)
            cy[coeff_index(a, b)] = rng.uniform(-1.0, 1.0) * 2.0 ** (-t)
    cx[coeff_index(0, 0)] = width / 2.0
    cy[coeff_index(0, 0)] = y_centre
    if degree >= 1:
        cx[coeff_index(1, 0)] = 0.45 * width
        cx[coeff_index(0, 1)] = rng.uniform(-1.0, 1.0)  # slit tilt
        cy[coeff_index(1, 0)] = rng.uniform(-1.0, 1.0) * 0.5
        cy[coeff_index(0, 1)] = slit_half_height
    if degree >= 2:
        cy[coeff_index(2, 0)] = rng.uniform(5.0, 20.0)  # order curvature
    if sigma is not None:
        sx = np.array(sigma, dtype=np.float64)
        sy = np.array(sigma, dtype=np.float64)
    else:
        lo, hi = sigma_range
        mid = 0.5 * (lo + hi)
        span = 0.5 * (hi - lo)

        def poly():
            c0 = rng.uniform(mid - 0.25 * span, mid + 0.25 * span)
            room = min(c0 - lo, hi - c0)
            c1 = rng.uniform(-0.5, 0.5) * room
            c2 = rng.uniform(-0.5, 0.5) * (room - abs(c1))
            return np.array([c0, c1, c2])

        sx = poly()
        sy = poly()
    return OrderSlice(
        detector=detector,
        order=order,
        fiber=fiber,
        slice=slc,
        degree=degree,
        K=K,
        n_lambda=n_lambda,
        n_slit=n_slit,
        lambda_lo=lam_c - half,
        lambda_hi=lam_c + half,
        cx=cx,
        cy=cy,
        sigma_x=sx,
        sigma_y=sy,
        theta=theta,
        slit_weights=np.full(n_slit, 1.0 / n_slit),
    )


def echelle_model(
    rng: np.random.Generator,
    *,
    n_detectors: int,
    height: int,
    width: int,
    orders_per_detector: int,
    fibers: int,
    slices: int,
    degree: int,
    K: int,
    n_lambda: int,
    n_slit: int,
    first_order: int,
    sigma: Tuple[float, float, float] | None = None,
    sigma_range: Tuple[float, float] | None = None,
    psf: int = PSF_SEPARABLE,
    max_theta_deg: float = 10.0,
    trace_pitch: float = 16.0,
) -> OpticalModel:
    """Evenly spaced orders; each order holds fibers x slices traces ``trace_pitch`` px apart."""
    out: List[OrderSlice] = []
    band = height / orders_per_detector
    n_tr = fibers * slices
    order = first_order
    for det in range(n_detectors):
        for m in range(orders_per_detector):
            yc = (m + 0.5) * band
            theta = 0.0
            if psf == PSF_ELLIPTICAL:
                theta = np.deg2rad(rng.uniform(-max_theta_deg, max_theta_deg))
            for f in range(fibers):
                for sl in range(slices):
                    i = f * slices + sl
                    off = (i - (n_tr - 1) / 2.0) * trace_pitch
                    out.append(
                        _make_slice(
                            rng,
                            detector=det,
                            order=order,
                            fiber=f,
                            slc=sl,
                            width=width,
                            y_centre=yc + off,
                            degree=degree,
                            K=K,
                            n_lambda=n_lambda,
                            n_slit=n_slit,
                            sigma=sigma,
                            sigma_range=sigma_range,
                            theta=theta,
                        )
                    )
            order += 1
    return OpticalModel([(height, width)] * n_detectors, out, psf)


def science_spectra(
    rng: np.random.Generator,
    model: OpticalModel,
    fiber: int,
    n_lines: int,
    continuum: float = 2.0e3,
    depth: Tuple[float, float] = (0.1, 0.9),
    width: Tuple[float, float] = (0.02, 0.1),
) -> Spectrum:
    """Continuum with ``n_lines`` seeded Gaussian absorption lines spread over all orders."""
    orders = {}
    for s in model.slices:
        if s.fiber == fiber:
            orders[s.order] = s
    keys = sorted(orders)
    lo = min(orders[k].lambda_lo for k in keys)
    hi = max(orders[k].lambda_hi for k in keys)
    centres = rng.uniform(lo, hi, n_lines)
    depths = rng.uniform(depth[0], depth[1], n_lines)
    widths = rng.uniform(width[0], width[1], n_lines)
    flux = {}
    for k in keys:
        s = orders[k]
        lam = bin_centres(s.lambda_lo, s.lambda_hi, s.n_lambda)
        sel = (centres > s.lambda_lo - 1.0) & (centres < s.lambda_hi + 1.0)
        flux[k] = absorption_spectrum(lam, continuum, centres[sel], depths[sel], widths[sel])
    return Spectrum(fiber, flux)


def comb_spectra(model: OpticalModel, fiber: int, continuum: float = 2.0e3) -> Spectrum:
    flux = {}
    for s in model.slices:
        if s.fiber == fiber and s.order not in flux:
            lam = bin_centres(s.lambda_lo, s.lambda_hi, s.n_lambda)
            flux[s.order] = fabry_perot_comb(lam, continuum, lam0=3000.0)
    return Spectrum(fiber, flux)


# --------------------------------------------------------------------------
# the named configurations
# --------------------------------------------------------------------------


def config1(seed: Optional[int] = None) -> Workload:
    """Plain method, FP64: one order, one fiber, 1024x256 FP64 frame, 2000 x 16 stamps."""
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    model = echelle_model(
        rng, n_detectors=1, height=256, width=1024, orders_per_detector=1, fibers=1, slices=1,
        degree=3, K=7, n_lambda=2000, n_slit=16, first_order=100, sigma=(1.5, 0.0, 0.0),
    )
    sp = {0: science_spectra(rng, model, 0, n_lines=50)}
    return Workload("cfg1-single-order-fp64", model, sp, "f64", "fp64",
                    "1 order x 1 fiber, 1024x256 FP64, 2000x16 samples, deg 3, sigma 1.5, K=7, 50 lines")


def config2(seed: Optional[int] = None, n_orders: int = 85, n_lambda: int = 6000, n_slit: int = 64,
            n_lines: int = 20000, size: int = 9216) -> Workload:
    """Full single-detector frame, mixed precision: 9216^2 FP32, 85 orders x 2 fibers x 2 slices."""
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    model = echelle_model(
        rng, n_detectors=1, height=size, width=size, orders_per_detector=n_orders, fibers=2, slices=2,
        degree=5, K=11, n_lambda=n_lambda, n_slit=n_slit, first_order=90, sigma_range=(1.2, 2.0),
    )
    sp = {0: science_spectra(rng, model, 0, n_lines=n_lines), 1: comb_spectra(model, 1)}
    return Workload("cfg2-full-detector-mixed", model, sp, "f32", "mixed",
                    f"{n_orders} orders x 2 fibers x 2 slices, {size}^2 FP32, {n_lambda}x{n_slit} samples, "
                    f"deg 5, sigma 1.2-2.0, K=11, science {n_lines} lines + FP comb")


def config3(seed: Optional[int] = None, orders_per_detector: int = 30, n_lambda: int = 8000,
            n_slit: int = 128, size: int = 9216, n_detectors: int = 4) -> Workload:
    """Large multi-detector instrument: 4 x 9216^2, 30 orders/detector x 4 fibers x 2 slices, 13x13 elliptical PSF."""
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    model = echelle_model(
        rng, n_detectors=n_detectors, height=size, width=size, orders_per_detector=orders_per_detector,
        fibers=4, slices=2, degree=5, K=13, n_lambda=n_lambda, n_slit=n_slit, first_order=60,
        sigma_range=(1.2, 2.0), psf=PSF_ELLIPTICAL,
    )
    sp = {f: science_spectra(rng, model, f, n_lines=60000) for f in range(4)}
    return Workload("cfg3-multi-detector-elliptical", model, sp, "f32", "mixed",
                    f"{n_detectors} detectors x {orders_per_detector} orders x 4 fibers x 2 slices, {size}^2 FP32, "
                    f"{n_lambda}x{n_slit} samples, deg 5, K=13 rotated elliptical PSF")


def config5(seed: Optional[int] = None) -> Workload:
    """Differentiation tile: 2048^2 FP32, 10 orders x 1 fiber, 4000 x 32 stamps, degree 4, 9x9 PSF."""
    rng = np.random.default_rng(SEED_BASE + 5 if seed is None else seed)
    model = echelle_model(
        rng, n_detectors=1, height=2048, width=2048, orders_per_detector=10, fibers=1, slices=1,
        degree=4, K=9, n_lambda=4000, n_slit=32, first_order=120, sigma_range=(1.2, 2.0),
    )
    sp = {0: science_spectra(rng, model, 0, n_lines=3000)}
    return Workload("cfg5-differentiation-tile", model, sp, "f32", "mixed",
                    "10 orders x 1 fiber, 2048^2 FP32, 4000x32 samples, deg 4, K=9")


def small_config(seed: int = 7, *, width: int = 300, height: int = 160, orders: int = 2, fibers: int = 2,
                 slices: int = 2, n_lambda: int = 333, n_slit: int = 13, degree: int = 5, K: int = 11,
                 psf: int = PSF_SEPARABLE, out_dtype: str = "f32", precision: str = "mixed",
                 n_detectors: int = 1, trace_pitch: float = 16.0,
                 sigma_range: Tuple[float, float] = (1.2, 2.0)) -> Workload:
    """A small seeded model the oracle renders in well under a second.

    Sizes are deliberately ragged (sample and slit counts that are not multiples of the
    renderer's chunking) and the traces run off the frame edges.
    """
    rng = np.random.default_rng(seed)
    model = echelle_model(
        rng, n_detectors=n_detectors, height=height, width=width, orders_per_detector=orders, fibers=fibers,
        slices=slices, degree=degree, K=K, n_lambda=n_lambda, n_slit=n_slit, first_order=110,
        sigma_range=sigma_range, psf=psf, trace_pitch=trace_pitch,
    )
    sp = {f: science_spectra(rng, model, f, n_lines=40) for f in range(fibers)}
    return Workload(f"small-{seed}", model, sp, out_dtype, precision, "test model")


CONFIGS = {1: config1, 2: config2, 3: config3, 5: config5}


# --------------------------------------------------------------------------
# serving request mix
# --------------------------------------------------------------------------


@dataclass
class JobClass:
    name: str
    make: object  # callable(seed) -> Workload
    share: float


def serving_classes() -> List[JobClass]:
    """Single-order 1024x256 tiles, 10-order 4096^2 tiles and full 9216^2 frames (40/40/20)."""

    def small(seed):
        rng = np.random.default_rng(seed)
        m = echelle_model(rng, n_detectors=1, height=256, width=1024, orders_per_detector=1, fibers=2,
                          slices=2, degree=5, K=11, n_lambda=2000, n_slit=16, first_order=100,
                          sigma_range=(1.2, 2.0))
        sp = {0: science_spectra(rng, m, 0, 50), 1: comb_spectra(m, 1)}
        return Workload("serve-small", m, sp, "f32", "mixed")

    def medium(seed):
        rng = np.random.default_rng(seed)
        m = echelle_model(rng, n_detectors=1, height=4096, width=4096, orders_per_detector=10, fibers=2,
                          slices=2, degree=5, K=11, n_lambda=4000, n_slit=32, first_order=100,
                          sigma_range=(1.2, 2.0))
        sp = {0: science_spectra(rng, m, 0, 2000), 1: comb_spectra(m, 1)}
        return Workload("serve-medium", m, sp, "f32", "mixed")

    def large(seed):
        return config2(seed)

    return [JobClass("small", small, 0.4), JobClass("medium", medium, 0.4), JobClass("large", large, 0.2)]


def poisson_arrivals(rng: np.random.Generator, n: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with ``rate`` jobs per second."""
    return np.cumsum(rng.exponential(1.0 / rate, n))
