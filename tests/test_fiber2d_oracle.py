"""Pins of the oracle's two-dimensional fiber sub-aperture (Sec. 2.2: each image is the fiber's
spatial profile convolved with the PSF; the one-dimensional pseudo-slit is the special case of
one aperture row).  A 2-D fiber's points are (s_k, t_l) with weights u[l n_slit + k], and the
image of row l moves by t_l (ax(lt), ay(lt)).  Checked here against things other than the 2-D
code itself: the 1-D render it must reduce to, a shifted 1-D model for a single row, flux
conservation, and the photocentre of a centred symmetric disk."""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W
from tests.test_oracle_pins import one_slice


def _base(n_slit=6, K=21, sig=1.3, n_lambda=12, degree=2):
    return one_slice(degree=degree, K=K, n_lambda=n_lambda, n_slit=n_slit,
                     cx={(0, 0): 60.2, (1, 0): 20.0, (0, 1): 0.6},
                     cy={(0, 0): 40.3, (0, 1): 4.0, (2, 0): 1.5} if degree >= 2 else {(0, 0): 40.3, (0, 1): 4.0},
                     sx=(sig, 0.05, 0), sy=(sig, -0.04, 0), lam=(6000.0, 6040.0))


def _render(s, flux=None, shape=(80, 120)):
    f = np.linspace(1.0, 2.0, s.n_lambda) if flux is None else flux
    return oracle.render(W.OpticalModel([shape], [s]), lambda _s: f)[0]


def test_one_row_is_the_pseudo_slit():
    s = _base()
    s2 = s.copy()
    s2.n_aper = 1
    s2.aper_x = np.array([3.0, 0.2, 0.1])
    s2.aper_y = np.array([0.4, 0.0, 0.0])
    assert np.array_equal(_render(s), _render(s2))  # t_0 = 0: no displacement at all


@pytest.mark.parametrize("l", [0, 3, 6])
def test_a_single_row_is_the_one_dimensional_model_moved_by_t_l(l):
    n_aper = 7
    s = _base()
    s.n_aper = n_aper
    s.aper_x = np.array([3.2, 0.3, -0.2])  # a quadratic in lt: moves the lt-polynomial's terms
    s.aper_y = np.array([-0.5, 0.1, 0.0])
    u = np.zeros((n_aper, s.n_slit))
    u[l] = np.linspace(0.5, 1.5, s.n_slit)
    s.slit_weights = u.ravel()
    t = -1.0 + (2 * l + 1) / n_aper
    ref = _base()
    ref.slit_weights = u[l].copy()
    for q in range(3):  # x(lt, s) + t ax(lt): the coefficients of lt^q s^0 move by t ax_q
        ref.cx[W.coeff_index(q, 0)] += t * s.aper_x[q]
        ref.cy[W.coeff_index(q, 0)] += t * s.aper_y[q]
    a, b = _render(s), _render(ref)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-14 * np.abs(b).max())
    assert np.abs(b).max() > 0


def test_flux_is_conserved_over_the_aperture():
    s = _base(K=25, sig=0.9)
    s.n_aper = 5
    s.aper_x = np.array([2.5, 0.0, 0.0])
    s.aper_y = np.array([0.3, 0.0, 0.0])
    rng = np.random.default_rng(12)
    s.slit_weights = rng.uniform(0.0, 1.0, 5 * s.n_slit)
    F = 3.25
    frame = _render(s, np.full(s.n_lambda, F), shape=(100, 140))
    assert frame.sum() == pytest.approx(F * (s.lambda_hi - s.lambda_lo) * s.slit_weights.sum(), rel=1e-11)


def test_centred_symmetric_disk_keeps_the_photocentre():
    # one wavelength sample, an affine model and a fiber whose weights are symmetric in s and in
    # t: the photocentre is the mapped centre of (s, t) = (0, 0); the displacement terms cancel
    n_slit, n_aper = 9, 9
    s = one_slice(degree=1, K=31, n_lambda=1, n_slit=n_slit, cx={(0, 0): 60.37, (0, 1): 0.8},
                  cy={(0, 0): 40.61, (0, 1): 4.0}, sx=(1.6, 0, 0), sy=(1.5, 0, 0), lam=(6000.0, 6001.0))
    s.n_aper = n_aper
    s.aper_x = np.array([3.4, 0.0, 0.0])
    s.aper_y = np.array([0.25, 0.0, 0.0])
    sk = (2 * np.arange(n_slit) + 1 - n_slit) / n_slit
    tl = (2 * np.arange(n_aper) + 1 - n_aper) / n_aper
    disk = ((tl[:, None] ** 2 + sk[None, :] ** 2) <= 1.0).astype(float)
    s.slit_weights = (disk / disk.sum()).ravel()
    frame = _render(s, np.array([1.0]), shape=(80, 120))
    ys, xs = np.mgrid[0:80, 0:120]
    tot = frame.sum()
    assert abs((frame * xs).sum() / tot - 60.37) < 1e-9
    assert abs((frame * ys).sum() / tot - 40.61) < 1e-9
    # and the disk's extent shows: the second moment along x grows by the aperture's spread
    var_x = (frame * (xs - 60.37) ** 2).sum() / tot
    spread = float((disk * (tl[:, None] * 3.4 + sk[None, :] * 0.8) ** 2).sum() / disk.sum())
    assert var_x == pytest.approx(1.6 ** 2 + 1.0 / 12.0 + spread, rel=1e-6)
