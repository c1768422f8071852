"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, a brute-force quadrature, a library
routine (numpy / scipy), or an invariant the paper's image model fixes (Sec. 2 and
Sec. 2.2: superposition of pixel-integrated fiber images, normalised illumination
profile times photons).  None of them uses the CUDA path.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2008_05858_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def one_slice(*, degree=1, K=11, n_lambda=5, n_slit=1, cx=None, cy=None, sx=(1.5, 0, 0), sy=(1.5, 0, 0),
              theta=0.0, lam=(5000.0, 5010.0), u=None):
    nc = W.n_coeffs(degree)
    cxa = np.zeros(nc)
    cya = np.zeros(nc)
    for (a, b), v in (cx or {}).items():
        cxa[W.coeff_index(a, b)] = v
    for (a, b), v in (cy or {}).items():
        cya[W.coeff_index(a, b)] = v
    return W.OrderSlice(
        detector=0, order=100, fiber=0, slice=0, degree=degree, K=K, n_lambda=n_lambda, n_slit=n_slit,
        lambda_lo=lam[0], lambda_hi=lam[1], cx=cxa, cy=cya, sigma_x=np.array(sx, float),
        sigma_y=np.array(sy, float), theta=theta,
        slit_weights=np.full(n_slit, 1.0 / n_slit) if u is None else np.asarray(u, float),
    )


def gauss2d_pixel_quadrature(xc, yc, sx, sy, i, r, nodes=16, rho=0.0, gx=None, gy=None):
    """Brute force: tensor Gauss-Legendre (numpy) of the (correlated) Gaussian density over pixel (i, r)."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    x = i + 0.5 * t
    y = r + 0.5 * t
    X, Y = np.meshgrid(x, y, indexing="xy")
    Wt = np.outer(w, w) * 0.25
    if rho == 0.0:
        d = np.exp(-0.5 * ((X - xc) / sx) ** 2) / (sx * math.sqrt(2 * math.pi)) * \
            np.exp(-0.5 * ((Y - yc) / sy) ** 2) / (sy * math.sqrt(2 * math.pi))
    else:
        u = (X - xc) / gx
        v = (Y - yc) / gy
        q = (u * u - 2 * rho * u * v + v * v) / (1 - rho * rho)
        d = np.exp(-0.5 * q) / (2 * math.pi * gx * gy * math.sqrt(1 - rho * rho))
    return float((d * Wt).sum())


# ----------------------------------------------------------------------------- normal interval


def test_normal_interval_matches_scipy_including_tails():
    # P(a<Z<b) against scipy's log-CDF routines (library), relative 1e-13 even 8 sigma out
    rng = np.random.default_rng(1)
    for _ in range(400):
        a = rng.uniform(-9, 9)
        b = a + rng.uniform(0.05, 1.5)
        got = oracle.normal_interval(a, b)
        if a >= 0:
            ref = np.exp(special.log_ndtr(-a)) * -np.expm1(special.log_ndtr(-b) - special.log_ndtr(-a))
        elif b <= 0:
            ref = np.exp(special.log_ndtr(b)) * -np.expm1(special.log_ndtr(a) - special.log_ndtr(b))
        else:
            ref = 1.0 - special.ndtr(a) - special.ndtr(-b)
        assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-300, (a, b, got, ref)


# ----------------------------------------------------------------------------- separable stamp


@pytest.mark.parametrize("xc,yc,sx,sy", [(20.3217, 30.8, 1.5, 1.5), (20.5, 30.0, 1.2, 2.0), (19.9, 31.49, 2.0, 1.3)])
def test_separable_stamp_equals_pixel_quadrature(xc, yc, sx, sy):
    # stamp value = 2-D Gauss-Legendre of the Gaussian density over each pixel (brute force)
    s = one_slice(degree=0, K=7, n_lambda=1, cx={(0, 0): xc}, cy={(0, 0): yc}, sx=(sx, 0, 0), sy=(sy, 0, 0))
    flux = np.array([3.0])
    st, i0, r0 = oracle.stamp(s, flux, 0, 0)
    w = 3.0 * (s.lambda_hi - s.lambda_lo)  # one sample: bin width is the whole order
    assert i0 == math.floor(xc + 0.5) - 3 and r0 == math.floor(yc + 0.5) - 3
    for n in range(7):
        for m in range(7):
            q = w * gauss2d_pixel_quadrature(xc, yc, sx, sy, i0 + m, r0 + n)
            assert abs(st[n, m] - q) <= 1e-12 * q + 1e-300, (n, m, st[n, m], q)


def test_paper_subpixel_sampling_converges_to_exact_integral():
    # Sec. 2.2 samples each pixel on a 0.1 px sub-grid (10 x 10 sub-pixels); the exact erf
    # pixel integral is its h -> 0 limit, approached at O(h^2) (midpoint rule).
    with open(os.path.join(GOLDEN, "sampling_recipe.json")) as f:
        rec = json.load(f)
    nsub = int(round(1.0 / rec["subpixel_step_px"]))
    assert nsub == 10
    xc, yc, sx, sy = 0.23, -0.41, 1.5, 1.5
    for (i, r) in [(0, 0), (1, -1), (3, 2)]:
        exact = oracle.normal_interval((i - 0.5 - xc) / sx, (i + 0.5 - xc) / sx) * \
            oracle.normal_interval((r - 0.5 - yc) / sy, (r + 0.5 - yc) / sy)
        e1 = oracle.subpixel_sample(xc, yc, sx, sy, i, r, nsub) - exact
        e2 = oracle.subpixel_sample(xc, yc, sx, sy, i, r, 2 * nsub) - exact
        e4 = oracle.subpixel_sample(xc, yc, sx, sy, i, r, 4 * nsub) - exact
        assert abs(e1) < 2e-3 * exact
        assert 3.8 < e1 / e2 < 4.2 and 3.8 < e2 / e4 < 4.2  # second order
        extrap = (4 * (exact + e4) - (exact + e2)) / 3
        assert abs(extrap - exact) < 1e-7 * exact


def test_window_rounds_half_up_and_is_centred():
    s = one_slice(degree=0, K=5, n_lambda=1, cx={(0, 0): 50.5}, cy={(0, 0): 20.5})
    _, i0, r0 = oracle.stamp(s, np.array([1.0]), 0, 0)
    assert (i0, r0) == (51 - 2, 21 - 2)
    s = one_slice(degree=0, K=5, n_lambda=1, cx={(0, 0): 50.4999999}, cy={(0, 0): 20.0})
    _, i0, r0 = oracle.stamp(s, np.array([1.0]), 0, 0)
    assert (i0, r0) == (50 - 2, 20 - 2)


def test_truncation_without_renormalisation_closed_form():
    # window K=3 centred at a pixel centre: captured flux = w * (erf(1.5/(sqrt2 sigma)))^2
    s = one_slice(degree=0, K=3, n_lambda=1, cx={(0, 0): 10.0}, cy={(0, 0): 12.0}, sx=(1.3, 0, 0), sy=(0.9, 0, 0))
    st, _, _ = oracle.stamp(s, np.array([1.0]), 0, 0)
    w = s.lambda_hi - s.lambda_lo
    ref = w * special.erf(1.5 / (math.sqrt(2) * 1.3)) * special.erf(1.5 / (math.sqrt(2) * 0.9))
    assert abs(st.sum() - ref) < 1e-13 * ref


def test_photocenter_of_symmetric_psf_is_the_mapped_position():
    # wide window: the pixel-integrated stamp's centroid equals (x_c, y_c).  The pixel grid
    # aliases the centroid by ~exp(-2 pi^2 sigma^2), so sigma must be >~1.2 for 1e-12; the
    # window must be wide enough that truncation is below that too (K=31 here).
    xc, yc = 40.3217, 25.6604
    s = one_slice(degree=0, K=31, n_lambda=1, cx={(0, 0): xc}, cy={(0, 0): yc}, sx=(1.6, 0, 0), sy=(1.5, 0, 0))
    st, i0, r0 = oracle.stamp(s, np.array([1.0]), 0, 0)
    ys, xs = np.mgrid[r0:r0 + 31, i0:i0 + 31]
    assert abs((st * xs).sum() / st.sum() - xc) < 1e-12
    assert abs((st * ys).sum() / st.sum() - yc) < 1e-12
    # any K, centre on a pixel centre: exactly symmetric window
    s = one_slice(degree=0, K=5, n_lambda=1, cx={(0, 0): 40.0}, cy={(0, 0): 25.0}, sx=(1.7, 0, 0), sy=(1.4, 0, 0))
    st, i0, r0 = oracle.stamp(s, np.array([1.0]), 0, 0)
    ys, xs = np.mgrid[r0:r0 + 5, i0:i0 + 5]
    assert abs((st * xs).sum() / st.sum() - 40.0) < 1e-13
    assert abs((st * ys).sum() / st.sum() - 25.0) < 1e-13


def test_second_moment_is_sigma_squared_plus_sheppard():
    # a pixelised Gaussian with sigma >= 1 has discrete variance sigma^2 + 1/12 (Sheppard's
    # correction; the error is ~exp(-2 pi^2 sigma^2)).  Pins the width polynomial in lt and
    # that sigma is a standard deviation (not FWHM or variance).
    s = one_slice(degree=1, K=31, n_lambda=9, cx={(0, 0): 50.3, (1, 0): 20.0}, cy={(0, 0): 30.1},
                  sx=(1.4, 0.2, -0.1), sy=(1.1, -0.1, 0.05))
    flux = np.ones(9)
    for j, lt in [(4, 0.0), (8, 8.0 / 9.0), (0, -8.0 / 9.0)]:
        st, i0, r0 = oracle.stamp(s, flux, j, 0)
        ys, xs = np.mgrid[r0:r0 + 31, i0:i0 + 31]
        tot = st.sum()
        mx = (st * xs).sum() / tot
        my = (st * ys).sum() / tot
        vx = (st * (xs - mx) ** 2).sum() / tot
        vy = (st * (ys - my) ** 2).sum() / tot
        sxv = 1.4 + 0.2 * lt - 0.1 * lt * lt
        syv = 1.1 - 0.1 * lt + 0.05 * lt * lt
        assert abs(vx - (sxv ** 2 + 1 / 12)) < 1e-8
        assert abs(vy - (syv ** 2 + 1 / 12)) < 1e-8


# ----------------------------------------------------------------------------- mapping


def test_sampling_grid_is_bin_centred_and_symmetric():
    # affine trace x = 100 + 40 lt + 2 s: the middle sample of an odd grid sits at lt = 0,
    # samples are symmetric about it and 2/N apart; slit points likewise in s.
    N, Ns = 7, 5
    s = one_slice(degree=1, K=7, n_lambda=N, n_slit=Ns, cx={(0, 0): 100.0, (1, 0): 40.0, (0, 1): 2.0},
                  cy={(0, 0): 50.0, (0, 1): 3.0})
    flux = np.ones(N)
    x_mid, y_mid, *_ = oracle.map_stamp(s, flux, N // 2, Ns // 2)
    assert x_mid == pytest.approx(100.0, abs=1e-12) and y_mid == pytest.approx(50.0, abs=1e-12)
    xs = [oracle.map_stamp(s, flux, j, Ns // 2)[0] for j in range(N)]
    assert np.allclose(np.diff(xs), 40.0 * 2.0 / N, atol=1e-11)
    assert xs[0] + xs[-1] == pytest.approx(200.0, abs=1e-11)
    ys = [oracle.map_stamp(s, flux, N // 2, k)[1] for k in range(Ns)]
    assert np.allclose(np.diff(ys), 3.0 * 2.0 / Ns, atol=1e-11)
    assert ys[0] == pytest.approx(50.0 - 3.0 * (1 - 1.0 / Ns), abs=1e-11)


@pytest.mark.parametrize("a,b", [(a, b) for t in range(4) for b in range(t + 1) for a in [t - b]])
def test_coefficient_order_total_degree_then_a_descending(a, b):
    # one unit coefficient in slot index(a,b) must place x_c at lt^a s^b (+ offset)
    N, Ns = 3, 3
    s = one_slice(degree=3, K=7, n_lambda=N, n_slit=Ns, cx={(0, 0): 100.0}, cy={(0, 0): 50.0})
    s.cx[W.coeff_index(a, b)] += 1.0
    lt_vals = [-2 / 3, 0.0, 2 / 3]
    for j in range(N):
        for k in range(Ns):
            x, y, *_ = oracle.map_stamp(s, np.ones(N), j, k)
            expect = 100.0 + lt_vals[j] ** a * lt_vals[k] ** b
            assert x == pytest.approx(expect, abs=1e-12), (a, b, j, k)
            assert y == pytest.approx(50.0, abs=1e-12)
    # the index formula itself: ordered by total degree, a descending
    order = [(t - bb, bb) for t in range(4) for bb in range(t + 1)]
    assert W.coeff_index(a, b) == order.index((a, b))


# ----------------------------------------------------------------------------- frame invariants


def _single_trace_model(K=15, sig=0.8, n_lambda=64, n_slit=8, width=200, height=60, degree=2):
    s = one_slice(degree=degree, K=K, n_lambda=n_lambda, n_slit=n_slit,
                  cx={(0, 0): width / 2, (1, 0): 0.3 * width, (0, 1): 0.7},
                  cy={(0, 0): height / 2, (0, 1): 4.0, (2, 0): 3.0} if degree >= 2 else {(0, 0): height / 2, (0, 1): 4.0},
                  sx=(sig, 0, 0), sy=(sig, 0, 0), lam=(6000.0, 6040.0))
    return W.OpticalModel([(height, width)], [s])


def test_flux_conservation_constant_spectrum():
    # every photon lands on the frame: sum I = F * (lambda_hi - lambda_lo) * sum(u)
    m = _single_trace_model()
    F = 7.5
    frame = oracle.render(m, lambda s: np.full(s.n_lambda, F))[0]
    s = m.slices[0]
    assert frame.sum() == pytest.approx(F * (s.lambda_hi - s.lambda_lo) * s.slit_weights.sum(), rel=1e-12)


def test_superposition_is_linear_in_the_spectrum():
    m = _single_trace_model(K=7, sig=1.5)
    rng = np.random.default_rng(3)
    f1 = rng.uniform(0.5, 2.0, m.slices[0].n_lambda)
    f2 = rng.uniform(0.0, 3.0, m.slices[0].n_lambda)
    a, b = 1.7, -0.3
    I1 = oracle.render(m, lambda s: f1)[0]
    I2 = oracle.render(m, lambda s: f2)[0]
    I12 = oracle.render(m, lambda s: a * f1 + b * f2)[0]
    assert np.allclose(I12, a * I1 + b * I2, rtol=1e-12, atol=1e-12 * np.abs(I12).max())


def test_pixels_outside_the_frame_are_dropped_not_wrapped():
    # trace runs off the left edge: in-frame flux equals the sum of the in-frame stamp pixels
    s = one_slice(degree=1, K=7, n_lambda=20, n_slit=2, cx={(0, 0): 2.0, (1, 0): 10.0}, cy={(0, 0): 15.0},
                  sx=(1.5, 0, 0), sy=(1.5, 0, 0))
    m = W.OpticalModel([(30, 40)], [s])
    flux = np.linspace(1, 2, 20)
    frame = oracle.render(m, lambda _s: flux)[0]
    tot = 0.0
    for j in range(20):
        for k in range(2):
            st, i0, r0 = oracle.stamp(s, flux, j, k)
            for n in range(7):
                for mm in range(7):
                    if 0 <= i0 + mm < 40 and 0 <= r0 + n < 30:
                        tot += st[n, mm]
    assert frame.sum() == pytest.approx(tot, rel=1e-13)
    assert frame[:, -3:].sum() == 0.0  # nothing wrapped to the right edge


def test_render_does_not_depend_on_thread_count():
    w = W.small_config(seed=11)
    a = oracle.render_workload(w, n_threads=1)[0]
    b = oracle.render_workload(w, n_threads=4)[0]
    assert np.array_equal(a, b)


# ----------------------------------------------------------------------------- elliptical PSF


def test_gauss_legendre_nodes_match_numpy():
    for n in [1, 2, 3, 5, 8, 13, 20, 24]:
        x, w = oracle.gauss_legendre(n)
        o = np.argsort(x)
        xn, wn = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x[o], xn, atol=2e-15) and np.allclose(w[o], wn, atol=2e-14)


def test_bvn_cdf_closed_forms():
    # rho = 0: product of marginals; h = k = 0: 1/4 + asin(rho)/(2 pi) (Sheppard);
    # rho -> symmetric: F(h,k,rho) = F(k,h,rho)
    for rho in [-0.9, -0.5, -0.1, 0.2, 0.6, 0.9]:
        assert oracle.bvn_cdf(0.0, 0.0, rho) == pytest.approx(0.25 + math.asin(rho) / (2 * math.pi), abs=1e-15)
    for h, k in [(-1.2, 0.4), (2.0, -3.0), (-5.0, -4.5)]:
        assert oracle.bvn_cdf(h, k, 0.0) == pytest.approx(special.ndtr(h) * special.ndtr(k), rel=1e-14)
        assert oracle.bvn_cdf(h, k, 0.37) == pytest.approx(oracle.bvn_cdf(k, h, 0.37), rel=1e-13)


def test_bvn_cdf_matches_scipy():
    mvn = stats.multivariate_normal
    for h, k, rho in [(-1.0, 0.5, 0.3), (0.7, 1.2, -0.6), (-2.0, -1.5, 0.8), (1.5, -0.3, 0.1)]:
        ref = mvn(mean=[0, 0], cov=[[1, rho], [rho, 1]]).cdf([h, k])
        assert oracle.bvn_cdf(h, k, rho) == pytest.approx(ref, abs=2e-6)


@pytest.mark.parametrize("rho", [0.0, 0.15, -0.3, 0.6])
def test_bvn_rectangles_equal_brute_force_quadrature(rho):
    gx, gy = 1.7, 1.3
    xc, yc = 0.31, -0.22
    for (i, r) in [(0, 0), (1, 0), (-2, 1), (3, -2), (5, 4), (-5, -5)]:
        h0, h1 = (i - 0.5 - xc) / gx, (i + 0.5 - xc) / gx
        k0, k1 = (r - 0.5 - yc) / gy, (r + 0.5 - yc) / gy
        got = oracle.bvn_rect(h0, h1, k0, k1, rho)
        ref = gauss2d_pixel_quadrature(xc, yc, gx, gy, i, r, nodes=24, rho=rho, gx=gx, gy=gy)
        assert abs(got - ref) <= 1e-11 * ref, (i, r, got, ref)


def test_elliptical_reduces_to_separable_at_theta_zero_and_swaps_at_90():
    base = dict(degree=0, K=9, n_lambda=1, cx={(0, 0): 30.37}, cy={(0, 0): 20.81}, sx=(1.8, 0, 0), sy=(1.25, 0, 0))
    sep, _, _ = oracle.stamp(one_slice(**base), np.array([1.0]), 0, 0, psf=oracle.PSF_SEPARABLE)
    ell, _, _ = oracle.stamp(one_slice(**base, theta=0.0), np.array([1.0]), 0, 0, psf=oracle.PSF_ELLIPTICAL)
    assert np.allclose(ell, sep, rtol=1e-13, atol=1e-300)
    b90 = dict(base, sx=(1.25, 0, 0), sy=(1.8, 0, 0))
    swapped, _, _ = oracle.stamp(one_slice(**b90), np.array([1.0]), 0, 0, psf=oracle.PSF_SEPARABLE)
    ell90, _, _ = oracle.stamp(one_slice(**base, theta=math.pi / 2), np.array([1.0]), 0, 0, psf=oracle.PSF_ELLIPTICAL)
    assert np.allclose(ell90, swapped, rtol=1e-12, atol=1e-18)


def test_elliptical_stamp_moments_follow_the_rotated_covariance():
    # wide window: second moments of the pixelised stamp = rotated covariance + 1/12 on the diagonal
    sa, sb, th = 1.6, 1.1, math.radians(8.0)
    s = one_slice(degree=0, K=31, n_lambda=1, cx={(0, 0): 30.2}, cy={(0, 0): 20.7}, sx=(sa, 0, 0), sy=(sb, 0, 0),
                  theta=th)
    st, i0, r0 = oracle.stamp(s, np.array([1.0]), 0, 0, psf=oracle.PSF_ELLIPTICAL)
    ys, xs = np.mgrid[r0:r0 + 31, i0:i0 + 31]
    t = st.sum()
    mx, my = (st * xs).sum() / t, (st * ys).sum() / t
    vxx = (st * (xs - mx) ** 2).sum() / t
    vyy = (st * (ys - my) ** 2).sum() / t
    vxy = (st * (xs - mx) * (ys - my)).sum() / t
    c, sn = math.cos(th), math.sin(th)
    assert vxx == pytest.approx(sa * sa * c * c + sb * sb * sn * sn + 1 / 12, abs=1e-6)
    assert vyy == pytest.approx(sa * sa * sn * sn + sb * sb * c * c + 1 / 12, abs=1e-6)
    assert vxy == pytest.approx((sa * sa - sb * sb) * sn * c, abs=1e-6)
    assert mx == pytest.approx(30.2, abs=1e-9) and my == pytest.approx(20.7, abs=1e-9)


# ----------------------------------------------------------------------------- gradient


def test_loss_gradient_matches_central_differences():
    w = W.small_config(seed=5, width=120, height=70, orders=1, fibers=1, slices=2, n_lambda=40, n_slit=5,
                       degree=3, K=9)
    m = w.model
    target = [f * 0.97 + 0.01 for f in oracle.render_workload(w)]
    L0, gcx, gcy, gsx, gsy = oracle.loss_grad(m, w.flux_for, target)

    def loss(model):
        fr = oracle.render(model, w.flux_for)
        return sum(float(((a - b) ** 2).sum()) for a, b in zip(fr, target))

    assert L0 == pytest.approx(loss(m), rel=1e-12)
    nc = W.n_coeffs(3)
    checks = [("cx", 0, 0), ("cx", 0, 1), ("cx", 1, 4), ("cy", 0, 2), ("cy", 1, 0), ("sx", 0, 0), ("sy", 1, 2)]
    for name, i, c in checks:
        h = 1e-5
        mp, mm = m.copy(), m.copy()
        arr_p = {"cx": mp.slices[i].cx, "cy": mp.slices[i].cy, "sx": mp.slices[i].sigma_x, "sy": mp.slices[i].sigma_y}[name]
        arr_m = {"cx": mm.slices[i].cx, "cy": mm.slices[i].cy, "sx": mm.slices[i].sigma_x, "sy": mm.slices[i].sigma_y}[name]
        arr_p[c] += h
        arr_m[c] -= h
        fd = (loss(mp) - loss(mm)) / (2 * h)
        g = gcx[i * nc + c] if name == "cx" else gcy[i * nc + c] if name == "cy" else \
            gsx[3 * i + c] if name == "sx" else gsy[3 * i + c]
        assert g == pytest.approx(fd, rel=2e-5, abs=1e-6 * abs(L0)), (name, i, c, g, fd)


def test_accuracy_requirement_golden_is_self_consistent():
    # Sec. 2.2: at R = 1e5 and 3 px per resolution element, 1 cm/s is ~1e-5 px
    with open(os.path.join(GOLDEN, "accuracy_requirement.json")) as f:
        g = json.load(f)
    px = g["resolving_power"] * g["pixels_per_resolution_element"] * g["velocity_cm_s"] * 1e-2 / 299792458.0
    assert px == pytest.approx(g["photocenter_shift_px"], rel=0.05)


@pytest.mark.parametrize("n", [0.75, 1.0, 1.25])
def test_flat_field_aliasing_matches_poisson_summation(n):
    # A flat field sampled n times per FWHM ripples with amplitude 2|P(1/h)| / P(0),
    # P(f) = exp(-2 pi^2 sigma^2 f^2) sinc(f) (Poisson summation over the sample comb; the
    # pixel box gives the sinc): written here from the Fourier transforms, not the oracle's
    # erf stamps.
    import math

    from paper_2008_05858_gb300 import aliasing as A

    w = A.flat_field(n)
    h = A.sample_spacing(w)
    f = 1.0 / h
    want = 2.0 * math.exp(-2.0 * math.pi ** 2 * 1.5 ** 2 * f * f) * abs(math.sin(math.pi * f) / (math.pi * f))
    got = A.measured_ripple(oracle.render_workload(w)[0], w)["ripple"]
    assert got == pytest.approx(want, rel=2e-3)


def test_ten_samples_per_resolution_element_alias_below_photon_noise():
    # the sampling the paper settles on (Sec. 2.2, Fig. 4): ~10 wavelength samples per
    # resolution element keep the aliasing under the photon noise of a ~40000 e-/px flat field
    from paper_2008_05858_gb300 import aliasing as A

    w = A.flat_field(10.0, peak_e=40000.0)
    r = A.measured_ripple(oracle.render_workload(w)[0], w)
    assert r["ripple"] < 1e-3 * r["photon_noise_peak_pixel"]
    w1 = A.flat_field(1.0, peak_e=40000.0)
    r1 = A.measured_ripple(oracle.render_workload(w1)[0], w1)
    assert r1["ripple"] > r1["photon_noise_peak_pixel"]  # one sample per FWHM is not enough


def _blazed(seed=501, m=110.0):
    w = W.small_config(seed=seed, orders=2)
    for s in w.model.slices:
        s.blaze_order = m
        s.blaze_lambda = 0.5 * (s.lambda_lo + s.lambda_hi) * (1.0 + 0.3 / m)  # off-centre peak
    return w


def test_blaze_is_a_weight_multiplier_with_the_grating_envelope():
    # Blaze (Sec. 4.2: each order weighted by its grating blaze profile): B = sinc^2(nu),
    # nu = m (1 - lambda_b / lambda).  The blazed render must equal the unblazed render of the
    # spectrum multiplied by B at the bin centres; B is 1 at lambda_b and 0 at nu = +-1.
    w = _blazed()
    plain = w.model.copy()
    for s in plain.slices:
        s.blaze_order = 0.0

    def blaze(s, lam):
        nu = s.blaze_order * (1.0 - s.blaze_lambda / lam)
        return np.sinc(nu) ** 2

    blazed_of = {id(p): q for p, q in zip(plain.slices, w.model.slices)}

    def flux_b(s):
        lam = s.lambda_lo + (np.arange(s.n_lambda) + 0.5) * (s.lambda_hi - s.lambda_lo) / s.n_lambda
        return w.flux_for(s) * blaze(blazed_of[id(s)], lam)

    a = oracle.render(w.model, w.flux_for)[0]
    b = oracle.render(plain, flux_b)[0]
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15 * np.abs(b).max())
    s = w.model.slices[0]
    assert blaze(s, s.blaze_lambda) == 1.0
    assert abs(blaze(s, s.blaze_lambda / (1.0 - 1.0 / s.blaze_order))) < 1e-25


def test_window_ties_and_flip_reporting():
    # Window rule ties (a centre within rounding of a pixel edge may round either way): the
    # oracle lists exactly the stamps a direct scan of the mapped centres finds, and the frame
    # comparator counts failing pixels inside a tie's boxes as flips, not as failures.
    from tests import framecompare as F

    w = W.small_config(seed=3, n_lambda=120, n_slit=7)
    margin = 2e-3
    ties = oracle.window_ties(w.model, w.flux_for, margin)
    want = []
    for i, s in enumerate(w.model.slices):
        f = w.flux_for(s)
        for j in range(s.n_lambda):
            for k in range(s.n_slit):
                c = oracle.map_stamp(s, f, j, k)[:2]
                for a in (0, 1):
                    d = (c[a] + 0.5) - np.floor(c[a] + 0.5)
                    if d < margin or 1 - d < margin:
                        want.append((i, s.detector, j, k, a))
    assert sorted(ties) == sorted(want) and len(want) > 0
    boxes = F.tie_boxes(w.model, w.flux_for, margin)[0]
    ref = oracle.render_workload(w)[0]
    x0, x1, y0, y1 = boxes[0]
    g = ref.copy()
    g[min(max(y0, 0) + 3, ref.shape[0] - 1), min(max(x0, 0) + 3, ref.shape[1] - 1)] *= 1.001
    rep = F.compare(g, ref, ties=boxes)
    assert rep.ok and rep.n_flip_px == 1 and rep.n_bad == 0 and rep.n_ties == len(boxes)
    rep = F.compare(g, ref)
    assert not rep.ok and rep.n_bad == 1
