"""Pins of the oracle's tabulated-PSF path (PSF maps per field point, Sec. 2.1; each image is
the PSF integrated over the pixels, Sec. 2.2).

The oracle's stamp is the pixel integral of the field-blended maps' bilinear density at the
stamp's exact sub-pixel centre.  These pins check it against things other than itself:

- brute-force quadrature of the bilinear density, evaluated by plain bilinear interpolation of
  the zero-padded samples and integrated exactly by 2-point Gauss-Legendre on every map cell
  (no tent integrals), for random maps, random phases and integer and non-integer sampling;
- the analytic pixel integrals (erf differences) of a sampled Gaussian, at the bilinear
  sampling error and independent of the sub-pixel phase;
- unit mass, symmetry, and the linear blend between field nodes.
"""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W


def _slice(K=11, oversample=10.0, half_px=8.0, seed=601):
    w = W.small_config(seed=seed, K=K, n_lambda=81, n_slit=5, orders=1, fibers=1, slices=1)
    s = w.model.slices[0]
    s.psf_map = W.psf_maps(s, oversample=oversample, half_px=half_px)
    return w, s


def _sig(s, lt):
    return (s.sigma_x[0] + s.sigma_x[1] * lt + s.sigma_x[2] * lt * lt,
            s.sigma_y[0] + s.sigma_y[1] * lt + s.sigma_y[2] * lt * lt)


def _bilinear(S, q, x, y):
    """Plain bilinear interpolation of samples S[v, u] at ((u - c)/q, (v - c)/q), zero outside."""
    M = S.shape[0]
    c = 0.5 * (M - 1)
    P = np.zeros((M + 2, M + 2))
    P[1:-1, 1:-1] = S
    gx, gy = q * x + c + 1.0, q * y + c + 1.0  # positions in the padded grid
    ix = np.clip(np.floor(gx).astype(int), 0, M)
    iy = np.clip(np.floor(gy).astype(int), 0, M)
    tx, ty = gx - ix, gy - iy
    inside = (gx >= 0) & (gx <= M + 1) & (gy >= 0) & (gy <= M + 1)
    v = ((1 - ty) * ((1 - tx) * P[iy, ix] + tx * P[iy, ix + 1]) + ty * ((1 - tx) * P[iy + 1, ix] + tx * P[iy + 1, ix + 1]))
    return np.where(inside, v, 0.0)


def _gl_nodes(a, b, knots):
    """2-point Gauss-Legendre nodes and weights on [a, b] split at the knots inside it: exact for
    piecewise-linear integrands with those knots."""
    cuts = np.concatenate([[a], knots[(knots > a) & (knots < b)], [b]])
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    lo, hi = cuts[:-1, None], cuts[1:, None]
    x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * g
    w = np.broadcast_to(0.5 * (hi - lo), x.shape)
    return x.ravel(), w.ravel()


def _brute_pixel(S, q, a, b, ay, by):
    M = S.shape[0]
    knots = (np.arange(-1, M + 1) - 0.5 * (M - 1)) / q
    x, wx = _gl_nodes(a, b, knots)
    y, wy = _gl_nodes(ay, by, knots)
    return float(wy @ _bilinear(S, q, x[None, :], y[:, None]) @ wx)


def _brute_norm(S, q):
    M = S.shape[0]
    c = 0.5 * (M - 1)
    return _brute_pixel(S, q, (-c - 1) / q, (M - c) / q, (-c - 1) / q, (M - c) / q)


@pytest.mark.parametrize("q,M,K", [(4.0, 29, 7), (2.5, 20, 5), (3.0, 24, 9)])
def test_epsf_equals_brute_force_quadrature_of_the_bilinear_density(q, M, K):
    rng = np.random.default_rng(int(10 * q) + M)
    w, s = _slice(K=K)
    maps = rng.uniform(0.0, 1.0, (2, M, M)) * np.exp(-0.5 * ((np.arange(M) - M / 2) / (M / 5)) ** 2)[None, None, :]
    s.psf_map = W.PsfMap(np.array([-1.0, 1.0]), maps, q)
    H = K // 2
    for f in range(2):
        norm = _brute_norm(maps[f], q)
        for phx, phy in [(0.0, 0.0), (-0.5, 0.31), (0.4999, -0.137), (rng.uniform(-.5, .5), rng.uniform(-.5, .5))]:
            got = oracle.epsf_window(s, f, phx, phy)
            for n in range(K):
                for m in range(K):
                    ax, ay = m - H - 0.5 - phx, n - H - 0.5 - phy
                    ref = _brute_pixel(maps[f], q, ax, ax + 1.0, ay, ay + 1.0) / norm
                    assert got[n, m] == pytest.approx(ref, rel=1e-12, abs=1e-15)
                    if (n + m) % 5 == 0:
                        assert oracle.epsf_pixel(s, f, phx, phy, m, n) == pytest.approx(ref, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("ph", [(0.0, 0.0), (0.2, -0.1), (-0.5, 0.45), (0.37, 0.13)])
def test_epsf_of_a_sampled_gaussian_is_its_pixel_integral(ph):
    from scipy.special import ndtr

    w, s = _slice()
    sx, sy = _sig(s, s.psf_map.field_lt[0])
    H = s.K // 2
    got = oracle.epsf_window(s, 0, ph[0], ph[1])
    m = np.arange(s.K)
    ax = ndtr((m - H + 0.5 - ph[0]) / sx) - ndtr((m - H - 0.5 - ph[0]) / sx)
    ay = ndtr((m - H + 0.5 - ph[1]) / sy) - ndtr((m - H - 0.5 - ph[1]) / sy)
    # the bilinear density of samples 0.1 px apart: the trapezoid rule's O(h^2) error, the same
    # at every sub-pixel phase (no phase tables in the definition)
    assert np.abs(got - np.outer(ay, ax)).max() < 1e-4


def test_epsf_table_has_unit_mass_and_symmetry():
    w, s = _slice(K=15, half_px=7.0)
    e = oracle.epsf_window(s, 2, 0.0, 0.0)
    assert e.sum() == pytest.approx(1.0, abs=1e-12)  # the window covers the whole map
    np.testing.assert_allclose(e, e[::-1, ::-1], rtol=1e-13, atol=1e-17)
    assert e[3, 5] == pytest.approx(oracle.epsf_pixel(s, 2, 0.0, 0.0, 5, 3), rel=1e-14)


def test_table_stamp_is_the_exact_integral_at_the_stamp_centre():
    # n_lambda = 81: the middle sample has lt = 0, a field node of the 5 nodes in [-1, 1]; the
    # others lie between nodes and take the linear blend of the two nodes' integrals
    w, s = _slice(K=9)
    flux = np.ones(s.n_lambda)
    H = s.K // 2
    lt_nodes = s.psf_map.field_lt
    for j, k in [(40, 2), (7, 0), (63, 4), (80, 1)]:
        st, i0, r0 = oracle.stamp(s, flux, j, k, psf=oracle.PSF_TABLE)
        xc, yc, _, _, wt = oracle.map_stamp(s, flux, j, k)
        fx, fy = xc - (i0 + H), yc - (r0 + H)
        assert -0.5 <= fx < 0.5 and -0.5 <= fy < 0.5
        lt = (2 * j + 1 - s.n_lambda) / s.n_lambda
        f0 = int(np.searchsorted(lt_nodes, lt, side="right") - 1)
        f0 = min(max(f0, 0), len(lt_nodes) - 1)
        f1 = min(f0 + 1, len(lt_nodes) - 1)
        t = 0.0 if f1 == f0 else (lt - lt_nodes[f0]) / (lt_nodes[f1] - lt_nodes[f0])
        ref = np.zeros((s.K, s.K))
        for f, wf in [(f0, 1 - t), (f1, t)]:
            if wf == 0:
                continue
            S = s.psf_map.maps[f]
            norm = _brute_norm(S, s.psf_map.oversample)
            for n in range(s.K):
                for m in range(s.K):
                    ax, ay = m - H - 0.5 - fx, n - H - 0.5 - fy
                    ref[n, m] += wf * _brute_pixel(S, s.psf_map.oversample, ax, ax + 1, ay, ay + 1) / norm
        np.testing.assert_allclose(st, wt * ref, rtol=1e-11, atol=1e-15 * wt)
        if j == 40:
            assert t == 0.0


def test_table_render_approximates_the_analytic_psf():
    # constant width: the maps at every node are one Gaussian, so the blend is exact and what
    # remains is the map's sampling error, at every phase the stamps take
    w, s0 = _slice()
    for s in w.model.slices:
        s.sigma_x = [1.5, 0.0, 0.0]
        s.sigma_y = [1.3, 0.0, 0.0]
    wt = W.Workload("t", W.with_psf_maps(w.model, oversample=10.0, half_px=8.0), w.spectra, "f64", "mixed")
    a = oracle.render_workload(wt)[0]
    b = oracle.render_workload(w)[0]
    # trapezoid error of samples h = 0.1 px apart, ~h^2 / (12 sigma^2) of the peak pixel
    assert np.abs(a - b).max() < 5e-4 * np.abs(b).max()
    # field-varying width: the linear blend of two nodes' Gaussians differs from the Gaussian of
    # the blended width by ~(d sigma / sigma)^2 / 8 between nodes 0.5 apart in lt
    w2, _ = _slice()
    wt2 = W.Workload("t", W.with_psf_maps(w2.model, oversample=10.0, half_px=8.0), w2.spectra, "f64", "mixed")
    a2 = oracle.render_workload(wt2)[0]
    b2 = oracle.render_workload(w2)[0]
    assert np.abs(a2 - b2).max() < 5e-3 * np.abs(b2).max()
    assert a2.sum() == pytest.approx(b2.sum(), rel=2e-3)
