"""GPU renderer vs the FP64 oracle, element by element, through the C ABI.

Tolerance (the renderer's fidelity target): relative per-pixel error below 1e-6 (with an
absolute floor of 1e-10 of the frame peak, see framecompare) and photocenter shifts of
16x16 px windows below 1e-5 px.  The plain FP64 renderer must agree to 5e-11 relative:
CUDA's FP64 erfc and glibc's differ by a few ulp, and the same-side tail differences of a
pixel integral amplify that by up to ~10 (measured worst 8.5e-12).
"""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W
from tests.framecompare import compare, tie_boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_ORACLE = {}
FP64_REL = 5e-11


def oracle_frames(w):
    key = id(w)
    if key not in _ORACLE or _ORACLE[key][0] is not w:
        _ORACLE[key] = (w, oracle.render_workload(w))  # keep w alive so its id is not reused
    return _ORACLE[key][1]


@pytest.fixture(scope="module")
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def gpu_frames(r, w, precision, dtype):
    mid = r.load_model(w.model)
    sids = r.load_spectra(w)
    out = r.render(mid, sids, precision, dtype)
    torch.cuda.synchronize()
    res = [t.double().cpu().numpy() for t in out]
    for s in sids:
        from paper_2008_05858_gb300.binding import e2e_unload_spectrum

        e2e_unload_spectrum(r.ctx, s)
    r.unload_model(mid)
    return res


SMALL = [
    dict(seed=7),
    dict(seed=8, K=7, degree=3, n_lambda=257, n_slit=16),
    dict(seed=9, K=9, degree=4, n_lambda=100, n_slit=33, width=180, height=120),
    dict(seed=10, K=5, degree=2, n_lambda=1000, n_slit=3, orders=3),
    dict(seed=11, K=13, degree=5, n_lambda=77, n_slit=64),
    dict(seed=12, K=3, degree=1, n_lambda=64, n_slit=5),
    dict(seed=13, K=1, degree=0, n_lambda=31, n_slit=2),
    dict(seed=14, K=15, degree=5, n_lambda=60, n_slit=7, width=400, height=200),
    dict(seed=15, K=11, degree=5, n_lambda=2000, n_slit=128, orders=1, fibers=1, slices=1, width=512, height=64),
    dict(seed=16, K=15, degree=8, n_lambda=150, n_slit=20),  # the largest window and degree accepted
    # PSFs up to 3 px wide: the tail edges' arguments fall below the cheaper rational's fit, so
    # the plan keeps the general rational there (every case above with K >= 3 takes the cheaper one)
    dict(seed=17, K=15, degree=4, n_lambda=120, n_slit=9, sigma_range=(2.2, 3.0)),
    dict(seed=18, K=5, degree=3, n_lambda=200, n_slit=6, sigma_range=(1.8, 2.6)),
]


@pytest.mark.parametrize("kw", SMALL, ids=[f"s{k['seed']}" for k in SMALL])
def test_mixed_matches_oracle_small(renderer, kw):
    w = W.small_config(**kw)
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "mixed", "f32")
    ties = tie_boxes(w.model, w.flux_for)  # window flips are reported, not hidden in the bound
    for d, (g, o) in enumerate(zip(got, ref)):
        rep = compare(g, o, ties=ties[d])
        print(f"detector {d}: {rep}")
        assert rep.ok, str(rep)


@pytest.mark.parametrize("kw", SMALL[:4], ids=[f"s{k['seed']}" for k in SMALL[:4]])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_fp64_matches_oracle_small(renderer, kw, dtype):
    w = W.small_config(**kw)
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "fp64", dtype)
    for g, o in zip(got, ref):
        if dtype == "f64":
            peak = np.abs(o).max()
            assert np.all(np.abs(g - o) <= FP64_REL * np.abs(o) + 1e-15 * peak)
        else:
            assert compare(g, o, rel=1.2e-7, floor=1e-12).ok


def test_mixed_f64_output_matches_oracle(renderer):
    w = W.small_config(seed=21)
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "mixed", "f64")
    assert compare(got[0], ref[0]).ok


def test_config1_fp64_full(renderer):
    w = W.config1()
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "fp64", "f64")
    peak = np.abs(ref[0]).max()
    assert np.all(np.abs(got[0] - ref[0]) <= FP64_REL * np.abs(ref[0]) + 1e-15 * peak)
    assert compare(gpu_frames(renderer, w, "mixed", "f64")[0], ref[0]).ok


def test_config5_mixed_full(renderer):
    w = W.config5()
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "mixed", "f32")
    rep = compare(got[0], ref[0], ties=tie_boxes(w.model, w.flux_for)[0])
    print(rep)
    assert rep.ok, str(rep)


def test_config2_reduced_orders(renderer):
    w = W.config2(n_orders=6, size=9216)
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "mixed", "f32")
    rep = compare(got[0], ref[0], ties=tie_boxes(w.model, w.flux_for)[0])
    print(rep)
    assert rep.ok, str(rep)


def test_multi_detector_and_empty_detector(renderer):
    w = W.small_config(seed=31, n_detectors=3)
    # detector 2 gets no slices at all: must come back all zeros
    w.model.slices = [s for s in w.model.slices if s.detector != 2]
    ref = oracle_frames(w)
    got = gpu_frames(renderer, w, "mixed", "f32")
    for g, o in zip(got, ref):
        assert compare(g, o).ok
    assert not got[2].any()


def test_model_without_slices_renders_zeros(renderer):
    m = W.OpticalModel([(40, 50)], [])
    mid = renderer.load_model(m)
    # prefilled: every pixel must be written (the merge writes the empty tiles as zeros)
    out = renderer.render(mid, [], "mixed", "f32", out=[torch.full((40, 50), 5.0, device="cuda:0")])
    torch.cuda.synchronize()
    assert not out[0].any().item()
    renderer.unload_model(mid)


def test_trace_entirely_off_frame(renderer):
    w = W.small_config(seed=41)
    for s in w.model.slices:
        s.cy[0] += 10000.0
    got = gpu_frames(renderer, w, "mixed", "f32")
    assert not np.any(got[0])


def test_pitched_destination(renderer):
    w = W.small_config(seed=51)
    ref = oracle_frames(w)[0]
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    h, wd = w.model.det_shape[0]
    big = torch.full((h, wd + 37), -1.0, dtype=torch.float32, device="cuda")
    view = big[:, :wd]
    renderer.render(mid, sids, "mixed", "f32", out=[view])
    torch.cuda.synchronize()
    assert compare(view.double().cpu().numpy(), ref).ok
    assert torch.all(big[:, wd:] == -1.0).item()


def test_render_is_deterministic(renderer):
    w = W.small_config(seed=61, n_lambda=500, n_slit=32)
    a = gpu_frames(renderer, w, "mixed", "f32")[0]
    b = gpu_frames(renderer, w, "mixed", "f32")[0]
    assert np.array_equal(a, b)


def test_linearity_in_the_spectrum(renderer):
    w = W.small_config(seed=71)
    w2 = W.small_config(seed=71)
    for f in w2.spectra:
        for o in w2.spectra[f].flux:
            w2.spectra[f].flux[o] = w2.spectra[f].flux[o] * 2.5
    a = gpu_frames(renderer, w, "mixed", "f64")[0]
    b = gpu_frames(renderer, w2, "mixed", "f64")[0]
    assert np.allclose(b, 2.5 * a, rtol=2e-6, atol=1e-10 * np.abs(b).max())


def _scaled(seed, fn):
    w = W.small_config(seed=seed, n_lambda=300, n_slit=17)
    for f in w.spectra:
        for o in w.spectra[f].flux:
            w.spectra[f].flux[o] = fn(f, o, np.asarray(w.spectra[f].flux[o], dtype=np.float64))
    return w


@pytest.mark.parametrize("scale", [1e-15, 1e15], ids=["1e-15", "1e15"])
def test_flux_far_from_unity(renderer, scale):
    """Each item's fixed-point scale follows its own flux bound: a spectrum at 1e-15 or 1e15
    renders to the same relative accuracy as one near 1."""
    w = _scaled(91, lambda f, o, x: x * scale)
    for dtype in ("f32", "f64"):
        g = gpu_frames(renderer, w, "mixed", dtype)
        ref = oracle_frames(w)
        for a, b in zip(g, ref):
            rep = compare(a, b)
            assert rep.ok, f"{dtype}: {rep}"


def test_fibers_six_decades_apart(renderer):
    """A bright fiber (x1e3) beside a faint one (x1e-3): the faint trace's pixels, 1e-6 of the
    frame's peak, keep the per-pixel relative accuracy (per-item scales, compensated merge)."""
    w = _scaled(92, lambda f, o, x: x * (1e3 if f == 0 else 1e-3))
    g = gpu_frames(renderer, w, "mixed", "f32")
    ref = oracle_frames(w)
    bright = _scaled(92, lambda f, o, x: x * (1e3 if f == 0 else 0.0))
    ref_bright = oracle.render_workload(bright)
    for a, b, bb in zip(g, ref, ref_bright):
        rep = compare(a, b)
        assert rep.ok, str(rep)
        # the faint trace's pixels that no bright stamp reaches, down to 1e-4 of the faint
        # fiber's peak (1e-10 of the frame's), keep the relative bound without its floor
        faint_peak = np.abs(np.where(bb == 0, b, 0)).max()
        sel = (bb == 0) & (np.abs(b) > 1e-4 * faint_peak)
        assert sel.sum() > 100 and faint_peak < 1e-5 * np.abs(b).max()
        assert np.all(np.abs(a[sel] - b[sel]) <= 1e-6 * np.abs(b[sel])), float(
            np.max(np.abs(a[sel] - b[sel]) / np.abs(b[sel])))


def test_signed_spectrum(renderer):
    """A spectrum of both signs (a continuum-subtracted template): the fixed-point words are
    signed, and the error is bounded by the relative bound applied to the render of |flux|
    (cancelling contributions cannot be more accurate than their parts)."""
    rng = np.random.default_rng(93)
    signs = {}

    def signed(f, o, x):
        signs[(f, o)] = rng.choice([-1.0, 1.0], size=x.shape)
        return x * signs[(f, o)]

    w = _scaled(93, signed)
    w_abs = _scaled(93, lambda f, o, x: x)
    g = gpu_frames(renderer, w, "mixed", "f64")
    ref = oracle_frames(w)
    ref_abs = oracle.render_workload(w_abs)
    for a, b, babs in zip(g, ref, ref_abs):
        assert np.any(b < 0) and np.any(b > 0)
        err = np.abs(a - b)
        assert np.all(err <= 1e-6 * np.abs(babs) + 1e-10 * np.abs(babs).max()), float(
            np.max(err / (np.abs(babs) + 1e-300)))


@pytest.mark.parametrize("mutate,msg", [
    (lambda s: setattr(s, "K", 8), "odd"),
    (lambda s: s.cx.__setitem__(1, float("nan")), "non-finite"),
    (lambda s: setattr(s, "sigma_x", np.array([-0.5, 0.0, 0.0])), "width"),
    (lambda s: setattr(s, "degree", 9), "degree"),
])
def test_invalid_models_are_rejected(renderer, mutate, msg):
    from paper_2008_05858_gb300.binding import E2EError, E2E_EINVAL

    w = W.small_config(seed=81)
    mutate(w.model.slices[0])
    with pytest.raises(E2EError) as e:
        renderer.load_model(w.model)
    assert e.value.code == E2E_EINVAL and msg in str(e.value)


def test_spectrum_length_mismatch_is_rejected(renderer):
    from paper_2008_05858_gb300.binding import E2EError, E2E_EINVAL

    w = W.small_config(seed=82)
    mid = renderer.load_model(w.model)
    bad = W.Spectrum(0, {o: f[:-1] for o, f in w.spectra[0].flux.items()})
    sids = [renderer.load_spectrum(bad), renderer.load_spectrum(w.spectra[1])]
    with pytest.raises(E2EError) as e:
        renderer.render(mid, sids, "mixed", "f32")
    assert e.value.code == E2E_EINVAL
    renderer.unload_model(mid)


@pytest.mark.parametrize("bad_value", [float("nan"), float("inf"), -float("inf")], ids=["nan", "inf", "-inf"])
@pytest.mark.parametrize("where", ["first", "last", "middle"])
def test_non_finite_flux_is_rejected(renderer, bad_value, where):
    # the upload is checked on the device: a single bad sample anywhere refuses the spectrum,
    # and a good spectrum still loads and renders afterwards
    from paper_2008_05858_gb300.binding import E2EError, E2E_EINVAL

    w = W.small_config(seed=83)
    orders = sorted(w.spectra[0].flux)
    flux = {o: np.array(w.spectra[0].flux[o], dtype=np.float64) for o in orders}
    cat = np.concatenate([flux[o] for o in orders])
    cat[{"first": 0, "last": len(cat) - 1, "middle": len(cat) // 2 + 1}[where]] = bad_value
    off = 0
    for o in orders:
        n = len(flux[o])
        flux[o] = cat[off:off + n]
        off += n
    with pytest.raises(E2EError) as e:
        renderer.load_spectrum(W.Spectrum(0, flux))
    assert e.value.code == E2E_EINVAL and "non-finite" in str(e.value)
    ref = oracle_frames(w)
    assert compare(gpu_frames(renderer, w, "mixed", "f32")[0], ref[0]).ok


def test_render_alloc_and_fetch(renderer):
    from paper_2008_05858_gb300 import binding as B

    w = W.small_config(seed=91)
    ref = oracle_frames(w)[0]
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    fid = B.e2e_render_alloc(renderer.ctx, mid, sids, B.E2E_PREC_MIXED, B.E2E_F32)
    h, wd = w.model.det_shape[0]
    host = np.zeros((h, wd), dtype=np.float32)
    B.e2e_fetch_frame(renderer.ctx, fid, 0, host.ctypes.data, False, host.nbytes)
    torch.cuda.synchronize()
    B.e2e_release_frame(renderer.ctx, fid)
    assert compare(host.astype(np.float64), ref).ok
    with pytest.raises(B.E2EError):
        B.e2e_release_frame(renderer.ctx, fid)


@pytest.mark.parametrize("kind", ["separable", "elliptical"])
def test_debug_checks_find_nothing_and_change_nothing(kind):
    # debug mode counts deposits outside the planned boxes; the plan covers every stamp, so
    # a checked render succeeds and is bitwise the unchecked one
    from paper_2008_05858_gb300.binding import Renderer

    psf = W.PSF_ELLIPTICAL if kind == "elliptical" else W.PSF_SEPARABLE
    ws = [W.small_config(seed=301, psf=psf), W.small_config(seed=302, K=7, n_lambda=500, n_slit=40, psf=psf),
          W.config2(n_orders=6)]
    plain, checked = Renderer(0), Renderer(0, debug_checks=1)
    try:
        for w in ws[: 3 if kind == "separable" else 2]:
            a = gpu_frames(plain, w, "mixed", "f32")
            b = gpu_frames(checked, w, "mixed", "f32")
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    finally:
        plain.close()
        checked.close()


@pytest.mark.parametrize("psf", [W.PSF_SEPARABLE, W.PSF_ELLIPTICAL], ids=["separable", "elliptical"])
def test_blazed_model_matches_oracle(renderer, psf):
    w = W.small_config(seed=511 + psf, orders=2, psf=psf)
    for s in w.model.slices:
        s.blaze_order = 110.0
        s.blaze_lambda = 0.5 * (s.lambda_lo + s.lambda_hi)
    ref = oracle.render_workload(w)[0]
    assert compare(gpu_frames(renderer, w, "mixed", "f32")[0], ref).ok
    g64 = gpu_frames(renderer, w, "fp64", "f64")[0]
    assert np.all(np.abs(g64 - ref) <= FP64_REL * np.abs(ref) + 1e-15 * np.abs(ref).max())


@pytest.mark.parametrize("psf", [W.PSF_SEPARABLE, W.PSF_ELLIPTICAL, W.PSF_TABLE], ids=["sep", "ellip", "table"])
@pytest.mark.parametrize("shape", [dict(n_lambda=1, n_slit=1), dict(n_lambda=1, n_slit=40), dict(n_lambda=33, n_slit=1),
                                   dict(n_lambda=5, n_slit=3, K=1)], ids=["1x1", "1x40", "33x1", "K1"])
def test_degenerate_sizes_every_psf(renderer, psf, shape):
    # single samples, single slit points and a one-pixel window, for every PSF kind and both
    # precisions
    kw = dict(seed=801, orders=2, fibers=1, slices=2)
    kw.update(shape)
    w = W.small_config(psf=psf if psf != W.PSF_TABLE else W.PSF_SEPARABLE, **kw)
    if psf == W.PSF_TABLE:
        w = W.Workload(w.name, W.with_psf_maps(w.model, oversample=6.0, half_px=6.0, n_field=3), w.spectra, "f32",
                       "mixed")
    ref = oracle_frames(w)
    for g, o in zip(gpu_frames(renderer, w, "mixed", "f32"), ref):
        assert compare(g, o).ok
    for g, o in zip(gpu_frames(renderer, w, "fp64", "f64"), ref):
        assert np.all(np.abs(g - o) <= FP64_REL * np.abs(o) + 1e-15 * max(np.abs(o).max(), 1e-300))


def test_several_window_sizes_in_one_model(renderer):
    # slices of K = 7, 11 and 9 on overlapping traces: one render launch per K, with tiles
    # shared between the launches (their fused merge counts items across launches)
    w = W.small_config(seed=71, orders=3, trace_pitch=6.0, height=200)
    for i, s in enumerate(w.model.slices):
        s.K = (7, 11, 9)[i % 3]
    ref = oracle.render_workload(w)
    got = gpu_frames(renderer, w, "mixed", "f32")
    for g, o in zip(got, ref):
        rep = compare(g, o)
        assert rep.ok, str(rep)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    try:
        host = renderer.render_host(mid, sids)
        assert all(np.array_equal(h.numpy(), g) for h, g in zip(host, got))
    finally:
        from paper_2008_05858_gb300.binding import e2e_unload_spectrum

        for s in sids:
            e2e_unload_spectrum(renderer.ctx, s)
        renderer.unload_model(mid)


def _poly2(c, degree, lt, s):
    """x or y of a slice's mapping on the grid lt x s (a plain evaluation for choosing windows)."""
    out = np.zeros((len(lt), len(s)))
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            out += c[W.coeff_index(a, b)] * np.outer(lt ** a, s ** b)
    return out


def test_config2_full_frame_sampled_windows(renderer):
    # The benchmark's frame itself (85 orders x 2 fibers x 2 slices x 6000 x 64 stamps, K = 11,
    # 9216^2), rendered as the benchmark renders it.  64 x 64 windows on the traces are checked
    # against the oracle, which renders each window alone: only the slices whose traces come
    # within reach of it, translated so the window is the oracle's whole frame.
    import dataclasses

    w = W.config2()
    got = gpu_frames(renderer, w, "mixed", "f32")[0]
    H, Wd = w.model.det_shape[0]
    lt, ss = np.linspace(-1.0, 1.0, 513), np.linspace(-1.0, 1.0, 9)
    yr = []
    for s in w.model.slices:
        y = _poly2(s.cy, s.degree, lt, ss)
        yr.append((y.min(), y.max()))
    rng = np.random.default_rng(2008)
    n_win, size = 6, 64
    for _ in range(n_win):
        s = w.model.slices[int(rng.integers(len(w.model.slices)))]
        t = rng.uniform(-0.95, 0.95)
        xc = float(_poly2(s.cx, s.degree, np.array([t]), np.array([0.0]))[0, 0])
        yc = float(_poly2(s.cy, s.degree, np.array([t]), np.array([0.0]))[0, 0])
        x0 = int(min(max(round(xc) - size // 2, 0), Wd - size))
        y0 = int(min(max(round(yc) - size // 2, 0), H - size))
        reach = 2 + s.K
        sub = []
        for q, (lo, hi) in zip(w.model.slices, yr):
            if hi + reach >= y0 and lo - reach <= y0 + size:
                c = q.copy()
                c.cx[0] -= x0
                c.cy[0] -= y0
                sub.append(c)
        ref = oracle.render(W.OpticalModel([(size, size)], sub, w.model.psf), w.flux_for)[0]
        assert np.abs(ref).max() > 0
        rep = compare(got[y0:y0 + size, x0:x0 + size], ref)
        assert rep.ok, f"window at ({x0}, {y0}): {rep}"


def test_width_updates_across_the_far_edge_threshold(renderer):
    # the plan's choice of tail rational follows the model's widest PSF through coefficient
    # updates: widths of 1.3-1.9 px (cheaper rational), scaled by 1.6 (up to ~3 px: general one)
    # and back, each state checked against the oracle's render of the updated model
    w = W.small_config(seed=19, K=11, degree=4, n_lambda=150, n_slit=12, sigma_range=(1.3, 1.9))
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    cx, cy, sx, sy = renderer.params(mid)
    try:
        for scale in (1.0, 1.6, 1.0):
            renderer.update(mid, cx, cy, sx * scale, sy * scale)
            got = renderer.render(mid, sids, "mixed", "f32")
            torch.cuda.synchronize()
            m = renderer.models[mid]
            ref = oracle.render(m, w.flux_for)
            ties = tie_boxes(m, w.flux_for)
            for d, g in enumerate(got):
                rep = compare(g.double().cpu().numpy(), ref[d], ties=ties[d])
                print(f"scale {scale} detector {d}: {rep}")
                assert rep.ok, str(rep)
    finally:
        renderer.unload_model(mid)
