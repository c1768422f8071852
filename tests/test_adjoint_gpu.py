"""Adjoint kernel (e2e_render_adjoint) against the FP64 oracle's vector-Jacobian product and
against central differences of the GPU render, through the C ABI and the autograd Function.

Tolerance: the adjoint sums FP32 pixel-integral derivatives weighted by dL/dI of both signs,
so its error is relative to the size of the gradient vector, not of each entry: per
coefficient group (cx, cy, sigma_x, sigma_y) |g - o| <= 2e-5 max|o| + 2e-4 |o|.
"""
import numpy as np
import pytest

import oracle
from paper_2008_05858_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def check_groups(got, ref, atol_frac=2e-5, rtol=2e-4):
    for name, g, o in zip(("cx", "cy", "sx", "sy"), got, ref):
        g = g.cpu().numpy() if hasattr(g, "cpu") else np.asarray(g)
        scale = np.abs(o).max() if o.size else 0.0
        err = np.abs(g - o)
        bad = err > atol_frac * scale + rtol * np.abs(o)
        assert not bad.any(), f"{name}: max err {err.max():.3e} scale {scale:.3e} at {np.argmax(err)}"


@pytest.mark.parametrize("kw", [dict(seed=5, K=9, degree=3, n_lambda=90, n_slit=9),
                                dict(seed=6, K=11, degree=5, n_lambda=200, n_slit=32),
                                dict(seed=7, K=7, degree=4, n_lambda=333, n_slit=13, orders=3),
                                dict(seed=8, K=15, degree=8, n_lambda=120, n_slit=20)],
                         ids=["k9", "k11", "k7", "k15-degree8"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_adjoint_matches_oracle_vjp(renderer, kw, dtype):
    w = W.small_config(**kw)
    rng = np.random.default_rng(kw["seed"])
    dldi = [rng.standard_normal((h, wd)) for h, wd in w.model.det_shape]
    ref = oracle.vjp(w.model, w.flux_for, dldi)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    td = torch.float32 if dtype == "f32" else torch.float64
    dev = [torch.tensor(d, dtype=td, device="cuda") for d in dldi]
    if dtype == "f32":  # the oracle sees the same (rounded) dL/dI
        ref = oracle.vjp(w.model, w.flux_for, [d.double().cpu().numpy() for d in dev])
    got = renderer.adjoint(mid, sids, dev)
    torch.cuda.synchronize()
    check_groups(got, ref)
    renderer.unload_model(mid)


def test_autograd_gradient_matches_central_differences(renderer):
    from paper_2008_05858_gb300 import autograd as AG

    # a wide window (K=15 at sigma ~1.05 truncates at > 7 sigma), so the jumps where a window
    # re-centres are far below the finite-difference signal
    w = W.small_config(seed=9, K=15, degree=3, n_lambda=60, n_slit=6, orders=1, fibers=1, slices=2,
                       width=160, height=70)
    for s in w.model.slices:
        s.sigma_x = np.array([1.05, 0.02, 0.0])
        s.sigma_y = np.array([1.0, -0.02, 0.0])
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    p0 = AG.pack(renderer.params(mid))
    frames0 = renderer.render(mid, sids, "mixed", "f64")
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    target = torch.tensor(frames0[0].cpu().numpy() * 0.98 + rng.normal(0, 0.01, frames0[0].shape),
                          dtype=torch.float32, device="cuda")

    def loss_of(vec):
        fr = AG.render(torch.tensor(vec, dtype=torch.float64), renderer, mid, sids)
        return ((fr[0].double() - target.double()) ** 2).sum()

    params = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    L = ((AG.render(params, renderer, mid, sids)[0].double() - target.double()) ** 2).sum()
    L.backward()
    g = params.grad.numpy()
    nc = sum(len(s.cx) for s in w.model.slices)
    idxs = [0, 1, 2, 5, nc + 0, nc + 2, nc + 7, 2 * nc + 0, 2 * nc + 3 + 1, 2 * nc + 6 + 0]
    for i in idxs:
        h = 2e-3 if i < 2 * nc else 1e-3
        vp, vm = p0.copy(), p0.copy()
        vp[i] += h
        vm[i] -= h
        fd = (loss_of(vp).item() - loss_of(vm).item()) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-3, abs=2e-3 * np.abs(g).max()), (i, g[i], fd)
    renderer.update(mid, *AG.unpack(p0, nc, len(w.model.slices)))
    renderer.unload_model(mid)


def test_config5_calibration_gradient(renderer):
    # differentiation workload: target rendered from coefficients shifted by up to 0.01 px,
    # plus seeded Poisson noise; the loss gradient from the adjoint equals the oracle's
    w = W.config5()
    rng = np.random.default_rng(W.SEED_BASE + 5)
    shifted = w.model.copy()
    for s in shifted.slices:
        s.cx[0] += rng.uniform(-0.01, 0.01)
        s.cy[0] += rng.uniform(-0.01, 0.01)
    T = oracle.render(shifted, w.flux_for)[0]
    T = rng.poisson(np.maximum(T, 0.0)).astype(np.float64)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    I = renderer.render(mid, sids, "mixed", "f32")[0]
    dldi = 2.0 * (I.double() - torch.tensor(T, device="cuda"))
    got = renderer.adjoint(mid, sids, [dldi])
    torch.cuda.synchronize()
    ref = oracle.vjp(w.model, w.flux_for, [dldi.cpu().numpy()])
    check_groups(got, ref)
    renderer.unload_model(mid)


def test_window_origins_are_the_oracle_windows(renderer):
    # every stamp's window origin floor(x_c + 1/2) - K/2 against the oracle's mapping; a stamp
    # whose centre lies within 1e-9 px of a half-integer may round either way (a tie)
    w = W.small_config(seed=21, K=9, degree=5, n_lambda=150, n_slit=11, orders=2)
    mid = renderer.load_model(w.model)
    got = renderer.window_origins(mid).cpu().numpy()
    torch.cuda.synchronize()
    assert got.shape == (w.model.n_stamps, 2)
    t = 0
    for s in w.model.slices:
        f = w.flux_for(s)
        for j in range(s.n_lambda):
            for k in range(s.n_slit):
                xc, yc, _, _, _ = oracle.map_stamp(s, f, j, k)
                for a, c in ((0, xc), (1, yc)):
                    want = int(np.floor(c + 0.5)) - s.K // 2
                    if got[t, a] != want:
                        assert abs((c + 0.5) - round(c + 0.5)) < 1e-9, (t, a, c, got[t, a], want)
                t += 1
    renderer.unload_model(mid)


def test_frozen_windows_central_differences_at_config5_window(renderer):
    # Differentiation workload at its own K = 9 (sigma 1.2..2.0: the window truncates at
    # ~2.2 sigma, so a re-centring window jumps by far more than a finite-difference signal).
    # With windows frozen at the unperturbed render's origins (the reading of the gradient as
    # the derivative with origins held), central differences of the FP64 frozen render agree
    # with the adjoint and with the oracle's vector-Jacobian product.
    w = W.config5()
    w.model.slices = w.model.slices[:4]  # 4 order-slices keep the oracle's reference quick
    rng = np.random.default_rng(W.SEED_BASE + 55)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    frozen = renderer.window_origins(mid)
    I0 = renderer.render(mid, sids, "fp64", "f64")[0]
    If = renderer.render_frozen(mid, sids, frozen)[0]
    torch.cuda.synchronize()
    # frozen at the mapping's own origins: the plain FP64 render (up to FP64 atomic ordering)
    assert torch.allclose(I0, If, rtol=1e-13, atol=1e-13 * float(I0.abs().max()))
    T = torch.tensor(rng.poisson(np.maximum(I0.cpu().numpy() * 1.01, 0.0)).astype(np.float64), device="cuda")
    dldi = 2.0 * (I0 - T)
    g = [x.cpu().numpy() for x in renderer.adjoint(mid, sids, [dldi], frozen=frozen)]
    g_nat = [x.cpu().numpy() for x in renderer.adjoint(mid, sids, [dldi])]
    ref = oracle.vjp(w.model, w.flux_for, [dldi.cpu().numpy()])
    check_groups(g, ref)
    for a, b in zip(g, g_nat):  # the same windows: the same gradient
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-9 * np.abs(b).max())
    p0 = renderer.params(mid)
    nc = len(p0[0])

    def loss(parts):
        renderer.update(mid, *parts)
        fr = renderer.render_frozen(mid, sids, frozen)[0]
        return float(((fr - T) ** 2).sum())

    cases = [(0, 0, 1e-3), (0, 1, 1e-3), (0, nc - 1, 1e-3), (1, 0, 1e-3), (1, 2, 1e-3), (1, 16, 1e-3),
             (2, 0, 1e-4), (2, 4, 1e-4), (3, 1, 1e-4), (3, 9, 1e-4)]
    for grp, i, h in cases:
        vp = [np.array(x, dtype=np.float64) for x in p0]
        vm = [np.array(x, dtype=np.float64) for x in p0]
        vp[grp][i] += h
        vm[grp][i] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        scale = np.abs(g[grp]).max()
        assert g[grp][i] == pytest.approx(fd, rel=2e-3, abs=2e-4 * scale), (grp, i, g[grp][i], fd)
        assert ref[grp][i] == pytest.approx(fd, rel=2e-3, abs=2e-4 * scale), (grp, i, ref[grp][i], fd)
    renderer.update(mid, *p0)
    renderer.unload_model(mid)
