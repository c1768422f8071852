"""Detector noise stage (e2e_add_noise) against the oracle's restatement of the same model.

Integer results are compared bit for bit: the Poisson counts (read back as the electrons of
a run with no read-out noise and no cross-talk) and the ADU codes.  The kernel reaches them
by FP32 arithmetic with error bounds and redoes a draw in FP64 where a comparison is too
close to call; a million-pixel frame exercises that fallback.  FP64 electrons are FP64 sums
of the integers and of FP64 normals whose sine, cosine and logarithm come from CUDA's and
the C library's FP64 functions (a few ulp apart): compared at 1e-13 relative (1e-12
absolute).  FP32 electrons carry FP32 read-out noise: within 4e-7 relative + 5e-5."""
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


def model_of(shapes):
    return W.OpticalModel(list(shapes), [])


def signal(shape, seed):
    # a rendered-frame-like signal: empty background, faint wings, bright traces
    rng = np.random.default_rng(seed)
    S = rng.exponential(3.0, shape)
    S[rng.random(shape) < 0.3] = 0.0
    bright = rng.random(shape) < 0.2
    S[bright] = rng.uniform(10, 60000, bright.sum())
    return S


def to_np(t):
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.int64)
    return t.double().cpu().numpy()


PARAMS = dict(seed=20201105, pattern_seed=17, dark_e=2.5, prnu=0.01, ron_e=3.2, xtalk=2e-4, gain=1.1,
              bias=1000.0, saturation=65535)


@pytest.mark.parametrize("shapes", [[(37, 53)], [(64, 64), (17, 1), (9, 2)]], ids=["odd", "multi"])
def test_poisson_counts_are_bit_exact(renderer, shapes):
    mid = renderer.load_model(model_of(shapes))
    Ss = [signal(s, 5 + i) for i, s in enumerate(shapes)]
    src = [torch.tensor(S, dtype=torch.float64, device="cuda") for S in Ss]
    p = dict(PARAMS, ron_e=0.0, xtalk=0.0)
    out = renderer.add_noise(mid, src, "f64", **p)
    torch.cuda.synchronize()
    for d, (S, o) in enumerate(zip(Ss, out)):
        _, _, N = oracle.add_noise(S, d, seed=p["seed"], pattern_seed=p["pattern_seed"], dark=p["dark_e"],
                                   prnu=p["prnu"])
        assert np.array_equal(to_np(o), N)
    renderer.unload_model(mid)


def test_poisson_counts_bit_exact_on_a_megapixel_frame(renderer):
    # ~1e6 draws from both samplers (inversion below 10 e-, transformed rejection above):
    # the FP32 filter's FP64 fallback fires on some of them
    shape = (1024, 1001)
    mid = renderer.load_model(model_of([shape]))
    S = signal(shape, 33)
    src = [torch.tensor(S, dtype=torch.float32, device="cuda")]
    p = dict(PARAMS, ron_e=0.0, xtalk=0.0)
    out = renderer.add_noise(mid, src, "f64", **p)
    torch.cuda.synchronize()
    _, _, N = oracle.add_noise(src[0].double().cpu().numpy(), 0, seed=p["seed"], pattern_seed=p["pattern_seed"],
                               dark=p["dark_e"], prnu=p["prnu"])
    got = to_np(out[0])
    assert np.array_equal(got, N), int((got != N).sum())
    renderer.unload_model(mid)


@pytest.mark.parametrize("src_dtype", ["f32", "f64"])
def test_electrons_and_adu_match_oracle(renderer, src_dtype):
    shapes = [(41, 70), (8, 33)]
    mid = renderer.load_model(model_of(shapes))
    td = torch.float32 if src_dtype == "f32" else torch.float64
    src = [torch.tensor(signal(s, 9 + i), dtype=td, device="cuda") for i, s in enumerate(shapes)]
    e = renderer.add_noise(mid, src, "f64", **PARAMS)
    a = renderer.add_noise(mid, src, "u16", **PARAMS)
    e32 = renderer.add_noise(mid, src, "f32", **PARAMS)
    torch.cuda.synchronize()
    for d, s in enumerate(src):
        S = s.double().cpu().numpy()
        E, A, _ = oracle.add_noise(S, d, seed=PARAMS["seed"], pattern_seed=PARAMS["pattern_seed"],
                                   dark=PARAMS["dark_e"], prnu=PARAMS["prnu"], ron=PARAMS["ron_e"],
                                   xtalk=PARAMS["xtalk"], gain=PARAMS["gain"], bias=PARAMS["bias"],
                                   saturation=PARAMS["saturation"])
        ge = to_np(e[d])
        assert np.all(np.abs(ge - E) <= 1e-13 * np.abs(E) + 1e-12)
        assert np.array_equal(to_np(a[d]), A)
        # FP32 electrons carry FP32 read-out noise: within a few ulp of E plus 1e-5 of ron
        assert np.all(np.abs(e32[d].double().cpu().numpy() - E) <= 4e-7 * np.abs(E) + 5e-5)
    renderer.unload_model(mid)


def test_in_place_and_saturation(renderer):
    shapes = [(16, 31)]
    mid = renderer.load_model(model_of(shapes))
    S = signal(shapes[0], 21)
    f = torch.tensor(S, dtype=torch.float64, device="cuda")
    p = dict(PARAMS, gain=0.5, saturation=4000)
    ref = renderer.add_noise(mid, [f], "f64", **p)[0].clone()
    renderer.add_noise(mid, [f], "f64", out=[f], **p)
    a = renderer.add_noise(mid, [torch.tensor(S, dtype=torch.float64, device="cuda")], "u16", **p)[0]
    torch.cuda.synchronize()
    assert torch.equal(ref, f)
    A = to_np(a)
    assert A.max() == 4000 and A.min() >= 0
    renderer.unload_model(mid)


def test_rendered_frame_full_size_rows(renderer):
    # the full-detector frame (9216^2) of the benchmark's workload, noise in the launch shape
    # the benchmark times; rows sampled across the frame are recomputed by the oracle
    w = W.config2(n_orders=85)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    frame = renderer.render(mid, sids, "mixed", "f32")
    out = renderer.add_noise(mid, frame, "u16", **PARAMS)
    torch.cuda.synchronize()
    H, Wd = w.model.det_shape[0]
    rows = [0, 1, 2047, 4608, 9215]
    S = frame[0][rows].double().cpu().numpy()
    A = out[0].view(torch.int16)[rows].cpu().numpy().view(np.uint16).astype(np.int64)
    for i, r in enumerate(rows):
        _, Ar, _ = oracle.add_noise(S[i:i + 1], 0, row0=r, seed=PARAMS["seed"], pattern_seed=PARAMS["pattern_seed"],
                                    dark=PARAMS["dark_e"], prnu=PARAMS["prnu"], ron=PARAMS["ron_e"],
                                    xtalk=PARAMS["xtalk"], gain=PARAMS["gain"], bias=PARAMS["bias"],
                                    saturation=PARAMS["saturation"])
        assert np.array_equal(A[i], Ar[0])
    renderer.unload_model(mid)


def test_bad_parameters_are_rejected(renderer):
    from paper_2008_05858_gb300.binding import E2EError, E2E_EINVAL

    mid = renderer.load_model(model_of([(4, 4)]))
    f = [torch.zeros((4, 4), dtype=torch.float32, device="cuda")]
    for bad in (dict(gain=0.0), dict(saturation=70000), dict(ron_e=-1.0), dict(xtalk=1.5)):
        with pytest.raises(E2EError) as e:
            renderer.add_noise(mid, f, "u16", **dict(PARAMS, **bad))
        assert e.value.code == E2E_EINVAL
    renderer.unload_model(mid)
