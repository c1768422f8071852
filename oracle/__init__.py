"""FP64 CPU oracle of the echelle frame renderer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product renderer (``paper_2008_05858_gb300``) never
imports it and shares no code with it; both take their inputs from the seeded
generators in ``paper_2008_05858_gb300.workloads``, which hold no renderer arithmetic.

The C source (``oracle.c``) is a plain FP64 restatement of the paper's image model
(Sec. 2, Sec. 2.2): the frame is the superposition over the wavelength grid of
pixel-integrated fiber images.  This module compiles it with gcc and wraps it with
ctypes.

Pins (checked by ``tests/test_oracle_pins.py`` against closed forms, brute-force
quadrature, library routines and invariants -- never against the CUDA path):
separable stamps, bivariate-normal rectangles, Gauss-Legendre nodes, the paper's
sub-pixel sampling limit, mapping/coefficient order, flux conservation, photocenter,
superposition, and the loss gradient (central differences).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "noise.c"), os.path.join(_HERE, "photons.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

PSF_SEPARABLE = 0
PSF_ELLIPTICAL = 1
PSF_TABLE = 2


class OracleNoise(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("pattern_seed", C.c_uint64), ("dark", C.c_double), ("prnu", C.c_double),
        ("ron", C.c_double), ("xtalk", C.c_double), ("gain", C.c_double), ("bias", C.c_double),
        ("saturation", C.c_int32), ("poisson", C.c_int32),
    ]


class OracleSlice(C.Structure):
    _fields_ = [
        ("detector", C.c_int),
        ("degree", C.c_int),
        ("K", C.c_int),
        ("n_lambda", C.c_int),
        ("n_slit", C.c_int),
        ("lambda_lo", C.c_double),
        ("lambda_hi", C.c_double),
        ("cx", C.POINTER(C.c_double)),
        ("cy", C.POINTER(C.c_double)),
        ("sx", C.c_double * 3),
        ("sy", C.c_double * 3),
        ("theta", C.c_double),
        ("u", C.POINTER(C.c_double)),
        ("flux", C.POINTER(C.c_double)),
        ("blaze_order", C.c_double),
        ("blaze_lambda", C.c_double),
        ("n_aper", C.c_int),
        ("ax", C.c_double * 3),
        ("ay", C.c_double * 3),
        ("n_field", C.c_int),
        ("field_lt", C.POINTER(C.c_double)),
        ("map_size", C.c_int),
        ("map_oversample", C.c_double),
        ("maps", C.POINTER(C.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        [os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(os.path.join(_HERE, "oracle.h"))]
    ):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.oracle_render.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                        C.POINTER(OracleSlice), C.c_int, C.POINTER(dp), C.c_int]
            L.oracle_render.restype = C.c_int
            L.oracle_map.argtypes = [C.POINTER(OracleSlice), C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_map.restype = None
            L.oracle_stamp.argtypes = [C.POINTER(OracleSlice), C.c_int, C.c_int, C.c_int, dp,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.oracle_stamp.restype = None
            L.oracle_normal_interval.argtypes = [C.c_double, C.c_double]
            L.oracle_normal_interval.restype = C.c_double
            L.oracle_bvn_cdf.argtypes = [C.c_double, C.c_double, C.c_double]
            L.oracle_bvn_cdf.restype = C.c_double
            L.oracle_bvn_rect.argtypes = [C.c_double] * 5
            L.oracle_bvn_rect.restype = C.c_double
            L.oracle_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.oracle_gauss_legendre.restype = None
            L.oracle_subpixel_sample.argtypes = [C.c_double] * 4 + [C.c_int] * 3
            L.oracle_subpixel_sample.restype = C.c_double
            L.oracle_loss_grad.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                           C.POINTER(OracleSlice), C.POINTER(dp), dp, dp, dp, dp, C.c_int]
            L.oracle_loss_grad.restype = C.c_double
            L.oracle_vjp.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                     C.POINTER(OracleSlice), C.POINTER(dp), dp, dp, dp, dp, C.c_int]
            L.oracle_vjp.restype = C.c_int
            L.oracle_epsf_pixel.argtypes = [C.POINTER(OracleSlice), C.c_int, C.c_double, C.c_double, C.c_int, C.c_int]
            L.oracle_epsf_pixel.restype = C.c_double
            L.oracle_epsf_window.argtypes = [C.POINTER(OracleSlice), C.c_int, C.c_double, C.c_double, dp]
            L.oracle_epsf_window.restype = None
            L.oracle_window_ties.argtypes = [C.POINTER(OracleSlice), C.c_double, C.c_int, C.POINTER(C.c_int)]
            L.oracle_window_ties.restype = C.c_int
            u32p = C.POINTER(C.c_uint32)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_philox4x32_10.restype = None
            L.oracle_normal_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, dp, dp]
            L.oracle_normal_pair.restype = None
            L.oracle_poisson.argtypes = [C.c_double, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
            L.oracle_poisson.restype = C.c_long
            L.oracle_add_noise.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, C.POINTER(OracleNoise), dp,
                                           C.POINTER(C.c_int32), dp]
            L.oracle_add_noise.restype = C.c_int
            L.oracle_render_photons.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                                C.POINTER(OracleSlice), C.c_int, C.c_uint64,
                                                C.POINTER(C.POINTER(C.c_uint32)), C.POINTER(C.c_uint64)]
            L.oracle_render_photons.restype = C.c_int
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Marshalled:
    """Keeps the numpy arrays alive while the C structs point into them."""

    def __init__(self, model, flux_of):
        self.keep = []
        n = len(model.slices)
        self.arr = (OracleSlice * max(n, 1))()
        for i, s in enumerate(model.slices):
            cx = np.ascontiguousarray(s.cx, dtype=np.float64)
            cy = np.ascontiguousarray(s.cy, dtype=np.float64)
            u = np.ascontiguousarray(s.slit_weights, dtype=np.float64)
            fl = np.ascontiguousarray(flux_of(s), dtype=np.float64)
            assert fl.shape == (s.n_lambda,), "flux length must equal n_lambda"
            assert cx.shape == ((s.degree + 1) * (s.degree + 2) // 2,)
            rows = max(1, int(getattr(s, "n_aper", 0)))
            assert u.shape == (s.n_slit * rows,), "slit weights: n_slit per aperture row"
            self.keep += [cx, cy, u, fl]
            o = self.arr[i]
            o.detector, o.degree, o.K, o.n_lambda, o.n_slit = s.detector, s.degree, s.K, s.n_lambda, s.n_slit
            o.lambda_lo, o.lambda_hi = s.lambda_lo, s.lambda_hi
            o.cx, o.cy, o.u, o.flux = _dptr(cx), _dptr(cy), _dptr(u), _dptr(fl)
            for p in range(3):
                o.sx[p] = float(s.sigma_x[p])
                o.sy[p] = float(s.sigma_y[p])
            o.theta = float(s.theta)
            o.blaze_order = float(getattr(s, "blaze_order", 0.0))
            o.blaze_lambda = float(getattr(s, "blaze_lambda", 0.0))
            o.n_aper = int(getattr(s, "n_aper", 0))
            for p in range(3):
                o.ax[p] = float(getattr(s, "aper_x", np.zeros(3))[p])
                o.ay[p] = float(getattr(s, "aper_y", np.zeros(3))[p])
            psf_map = getattr(s, "psf_map", None)
            if psf_map is not None:
                lt = np.ascontiguousarray(psf_map.field_lt, dtype=np.float64)
                mp = np.ascontiguousarray(psf_map.maps, dtype=np.float64)
                self.keep += [lt, mp]
                o.n_field, o.field_lt = len(lt), _dptr(lt)
                o.map_size, o.map_oversample, o.maps = mp.shape[-1], float(psf_map.oversample), _dptr(mp)
        self.n = n


def _flux_getter(workload=None, flux: Optional[Dict] = None):
    if flux is not None:
        return lambda s: flux[(s.order, s.fiber)]
    return workload.flux_for


def render(model, flux_of, n_threads: int = 0) -> List[np.ndarray]:
    """FP64 frames (one per detector) of ``model`` lit by ``flux_of(slice) -> flux[n_lambda]``."""
    L = lib()
    m = _Marshalled(model, flux_of)
    H = (C.c_int * len(model.det_shape))(*[h for h, w in model.det_shape])
    W = (C.c_int * len(model.det_shape))(*[w for h, w in model.det_shape])
    frames = [np.zeros((h, w), dtype=np.float64) for h, w in model.det_shape]
    ptrs = (C.POINTER(C.c_double) * len(frames))(*[_dptr(f) for f in frames])
    rc = L.oracle_render(len(frames), H, W, m.n, m.arr, int(model.psf), ptrs, int(n_threads))
    if rc != 0:
        raise ValueError("oracle_render rejected the model")
    return frames


def render_photons(model, flux_of, seed: int) -> Tuple[List[np.ndarray], int]:
    """Photon Monte-Carlo frames (uint32 counts per detector) and the number of photons drawn."""
    L = lib()
    m = _Marshalled(model, flux_of)
    H = (C.c_int * len(model.det_shape))(*[h for h, w in model.det_shape])
    W = (C.c_int * len(model.det_shape))(*[w for h, w in model.det_shape])
    frames = [np.zeros((h, w), dtype=np.uint32) for h, w in model.det_shape]
    ptrs = (C.POINTER(C.c_uint32) * len(frames))(*[f.ctypes.data_as(C.POINTER(C.c_uint32)) for f in frames])
    total = C.c_uint64()
    rc = L.oracle_render_photons(len(frames), H, W, m.n, m.arr, int(model.psf), seed, ptrs, C.byref(total))
    if rc != 0:
        raise ValueError("oracle_render_photons rejected the model")
    return frames, total.value


def render_workload(w, n_threads: int = 0) -> List[np.ndarray]:
    return render(w.model, w.flux_for, n_threads)


def stamp(s, flux: np.ndarray, j: int, k: int, psf: int = PSF_SEPARABLE) -> Tuple[np.ndarray, int, int]:
    """The K x K FP64 values of stamp (j, k) of one order-slice and its window origin (i0, r0)."""
    L = lib()
    from paper_2008_05858_gb300.workloads import OpticalModel  # input container only

    m = _Marshalled(OpticalModel([(1, 1)], [s]), lambda _s: flux)
    out = np.zeros(s.K * s.K)
    i0, r0 = C.c_int(), C.c_int()
    L.oracle_stamp(m.arr, psf, j, k, _dptr(out), C.byref(i0), C.byref(r0))
    return out.reshape(s.K, s.K), i0.value, r0.value


def map_stamp(s, flux: np.ndarray, j: int, k: int) -> Tuple[float, float, float, float, float]:
    """(x_c, y_c, sigma_x, sigma_y, weight) of stamp (j, k)."""
    L = lib()
    from paper_2008_05858_gb300.workloads import OpticalModel

    m = _Marshalled(OpticalModel([(1, 1)], [s]), lambda _s: flux)
    v = [C.c_double() for _ in range(5)]
    L.oracle_map(m.arr, j, k, *[C.byref(x) for x in v])
    return tuple(x.value for x in v)


def normal_interval(a: float, b: float) -> float:
    return lib().oracle_normal_interval(a, b)


def bvn_cdf(h: float, k: float, rho: float) -> float:
    return lib().oracle_bvn_cdf(h, k, rho)


def bvn_rect(h0: float, h1: float, k0: float, k1: float, rho: float) -> float:
    return lib().oracle_bvn_rect(h0, h1, k0, k1, rho)


def gauss_legendre(n: int) -> Tuple[np.ndarray, np.ndarray]:
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _dptr(x), _dptr(w))
    return x, w


def subpixel_sample(xc, yc, sx, sy, i, r, nsub) -> float:
    return lib().oracle_subpixel_sample(xc, yc, sx, sy, i, r, nsub)


def loss_grad(model, flux_of, targets: Sequence[np.ndarray], n_threads: int = 0):
    """(L, g_cx, g_cy, g_sx, g_sy) for L = sum (I - T)^2, windows frozen at the forward render's."""
    L = lib()
    m = _Marshalled(model, flux_of)
    H = (C.c_int * len(model.det_shape))(*[h for h, w in model.det_shape])
    W = (C.c_int * len(model.det_shape))(*[w for h, w in model.det_shape])
    tg = [np.ascontiguousarray(t, dtype=np.float64) for t in targets]
    tp = (C.POINTER(C.c_double) * len(tg))(*[_dptr(t) for t in tg])
    ncs = [(s.degree + 1) * (s.degree + 2) // 2 for s in model.slices]
    gcx = np.zeros(sum(ncs))
    gcy = np.zeros(sum(ncs))
    gsx = np.zeros(3 * len(model.slices))
    gsy = np.zeros(3 * len(model.slices))
    loss = L.oracle_loss_grad(len(tg), H, W, m.n, m.arr, tp, _dptr(gcx), _dptr(gcy), _dptr(gsx), _dptr(gsy),
                              int(n_threads))
    return loss, gcx, gcy, gsx, gsy


def vjp(model, flux_of, dLdI: Sequence[np.ndarray], n_threads: int = 0):
    """(g_cx, g_cy, g_sx, g_sy) = sum over pixels of dL/dI * dI/dtheta, windows frozen."""
    L = lib()
    m = _Marshalled(model, flux_of)
    H = (C.c_int * len(model.det_shape))(*[h for h, w in model.det_shape])
    W = (C.c_int * len(model.det_shape))(*[w for h, w in model.det_shape])
    gs = [np.ascontiguousarray(g, dtype=np.float64) for g in dLdI]
    gp = (C.POINTER(C.c_double) * len(gs))(*[_dptr(g) for g in gs])
    ncs = [(s.degree + 1) * (s.degree + 2) // 2 for s in model.slices]
    gcx = np.zeros(sum(ncs))
    gcy = np.zeros(sum(ncs))
    gsx = np.zeros(3 * len(model.slices))
    gsy = np.zeros(3 * len(model.slices))
    rc = L.oracle_vjp(len(gs), H, W, m.n, m.arr, gp, _dptr(gcx), _dptr(gcy), _dptr(gsx), _dptr(gsy), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_vjp rejected the model")
    return gcx, gcy, gsx, gsy


# ---------------------------------------------------------------------------- detector noise


def philox4x32_10(counter: Sequence[int], key: Sequence[int]) -> List[int]:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = (C.c_uint32 * 4)(*counter)
    k = (C.c_uint32 * 2)(*key)
    out = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, out)
    return list(out)


def normal_pair(seed: int, q: int, d: int, stream: int) -> Tuple[float, float]:
    a, b = C.c_double(), C.c_double()
    lib().oracle_normal_pair(seed, q, d, stream, C.byref(a), C.byref(b))
    return a.value, b.value


def poisson(lam: float, seed: int, q: int, d: int, side: int = 0) -> int:
    return int(lib().oracle_poisson(lam, seed, q, d, side))


def add_noise(S: np.ndarray, det: int, *, seed: int, pattern_seed: int, dark: float = 0.0, prnu: float = 0.0,
              ron: float = 0.0, xtalk: float = 0.0, gain: float = 1.0, bias: float = 0.0,
              saturation: int = 65535, poisson: bool = True, row0: int = 0):
    """Noise stage of one detector frame, or of its rows row0.. (S holds those rows, full
    width): (electrons, ADU, Poisson counts)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    H, W = S.shape
    p = OracleNoise(seed, pattern_seed, dark, prnu, ron, xtalk, gain, bias, saturation, 1 if poisson else 0)
    E = np.empty((H, W))
    A = np.empty((H, W), dtype=np.int32)
    N = np.empty((H, W))
    rc = lib().oracle_add_noise(H, W, row0, det, _dptr(S), C.byref(p), _dptr(E),
                                A.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(N))
    if rc != 0:
        raise ValueError("oracle_add_noise: invalid argument")
    return E, A, N


def epsf_pixel(s, f: int, phx: float, phy: float, m: int, n: int) -> float:
    """Effective-PSF value of window pixel (m, n) of slice s's map f at phase (phx, phy)."""
    mm = _Marshalled(W_OpticalModel_one(s), lambda _s: np.zeros(_s.n_lambda))
    return float(lib().oracle_epsf_pixel(C.byref(mm.arr[0]), f, phx, phy, m, n))


def epsf_window(s, f: int, phx: float, phy: float) -> np.ndarray:
    """All K x K effective-PSF values (rows n, columns m) of slice s's map f at phase (phx, phy)."""
    mm = _Marshalled(W_OpticalModel_one(s), lambda _s: np.zeros(_s.n_lambda))
    out = np.empty((s.K, s.K))
    lib().oracle_epsf_window(C.byref(mm.arr[0]), f, phx, phy, _dptr(out))
    return out


def window_ties(model, flux_of, margin: float = 1e-9) -> List[Tuple[int, int, int, int, int]]:
    """(slice index, detector, j, k, axis) of every stamp whose mapped centre lies within
    `margin` px of a half-integer in x (axis 0) or y (axis 1): where the window rule may round
    either way."""
    from concurrent.futures import ThreadPoolExecutor

    m = _Marshalled(model, flux_of)
    L = lib()

    def one(i):  # ctypes releases the GIL during the call, so slices scan in parallel
        cap = 64
        while True:
            buf = (C.c_int * (3 * cap))()
            n = L.oracle_window_ties(C.byref(m.arr[i]), margin, cap, buf)
            if n <= cap:
                return [(i, model.slices[i].detector, buf[3 * t], buf[3 * t + 1], buf[3 * t + 2]) for t in range(n)]
            cap = n

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        parts = list(ex.map(one, range(len(model.slices))))
    return [t for p in parts for t in p]


def W_OpticalModel_one(s):
    class _M:
        slices = [s]
    return _M
