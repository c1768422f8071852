"""Thin ctypes binding of the renderer's C ABI (``include/e2e_render.h``).

Functions named ``e2e_*`` marshal arguments to the C entry points of the same name and
nothing else: every step of the render runs in the library's CUDA kernels.  PyTorch only
supplies device memory and streams.  The :class:`Renderer` class is a convenience layer
over those calls for optical models and spectra built by :mod:`.workloads`.

There is no CPU fallback: if the library cannot be loaded, or no GPU is present, calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import workloads as W

E2E_OK = 0
E2E_EINVAL = -1
E2E_ENOMEM = -2
E2E_ECUDA = -3
E2E_ENOTFOUND = -4
E2E_EBUSY = -5
E2E_ETOOBIG = -6
E2E_ETIMEOUT = -7
E2E_ECANCELLED = -8
E2E_EDEVICE = -9

E2E_PSF_SEPARABLE = 0
E2E_PSF_ELLIPTICAL = 1
E2E_PSF_TABLE = 2
E2E_PREC_MIXED = 0
E2E_PREC_FP64 = 1
E2E_F32 = 0
E2E_F64 = 1
E2E_U16 = 2

PRECISION = {"mixed": E2E_PREC_MIXED, "fp64": E2E_PREC_FP64}
DTYPE = {"f32": E2E_F32, "f64": E2E_F64}


class E2EError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"e2e error {code}: {msg}")
        self.code = code


class e2e_opts(C.Structure):
    _fields_ = [("pool_bytes", C.c_size_t), ("max_inflight", C.c_int32), ("debug_checks", C.c_int32),
                ("kernel_timing", C.c_int32)]


class e2e_order_slice(C.Structure):
    _fields_ = [
        ("detector", C.c_int32), ("order", C.c_int32), ("fiber", C.c_int32), ("slice", C.c_int32),
        ("degree", C.c_int32), ("K", C.c_int32), ("n_lambda", C.c_int32), ("n_slit", C.c_int32),
        ("lambda_lo", C.c_double), ("lambda_hi", C.c_double),
        ("cx", C.POINTER(C.c_double)), ("cy", C.POINTER(C.c_double)),
        ("sigma_x", C.c_double * 3), ("sigma_y", C.c_double * 3), ("theta", C.c_double),
        ("slit_weights", C.POINTER(C.c_double)), ("blaze_order", C.c_double), ("blaze_lambda", C.c_double),
        ("n_field", C.c_int32), ("field_lt", C.POINTER(C.c_double)), ("map_size", C.c_int32),
        ("map_oversample", C.c_double), ("maps", C.POINTER(C.c_double)),
        ("n_aper", C.c_int32), ("aper_x", C.c_double * 3), ("aper_y", C.c_double * 3),
    ]


class e2e_model_desc(C.Structure):
    _fields_ = [
        ("n_detectors", C.c_int32), ("height", C.POINTER(C.c_int32)), ("width", C.POINTER(C.c_int32)),
        ("n_slices", C.c_int32), ("slices", C.POINTER(e2e_order_slice)), ("psf", C.c_int32),
    ]


class e2e_plan_info(C.Structure):
    _fields_ = [
        ("chunk_lambda", C.c_int32), ("run_slit", C.c_int32), ("slack_x", C.c_int32), ("slack_y", C.c_int32),
        ("n_items", C.c_int64), ("n_tiles", C.c_int64), ("scratch_bytes", C.c_int64),
        ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("boxes_per_cta", C.c_int32), ("max_box_area", C.c_int32),
    ]


class e2e_noise_params(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("pattern_seed", C.c_uint64), ("dark_e", C.c_double), ("prnu", C.c_double),
        ("ron_e", C.c_double), ("xtalk", C.c_double), ("gain", C.c_double), ("bias", C.c_double),
        ("saturation", C.c_int32), ("poisson", C.c_int32),
    ]


class e2e_server_cfg(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("budget_bytes", C.c_size_t), ("express_stamps", C.c_int64),
                ("express_slots", C.c_int32)]


class e2e_job(C.Structure):
    _fields_ = [
        ("model_id", C.c_uint64), ("n_spec", C.c_int32), ("spec_ids", C.POINTER(C.c_uint64)),
        ("precision", C.c_int32), ("dtype", C.c_int32), ("dst", C.POINTER(C.c_void_p)),
        ("pitch_elems", C.POINTER(C.c_int64)),
    ]


class e2e_job_info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("submit_ms", C.c_double), ("admit_ms", C.c_double), ("done_ms", C.c_double),
        ("device_ms", C.c_double), ("budget_bytes", C.c_int64), ("frame_id", C.c_uint64), ("stamps", C.c_int64),
    ]


E2E_JOB_DONE = 0
E2E_JOB_RUNNING = 1
E2E_JOB_QUEUED = 2

HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()

_SIGS = {
    "e2e_last_error": ([], C.c_char_p),
    "e2e_create": ([C.POINTER(C.c_void_p), C.c_int32, C.POINTER(e2e_opts)], C.c_int),
    "e2e_destroy": ([C.c_void_p], None),
    "e2e_load_model": ([C.c_void_p, C.POINTER(e2e_model_desc), C.POINTER(C.c_uint64)], C.c_int),
    "e2e_unload_model": ([C.c_void_p, C.c_uint64], C.c_int),
    "e2e_load_spectrum": ([C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                           C.POINTER(C.c_double), C.POINTER(C.c_uint64)], C.c_int),
    "e2e_unload_spectrum": ([C.c_void_p, C.c_uint64], C.c_int),
    "e2e_render": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_int32, C.c_int32,
                    C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "e2e_render_host": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_int32, C.c_int32,
                         C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "e2e_render_alloc": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_int32, C.c_int32,
                          C.c_void_p, C.POINTER(C.c_uint64)], C.c_int),
    "e2e_fetch_frame": ([C.c_void_p, C.c_uint64, C.c_int32, C.c_void_p, C.c_int32, C.c_size_t, C.c_void_p], C.c_int),
    "e2e_release_frame": ([C.c_void_p, C.c_uint64], C.c_int),
    "e2e_model_plan": ([C.c_void_p, C.c_uint64, C.POINTER(e2e_plan_info)], C.c_int),
    "e2e_kernel_times": ([C.c_void_p, C.POINTER(C.c_char_p), C.POINTER(C.c_float), C.c_int32,
                          C.POINTER(C.c_int32)], C.c_int),
    "e2e_eval_tail": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "e2e_eval_tail_far": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "e2e_fma_probe": ([C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "e2e_render_static": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_int32,
                           C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "e2e_render_adjoint": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_int32,
                            C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "e2e_window_origins": ([C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p], C.c_int),
    "e2e_render_frozen": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_void_p, C.c_int32,
                           C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "e2e_update_model": ([C.c_void_p, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                          C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "e2e_render_photons": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_uint64), C.c_uint64,
                            C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(C.c_uint64), C.c_void_p], C.c_int),
    "e2e_add_noise": ([C.c_void_p, C.c_uint64, C.POINTER(e2e_noise_params), C.c_int32, C.POINTER(C.c_void_p),
                       C.POINTER(C.c_int64), C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p],
                      C.c_int),
    "e2e_server_start": ([C.c_void_p, C.POINTER(e2e_server_cfg)], C.c_int),
    "e2e_submit": ([C.c_void_p, C.POINTER(e2e_job), C.POINTER(C.c_uint64)], C.c_int),
    "e2e_poll": ([C.c_void_p, C.c_uint64, C.POINTER(e2e_job_info)], C.c_int),
    "e2e_wait": ([C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(e2e_job_info)], C.c_int),
    "e2e_cancel": ([C.c_void_p, C.c_uint64], C.c_int),
    "e2e_forget": ([C.c_void_p, C.c_uint64], C.c_int),
    "e2e_server_stop": ([C.c_void_p], C.c_int),
}

#: size of the library's fixed device scratch used by e2e_render_static
E2E_STATIC_SCRATCH_BYTES = 64 << 20


def lib_path() -> str:
    return os.path.join(HERE, "_build", "libe2e_render.so")


def load_library(build_if_missing: bool = True):
    """Load (building first if needed) the C-ABI library.  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if build_if_missing:
                from . import build as _build

                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"renderer library not built: {path}")
            L = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def exported_symbols() -> List[str]:
    return list(_SIGS)


def _check(rc: int):
    if rc != E2E_OK:
        raise E2EError(rc, load_library().e2e_last_error().decode())


# ------------------------------------------------------------------ raw C ABI (same names)


def e2e_create(device: int = 0, pool_bytes: int = 0, max_inflight: int = 0, debug_checks: int = 0,
               kernel_timing: int = 0) -> int:
    L = load_library()
    h = C.c_void_p()
    o = e2e_opts(pool_bytes, max_inflight, debug_checks, kernel_timing)
    _check(L.e2e_create(C.byref(h), device, C.byref(o)))
    return h.value


def e2e_destroy(ctx: int) -> None:
    load_library().e2e_destroy(C.c_void_p(ctx))


class _ModelDesc:
    """C view of an OpticalModel; keeps the numpy arrays alive."""

    def __init__(self, model: W.OpticalModel):
        self.keep = []
        n = len(model.slices)
        self.sl = (e2e_order_slice * max(n, 1))()
        dp = C.POINTER(C.c_double)
        for i, s in enumerate(model.slices):
            cx = np.ascontiguousarray(s.cx, dtype=np.float64)
            cy = np.ascontiguousarray(s.cy, dtype=np.float64)
            u = np.ascontiguousarray(s.slit_weights, dtype=np.float64)
            self.keep += [cx, cy, u]
            o = self.sl[i]
            o.detector, o.order, o.fiber, o.slice = s.detector, s.order, s.fiber, s.slice
            o.degree, o.K, o.n_lambda, o.n_slit = s.degree, s.K, s.n_lambda, s.n_slit
            o.lambda_lo, o.lambda_hi = s.lambda_lo, s.lambda_hi
            o.cx, o.cy, o.slit_weights = cx.ctypes.data_as(dp), cy.ctypes.data_as(dp), u.ctypes.data_as(dp)
            for p in range(3):
                o.sigma_x[p] = float(s.sigma_x[p])
                o.sigma_y[p] = float(s.sigma_y[p])
            o.theta = float(s.theta)
            o.blaze_order = float(getattr(s, "blaze_order", 0.0))
            o.blaze_lambda = float(getattr(s, "blaze_lambda", 0.0))
            o.n_aper = int(getattr(s, "n_aper", 0))
            for p in range(3):
                o.aper_x[p] = float(getattr(s, "aper_x", np.zeros(3))[p])
                o.aper_y[p] = float(getattr(s, "aper_y", np.zeros(3))[p])
            pm = getattr(s, "psf_map", None)
            if pm is not None:
                lt = np.ascontiguousarray(pm.field_lt, dtype=np.float64)
                mp = np.ascontiguousarray(pm.maps, dtype=np.float64)
                self.keep += [lt, mp]
                o.n_field, o.field_lt = len(lt), lt.ctypes.data_as(dp)
                o.map_size, o.map_oversample, o.maps = mp.shape[-1], float(pm.oversample), mp.ctypes.data_as(dp)
        nd = len(model.det_shape)
        self.h = (C.c_int32 * nd)(*[h for h, w in model.det_shape])
        self.w = (C.c_int32 * nd)(*[w for h, w in model.det_shape])
        self.desc = e2e_model_desc(nd, self.h, self.w, n, self.sl, int(model.psf))


def e2e_load_model(ctx: int, model: W.OpticalModel) -> int:
    d = _ModelDesc(model)
    mid = C.c_uint64()
    _check(load_library().e2e_load_model(C.c_void_p(ctx), C.byref(d.desc), C.byref(mid)))
    return mid.value


def e2e_unload_model(ctx: int, model_id: int) -> None:
    _check(load_library().e2e_unload_model(C.c_void_p(ctx), model_id))


def e2e_load_spectrum(ctx: int, fiber: int, orders: Sequence[int], fluxes: Sequence[np.ndarray]) -> int:
    flux = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64) for f in fluxes])
                                if len(fluxes) else np.zeros(0))
    n = len(orders)
    oid = (C.c_int32 * max(n, 1))(*orders)
    nl = (C.c_int32 * max(n, 1))(*[len(f) for f in fluxes])
    sid = C.c_uint64()
    _check(load_library().e2e_load_spectrum(C.c_void_p(ctx), fiber, n, oid, nl,
                                            flux.ctypes.data_as(C.POINTER(C.c_double)), C.byref(sid)))
    return sid.value


def e2e_unload_spectrum(ctx: int, spec_id: int) -> None:
    _check(load_library().e2e_unload_spectrum(C.c_void_p(ctx), spec_id))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def e2e_render(ctx: int, model_id: int, spec_ids: Sequence[int], precision: int, dtype: int,
               dst_ptrs: Sequence[int], pitch_elems: Optional[Sequence[int]] = None, stream=None) -> None:
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    dst = (C.c_void_p * len(dst_ptrs))(*dst_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * len(pitch_elems))(*pitch_elems)
    _check(load_library().e2e_render(C.c_void_p(ctx), model_id, n, sids, precision, dtype, dst, pit,
                                     C.c_void_p(_stream_handle(stream))))


def e2e_render_host(ctx: int, model_id: int, spec_ids: Sequence[int], precision: int, dtype: int,
                    host_ptrs: Sequence[int], pitch_elems: Optional[Sequence[int]] = None, stream=None) -> None:
    """Render into host memory, the device-to-host copy of each finished band of rows
    overlapping the render of the later bands; complete when ``stream`` is."""
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    dst = (C.c_void_p * len(host_ptrs))(*host_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * len(pitch_elems))(*pitch_elems)
    _check(load_library().e2e_render_host(C.c_void_p(ctx), model_id, n, sids, precision, dtype, dst, pit,
                                          C.c_void_p(_stream_handle(stream))))


def e2e_render_static(ctx: int, model_id: int, spec_ids: Sequence[int], dtype: int, dst_ptrs: Sequence[int],
                      pitch_elems: Optional[Sequence[int]] = None, stream=None) -> None:
    """Mixed-precision render that allocates nothing: scratch comes from the library's fixed
    device buffer (E2E_STATIC_SCRATCH_BYTES).  For callers that cannot allocate device memory
    while running; calls that overlap on the GPU share that buffer and must be serialised."""
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    dst = (C.c_void_p * len(dst_ptrs))(*dst_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * len(pitch_elems))(*pitch_elems)
    _check(load_library().e2e_render_static(C.c_void_p(ctx), model_id, n, sids, dtype, dst, pit,
                                            C.c_void_p(_stream_handle(stream))))


def e2e_render_alloc(ctx: int, model_id: int, spec_ids: Sequence[int], precision: int, dtype: int, stream=None) -> int:
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    fid = C.c_uint64()
    _check(load_library().e2e_render_alloc(C.c_void_p(ctx), model_id, n, sids, precision, dtype,
                                           C.c_void_p(_stream_handle(stream)), C.byref(fid)))
    return fid.value


def e2e_fetch_frame(ctx: int, frame_id: int, detector: int, dst_ptr: int, dst_is_device: bool, nbytes: int,
                    stream=None) -> None:
    _check(load_library().e2e_fetch_frame(C.c_void_p(ctx), frame_id, detector, C.c_void_p(dst_ptr),
                                          1 if dst_is_device else 0, nbytes, C.c_void_p(_stream_handle(stream))))


def e2e_release_frame(ctx: int, frame_id: int) -> None:
    _check(load_library().e2e_release_frame(C.c_void_p(ctx), frame_id))


def e2e_render_adjoint(ctx: int, model_id: int, spec_ids: Sequence[int], dtype: int, dldi_ptrs: Sequence[int],
                       pitch_elems: Optional[Sequence[int]], g_cx: int, g_cy: int, g_sx: int, g_sy: int,
                       frozen_windows: int = 0, stream=None) -> None:
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    dl = (C.c_void_p * len(dldi_ptrs))(*dldi_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * len(pitch_elems))(*pitch_elems)
    _check(load_library().e2e_render_adjoint(C.c_void_p(ctx), model_id, n, sids, dtype, dl, pit, C.c_void_p(g_cx),
                                             C.c_void_p(g_cy), C.c_void_p(g_sx), C.c_void_p(g_sy),
                                             C.c_void_p(frozen_windows or None),
                                             C.c_void_p(_stream_handle(stream))))


def e2e_window_origins(ctx: int, model_id: int, origins_ptr: int, stream=None) -> None:
    _check(load_library().e2e_window_origins(C.c_void_p(ctx), model_id, C.c_void_p(origins_ptr),
                                             C.c_void_p(_stream_handle(stream))))


def e2e_render_frozen(ctx: int, model_id: int, spec_ids: Sequence[int], frozen_ptr: int, dtype: int,
                      dst_ptrs: Sequence[int], pitch_elems: Optional[Sequence[int]] = None, stream=None) -> None:
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    dst = (C.c_void_p * len(dst_ptrs))(*dst_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * len(pitch_elems))(*pitch_elems)
    _check(load_library().e2e_render_frozen(C.c_void_p(ctx), model_id, n, sids, C.c_void_p(frozen_ptr), dtype, dst,
                                            pit, C.c_void_p(_stream_handle(stream))))


def e2e_update_model(ctx: int, model_id: int, cx: np.ndarray, cy: np.ndarray, sx: np.ndarray, sy: np.ndarray) -> None:
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (cx, cy, sx, sy)]
    dp = C.POINTER(C.c_double)
    _check(load_library().e2e_update_model(C.c_void_p(ctx), model_id, *[a.ctypes.data_as(dp) for a in arrs]))


# -------------------------------------------------------------------- photon Monte-Carlo


def e2e_render_photons(ctx: int, model_id: int, spec_ids: Sequence[int], seed: int, dst_ptrs: Sequence[int],
                       pitch_elems: Optional[Sequence[int]] = None, want_total: bool = True, stream=None):
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    nd = len(dst_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * nd)(*pitch_elems)
    tot = C.c_uint64()
    _check(load_library().e2e_render_photons(C.c_void_p(ctx), model_id, n, sids, seed, (C.c_void_p * nd)(*dst_ptrs),
                                             pit, C.byref(tot) if want_total else None,
                                             C.c_void_p(_stream_handle(stream))))
    return tot.value if want_total else None


# -------------------------------------------------------------------- detector noise


def e2e_add_noise(ctx: int, model_id: int, params: e2e_noise_params, src_dtype: int, src_ptrs: Sequence[int],
                  src_pitch: Optional[Sequence[int]], dst_dtype: int, dst_ptrs: Sequence[int],
                  dst_pitch: Optional[Sequence[int]], stream=None) -> None:
    n = len(src_ptrs)
    sp = None if src_pitch is None else (C.c_int64 * n)(*src_pitch)
    dp = None if dst_pitch is None else (C.c_int64 * n)(*dst_pitch)
    _check(load_library().e2e_add_noise(C.c_void_p(ctx), model_id, C.byref(params), src_dtype,
                                        (C.c_void_p * n)(*src_ptrs), sp, dst_dtype, (C.c_void_p * n)(*dst_ptrs), dp,
                                        C.c_void_p(_stream_handle(stream))))


# -------------------------------------------------------------------- serving


def e2e_server_start(ctx: int, max_inflight: int = 0, budget_bytes: int = 0, express_stamps: int = 0,
                     express_slots: int = 0) -> None:
    cfg = e2e_server_cfg(max_inflight, budget_bytes, express_stamps, express_slots)
    _check(load_library().e2e_server_start(C.c_void_p(ctx), C.byref(cfg)))


def e2e_submit(ctx: int, model_id: int, spec_ids: Sequence[int], precision: int, dtype: int,
               dst_ptrs: Optional[Sequence[int]] = None, pitch_elems: Optional[Sequence[int]] = None) -> int:
    n = len(spec_ids)
    sids = (C.c_uint64 * max(n, 1))(*spec_ids)
    dst = None if dst_ptrs is None else (C.c_void_p * len(dst_ptrs))(*dst_ptrs)
    pit = None if pitch_elems is None else (C.c_int64 * len(pitch_elems))(*pitch_elems)
    job = e2e_job(model_id, n, sids, precision, dtype, dst, pit)
    rid = C.c_uint64()
    _check(load_library().e2e_submit(C.c_void_p(ctx), C.byref(job), C.byref(rid)))
    return rid.value


def _info_dict(info: e2e_job_info) -> Dict[str, float]:
    return {name: getattr(info, name) for name, _ in e2e_job_info._fields_}


def e2e_poll(ctx: int, request_id: int) -> Dict[str, float]:
    info = e2e_job_info()
    _check(load_library().e2e_poll(C.c_void_p(ctx), request_id, C.byref(info)))
    return _info_dict(info)


def e2e_wait(ctx: int, request_id: int, timeout_ms: int = -1) -> Dict[str, float]:
    info = e2e_job_info()
    _check(load_library().e2e_wait(C.c_void_p(ctx), request_id, timeout_ms, C.byref(info)))
    return _info_dict(info)


def e2e_cancel(ctx: int, request_id: int) -> None:
    _check(load_library().e2e_cancel(C.c_void_p(ctx), request_id))


def e2e_forget(ctx: int, request_id: int) -> None:
    _check(load_library().e2e_forget(C.c_void_p(ctx), request_id))


def e2e_server_stop(ctx: int) -> None:
    _check(load_library().e2e_server_stop(C.c_void_p(ctx)))


def e2e_kernel_times(ctx: int, cap: int = 64):
    """[(kernel name, ms)] of the context's most recent render (needs kernel_timing=1)."""
    names = (C.c_char_p * cap)()
    ms = (C.c_float * cap)()
    n = C.c_int32()
    _check(load_library().e2e_kernel_times(C.c_void_p(ctx), names, ms, cap, C.byref(n)))
    return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, cap))]


def e2e_eval_tail(u_dev_ptr: int, n: int, out_dev_ptr: int, stream=None) -> None:
    """out[i] = the renderer's FP32 erfc(|u[i]|) (device pointers to n doubles / n floats)."""
    rc = load_library().e2e_eval_tail(C.c_void_p(u_dev_ptr), n, C.c_void_p(out_dev_ptr),
                                      C.c_void_p(_stream_handle(stream)))
    if rc != E2E_OK:
        raise E2EError(rc, "e2e_eval_tail failed")


def e2e_eval_tail_far(u_dev_ptr: int, n: int, out_dev_ptr: int, stream=None) -> None:
    """out[i] = the renderer's cheaper FP32 erfc(|u[i]|) of narrow PSFs' tail edges, for
    |u[i]| >= 0.333 (device pointers to n doubles / n floats)."""
    rc = load_library().e2e_eval_tail_far(C.c_void_p(u_dev_ptr), n, C.c_void_p(out_dev_ptr),
                                          C.c_void_p(_stream_handle(stream)))
    if rc != E2E_OK:
        raise E2EError(rc, "e2e_eval_tail_far failed")


def e2e_fma_probe(fp64: bool, blocks: int, iters: int, sink_dev_ptr: int, stream=None) -> int:
    """Launch the FMA-rate probe (blocks x 256 threads x 8 chains x iters FMAs); returns the FMA count."""
    n = C.c_int64()
    rc = load_library().e2e_fma_probe(1 if fp64 else 0, blocks, iters, C.c_void_p(sink_dev_ptr), C.byref(n),
                                      C.c_void_p(_stream_handle(stream)))
    if rc != E2E_OK:
        raise E2EError(rc, "e2e_fma_probe failed")
    return n.value


def e2e_model_plan(ctx: int, model_id: int) -> Dict[str, int]:
    info = e2e_plan_info()
    _check(load_library().e2e_model_plan(C.c_void_p(ctx), model_id, C.byref(info)))
    return {name: getattr(info, name) for name, _ in e2e_plan_info._fields_}


# ------------------------------------------------------------------ convenience layer


class Renderer:
    """A context on one GPU holding resident models and spectra.

    >>> r = Renderer()
    >>> mid = r.load_model(workload.model)
    >>> sids = r.load_spectra(workload)
    >>> frames = r.render(mid, sids, "mixed", "f32")   # list of torch tensors, one per detector
    """

    def __init__(self, device: int = 0, pool_bytes: int = 0, max_inflight: int = 0, debug_checks: int = 0,
                 kernel_timing: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the renderer needs a CUDA GPU; there is no CPU fallback")
        self.device = device
        self.ctx = e2e_create(device, pool_bytes, max_inflight, debug_checks, kernel_timing)
        self.models: Dict[int, W.OpticalModel] = {}

    def close(self):
        if self.ctx:
            e2e_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_model(self, model: W.OpticalModel) -> int:
        mid = e2e_load_model(self.ctx, model)
        self.models[mid] = model
        return mid

    def unload_model(self, mid: int):
        e2e_unload_model(self.ctx, mid)
        self.models.pop(mid, None)

    def load_spectrum(self, spectrum: W.Spectrum) -> int:
        orders = sorted(spectrum.flux)
        return e2e_load_spectrum(self.ctx, spectrum.fiber, orders, [spectrum.flux[o] for o in orders])

    def load_spectra(self, workload: W.Workload) -> List[int]:
        return [self.load_spectrum(workload.spectra[f]) for f in sorted(workload.spectra)]

    def plan(self, mid: int) -> Dict[str, int]:
        return e2e_model_plan(self.ctx, mid)

    def empty_frames(self, mid: int, dtype: str = "f32"):
        import torch

        td = torch.float32 if dtype == "f32" else torch.float64
        return [torch.empty((h, w), dtype=td, device=f"cuda:{self.device}") for h, w in self.models[mid].det_shape]

    def render_host(self, mid: int, spec_ids: Sequence[int], precision: str = "mixed", dtype: str = "f32",
                    out=None, stream=None, sync: bool = True):
        """Frames rendered into page-locked host tensors (allocated when ``out`` is None), the
        copies overlapping the render; waits for ``stream`` unless ``sync`` is False."""
        import torch

        if out is None:
            td = torch.float32 if dtype == "f32" else torch.float64
            out = [torch.empty((h, w), dtype=td).pin_memory() for h, w in self.models[mid].det_shape]
        e2e_render_host(self.ctx, mid, spec_ids, PRECISION[precision], DTYPE[dtype],
                        [int(t.data_ptr()) for t in out], [int(t.stride(0)) for t in out], stream)
        if sync:
            if stream is None:
                torch.cuda.current_stream(self.device).synchronize()
            elif hasattr(stream, "synchronize"):
                stream.synchronize()
            elif stream:
                torch.cuda.ExternalStream(stream).synchronize()
            else:
                torch.cuda.synchronize(self.device)
        return out

    # -------------------------------------------------------------- photon Monte-Carlo
    def render_photons(self, mid: int, spec_ids: Sequence[int], seed: int, out=None, stream=None,
                       want_total: bool = True):
        """Photon-by-photon frames (int32 tensors holding the uint32 counts) and the photon total."""
        import torch

        if out is None:
            out = [torch.empty((h, w), dtype=torch.int32, device=f"cuda:{self.device}")
                   for h, w in self.models[mid].det_shape]
        total = e2e_render_photons(self.ctx, mid, spec_ids, seed, [int(t.data_ptr()) for t in out],
                                   [int(t.stride(0)) for t in out], want_total, stream)
        return out, total

    # -------------------------------------------------------------- detector noise
    def add_noise(self, mid: int, frames, dtype: str = "f32", out=None, stream=None, *, seed: int,
                  pattern_seed: int = 1, dark_e: float = 0.0, prnu: float = 0.0, ron_e: float = 0.0,
                  xtalk: float = 0.0, gain: float = 1.0, bias: float = 0.0, saturation: int = 65535,
                  poisson: bool = True):
        """Noise stage on rendered frames (see e2e_add_noise); dtype "f32"/"f64" (electrons)
        or "u16" (ADU).  out defaults to new frames; out=frames applies it in place."""
        import torch

        if out is None:
            td = {"f32": torch.float32, "f64": torch.float64, "u16": torch.uint16}[dtype]
            out = [torch.empty(f.shape, dtype=td, device=f.device) for f in frames]
        p = e2e_noise_params(seed, pattern_seed, dark_e, prnu, ron_e, xtalk, gain, bias, saturation,
                             1 if poisson else 0)
        sdt = E2E_F32 if frames[0].dtype == torch.float32 else E2E_F64
        e2e_add_noise(self.ctx, mid, p, sdt, [int(f.data_ptr()) for f in frames], [int(f.stride(0)) for f in frames],
                      {"f32": E2E_F32, "f64": E2E_F64, "u16": E2E_U16}[dtype], [int(t.data_ptr()) for t in out],
                      [int(t.stride(0)) for t in out], stream)
        return out

    # -------------------------------------------------------------- differentiation
    def params(self, mid: int):
        """(cx, cy, sx, sy) of the model, concatenated per order-slice (the adjoint's layout)."""
        m = self.models[mid]
        return (np.concatenate([s.cx for s in m.slices]) if m.slices else np.zeros(0),
                np.concatenate([s.cy for s in m.slices]) if m.slices else np.zeros(0),
                np.concatenate([s.sigma_x for s in m.slices]) if m.slices else np.zeros(0),
                np.concatenate([s.sigma_y for s in m.slices]) if m.slices else np.zeros(0))

    def update(self, mid: int, cx, cy, sx, sy) -> None:
        """Replace the model's coefficients on the device (re-plans) and in the host copy."""
        e2e_update_model(self.ctx, mid, cx, cy, sx, sy)
        m = self.models[mid].copy()
        o = 0
        for i, s in enumerate(m.slices):
            nc = W.n_coeffs(s.degree)
            s.cx = np.array(cx[o:o + nc], dtype=np.float64)
            s.cy = np.array(cy[o:o + nc], dtype=np.float64)
            s.sigma_x = np.array(sx[3 * i:3 * i + 3], dtype=np.float64)
            s.sigma_y = np.array(sy[3 * i:3 * i + 3], dtype=np.float64)
            o += nc
        self.models[mid] = m

    def adjoint(self, mid: int, spec_ids: Sequence[int], dldi, stream=None, frozen=None):
        """(g_cx, g_cy, g_sx, g_sy) device FP64 tensors: sum over pixels of dL/dI * dI/dtheta;
        frozen: optional int32 device tensor of window origins (window_origins' layout)."""
        import torch

        m = self.models[mid]
        nc = sum(W.n_coeffs(s.degree) for s in m.slices)
        dev = f"cuda:{self.device}"
        g = [torch.empty(n, dtype=torch.float64, device=dev) for n in (nc, nc, 3 * len(m.slices), 3 * len(m.slices))]
        dt = E2E_F32 if dldi[0].dtype == torch.float32 else E2E_F64
        e2e_render_adjoint(self.ctx, mid, spec_ids, dt, [int(t.data_ptr()) for t in dldi],
                           [int(t.stride(0)) for t in dldi], *[int(t.data_ptr()) for t in g],
                           frozen_windows=0 if frozen is None else int(frozen.data_ptr()), stream=stream)
        return tuple(g)

    def window_origins(self, mid: int, stream=None):
        """int32 device tensor (n_stamps, 2): every stamp's window origin (i0, r0)."""
        import torch

        m = self.models[mid]
        out = torch.empty((m.n_stamps, 2), dtype=torch.int32, device=f"cuda:{self.device}")
        e2e_window_origins(self.ctx, mid, int(out.data_ptr()), stream)
        return out

    def render_frozen(self, mid: int, spec_ids: Sequence[int], frozen, dtype: str = "f64", out=None, stream=None):
        """FP64 render with every window held at the origins in `frozen` (window_origins' layout)."""
        if out is None:
            out = self.empty_frames(mid, dtype)
        e2e_render_frozen(self.ctx, mid, spec_ids, int(frozen.data_ptr()), DTYPE[dtype],
                          [int(t.data_ptr()) for t in out], [int(t.stride(0)) for t in out], stream)
        return out

    def render(self, mid: int, spec_ids: Sequence[int], precision: str = "mixed", dtype: str = "f32",
               out=None, stream=None):
        if out is None:
            out = self.empty_frames(mid, dtype)
        pitches = [int(t.stride(0)) for t in out]
        e2e_render(self.ctx, mid, spec_ids, PRECISION[precision], DTYPE[dtype], [int(t.data_ptr()) for t in out],
                   pitches, stream)
        return out


class Server:
    """Continuous-batching request loop on a Renderer's context (see e2e_server_start)."""

    def __init__(self, renderer: Renderer, max_inflight: int = 4, budget_bytes: int = 0, express_stamps: int = 0,
                 express_slots: int = 0):
        self.r = renderer
        e2e_server_start(renderer.ctx, max_inflight, budget_bytes, express_stamps, express_slots)
        self._keep: Dict[int, object] = {}

    def submit(self, mid: int, spec_ids: Sequence[int], precision: str = "mixed", dtype: str = "f32", out=None) -> int:
        ptrs = None if out is None else [int(t.data_ptr()) for t in out]
        pitches = None if out is None else [int(t.stride(0)) for t in out]
        rid = e2e_submit(self.r.ctx, mid, spec_ids, PRECISION[precision], DTYPE[dtype], ptrs, pitches)
        if out is not None:
            self._keep[rid] = out  # the frames must outlive the job
        return rid

    def poll(self, rid: int):
        return e2e_poll(self.r.ctx, rid)

    def wait(self, rid: int, timeout_ms: int = -1):
        info = e2e_wait(self.r.ctx, rid, timeout_ms)
        self._keep.pop(rid, None)
        return info

    def cancel(self, rid: int):
        e2e_cancel(self.r.ctx, rid)

    def forget(self, rid: int):
        e2e_forget(self.r.ctx, rid)

    def stop(self):
        e2e_server_stop(self.r.ctx)
        self._keep.clear()
