#!/usr/bin/env python
"""Benchmark: PSF stamps rendered per second on the full single-detector frame workload.

Workload: 9216 x 9216 FP32 frame, 85 orders x 2 fibers x 2 slices, 6000 wavelength samples x
64 slit points per order-slice, degree-5 polynomials, field-varying Gaussian PSF (sigma
1.2-2.0 px), 11 x 11 stamps; science fiber = continuum + 20000 lines, reference fiber =
Fabry-Perot comb (seeded synthetic stand-ins for an ESPRESSO/HIRES-class echellogram).

One step = one render of the whole frame (mapping, PSF stamps, on-chip accumulation, tile
merge, frame write) through the C ABI.  ``value`` is stamps/s with the model and spectra
resident in HBM, timed with CUDA events on the render stream; L2 is flushed between steps
(a 256 MiB memset outside the timed events).  ``e2e`` is the same metric through the public
API from pinned host memory: per step the spectra are uploaded (e2e_load_spectrum), the
frame is rendered into pinned host memory (e2e_render_host: bands of rows are copied out as
they finish, overlapping the render of the later bands) and the spectra are unloaded; steps
are pipelined as a streaming caller runs them (the next step's upload overlaps this render).

Accuracy: every leg that times a renderer carries the error of what it rendered against the
FP64 oracle (per-pixel relative error, the tolerance's worst excess, photocenter shifts of
16 x 16 px windows, window-rule ties): the headline on six seeded 64 x 64 windows of the timed
frame, the other legs on a cut sample.  The oracle runs only in these CPU-baseline legs, where
it is also timed as the baseline.  Other legs: the plain single-fiber case (config 1), the
elliptical PSF, tabulated PSF, adjoint, detector noise, photon Monte-Carlo and serving, and an
FMA probe that measures the FP32 and FP64 pipes the roofline is quoted against.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (one step renders a
bounded sample of the same workload: its first order-slices, one per host core).  Under torchrun each rank renders its own detector frame
(independent frames, no collective: weak scaling), or with ``--shard band`` its band of rows of
one frame (halo stamps rendered by both neighbours, no collective: strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2008_05858_gb300 import workloads as W  # noqa: E402

METRIC = "PSF stamps/s at <1e-5 px photocenter err, mixed vs FP64; p99 render latency"
UNIT = "stamps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 FLOP of one separable stamp of window K and degree d, counted algorithmically (an FMA
# is 2 FLOP, an SFU operation 1): 2(K+1) pixel-edge tail evaluations at 28 FLOP each (the
# double-float edge argument: 6; its exact square: 3; the exponential: 1 + 2; the (4,5)
# rational: 18 - 2 = 16, with its reciprocal), 2K edge differences, the K^2 products with the
# weight folded in, accumulated by FMA (2 K^2), and the mapping's Horner in s of both
# coordinates (2d FMAs; evaluated in double-float FP32 arithmetic, counted once).
def fp32_flop_per_stamp(K: int, d: int = 5) -> float:
    return 2 * (K + 1) * 28 + 2 * K + 2 * K * K + 4 * d


# FP64 FMAs of one stamp: the per-sample Horner in lambda of the coefficients of s (2 n_c per
# wavelength sample, spread over the n_slit stamps of the sample); the rest of the mapping runs
# in double-float FP32 arithmetic.
def fp64_fma_per_stamp(d: int, n_slit: int) -> float:
    nc = (d + 1) * (d + 2) / 2
    return 2 * nc / n_slit


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # let the sampler start before the timed region
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ accuracy (oracle legs)
#
# The stamps/s figures count only frames that meet the accuracy target, so every leg that
# times a renderer also compares what it rendered with the FP64 oracle.  The oracle runs only
# inside these CPU-baseline legs (it is timed there as the baseline too), on a bounded sample.


def _poly2(c, degree, lt, s):
    """x or y of a slice's mapping on the grid lt x s (a plain evaluation for choosing windows)."""
    out = np.zeros((len(lt), len(s)))
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            out += c[W.coeff_index(a, b)] * np.outer(lt ** a, s ** b)
    return out


def _summarise(reps):
    """Worst figures over a list of framecompare reports."""
    return {"max_rel": max(r.max_rel for r in reps), "worst_excess": max(r.worst_excess for r in reps),
            "bad_pixels": sum(r.n_bad for r in reps),
            "photocenter_dx_px": max(r.photocenter_dx for r in reps),
            "photocenter_dy_px": max(r.photocenter_dy for r in reps),
            "photocenter_windows": sum(r.n_windows for r in reps),
            "window_ties": sum(r.n_ties for r in reps), "flip_pixels": sum(r.n_flip_px for r in reps),
            "ok": all(r.ok for r in reps),
            "bound": "|g-o| <= 1e-6 |o| + 1e-10 max|o| per pixel; photocenter of 16x16 px windows < 1e-5 px"}


def frame_windows_oracle(w: W.Workload, frame: np.ndarray, n_win: int = 6, size: int = 64, seed: int = 2008):
    """The CPU-baseline leg of the headline: the oracle renders n_win seeded size x size windows
    on the traces of the timed frame (each window one detector of a model holding every slice
    whose trace comes within reach of it, translated so the window is that detector), timed as
    the baseline, and the windows of the GPU frame are compared with them."""
    import oracle
    from tests.framecompare import compare, tie_boxes

    H, Wd = w.model.det_shape[0]
    lt, ss = np.linspace(-1.0, 1.0, 513), np.linspace(-1.0, 1.0, 9)
    yr = [(_poly2(s.cy, s.degree, lt, ss).min(), _poly2(s.cy, s.degree, lt, ss).max()) for s in w.model.slices]
    rng = np.random.default_rng(seed)
    wins, sub, src = [], [], {}
    for d in range(n_win):
        s = w.model.slices[int(rng.integers(len(w.model.slices)))]
        t = rng.uniform(-0.95, 0.95)
        xc = float(_poly2(s.cx, s.degree, np.array([t]), np.array([0.0]))[0, 0])
        yc = float(_poly2(s.cy, s.degree, np.array([t]), np.array([0.0]))[0, 0])
        x0 = int(min(max(round(xc) - size // 2, 0), Wd - size))
        y0 = int(min(max(round(yc) - size // 2, 0), H - size))
        wins.append((x0, y0))
        for q, (lo, hi) in zip(w.model.slices, yr):
            if hi + 2 + q.K >= y0 and lo - 2 - q.K <= y0 + size:
                c = q.copy()
                c.cx[0] -= x0
                c.cy[0] -= y0
                c.detector = d
                src[id(c)] = q
                sub.append(c)
    model = W.OpticalModel([(size, size)] * n_win, sub, w.model.psf)
    flux_of = lambda c: w.flux_for(src[id(c)])  # noqa: E731
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = oracle.render(model, flux_of, n_threads=cores)
    dt = time.perf_counter() - t0
    ties = tie_boxes(model, flux_of)
    reps = [compare(frame[y0:y0 + size, x0:x0 + size], ref[d], ties=ties[d]) for d, (x0, y0) in enumerate(wins)]
    acc = _summarise(reps)
    acc.update(windows=[list(p) for p in wins], window_px=size, source="cpu_baseline leg (oracle windows)")
    stamps = model.n_stamps
    base = {"value": stamps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(sub)} order-slices ({stamps} stamps) reaching {n_win} seeded {size}x{size} windows of "
                      f"the timed frame, each rendered in full and clipped to its window, FP64, {dt:.1f} s"}
    return base, acc


def cut_model(w: W.Workload, n_slices: int, n_slit: int, model=None):
    """The first n_slices order-slices of w (or of `model`), each with its wavelength grid and
    geometry kept but only n_slit slit points (bin centres of [-1, 1], uniform weights of the
    same total), and a flux lookup for them."""
    import dataclasses

    m = w.model if model is None else model
    cut, flux = [], {}
    for s in m.slices[:n_slices]:
        k = min(n_slit, s.n_slit)
        tot = float(np.sum(s.slit_weights))
        c = dataclasses.replace(s.copy(), n_slit=k, slit_weights=np.full(k, tot / k))
        flux[id(c)] = w.flux_for(s)
        cut.append(c)
    return W.OpticalModel(m.det_shape, cut, m.psf), (lambda c: flux[id(c)])


def cut_sample_oracle(B, dev, w: W.Workload, model, n_slices: int, n_slit: int, precisions=("mixed",)):
    """CPU-baseline leg on a cut sample (cut_model): the oracle renders it (timed as the
    baseline) and the GPU renders of the same sample are compared with it, per precision.
    Comparisons run on the rows and columns the sample touches (16-px aligned, so the
    photocenter windows are the frame's own)."""
    import torch

    import oracle
    from tests.framecompare import compare, tie_boxes

    sub, flux_of = cut_model(w, n_slices, n_slit, model)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = oracle.render(sub, flux_of, n_threads=cores)
    dt = time.perf_counter() - t0
    ties = tie_boxes(sub, flux_of)
    r = B.Renderer(dev)
    acc = {}
    try:
        mid = r.load_model(sub)
        sids = []
        for f in sorted({s.fiber for s in sub.slices}):
            orders = {s.order: flux_of(s) for s in sub.slices if s.fiber == f}
            sids.append(r.load_spectrum(W.Spectrum(f, orders)))
        for prec in precisions:
            got = r.render(mid, sids, prec, "f32" if prec == "mixed" else "f64")
            torch.cuda.synchronize()
            reps = []
            for d, (g, o) in enumerate(zip(got, ref)):
                nz = np.nonzero(o)
                if len(nz[0]) == 0:
                    continue
                y0, y1 = nz[0].min() // 16 * 16, min(o.shape[0], (nz[0].max() // 16 + 2) * 16)
                x0, x1 = nz[1].min() // 16 * 16, min(o.shape[1], (nz[1].max() // 16 + 2) * 16)
                bx = [(a - x0, b - x0, c - y0, e - y0) for a, b, c, e in ties[d]]
                reps.append(compare(g[y0:y1, x0:x1].double().cpu().numpy(), o[y0:y1, x0:x1], ties=bx))
            acc[prec] = _summarise(reps)
            if prec == "fp64":
                acc[prec]["bound"] = "FP64 renderer: reported against the 1e-6 bound (its own tests hold it to 5e-11)"
    finally:
        r.close()
    stamps = sub.n_stamps
    base = {"value": stamps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {len(sub.slices)} of {len(model.slices)} order-slices, each with its full wavelength grid "
                      f"and {n_slit} slit points ({stamps} stamps), FP64, {dt:.1f} s"}
    return base, acc


def headline_config(w: W.Workload, K: int, stamps: int, world: int, band: bool) -> dict:
    """`config` of the headline line, shared by both arms: the workload the metric is quoted on
    and how its steps are run."""
    return {"workload": w.name, "frame": "9216x9216 f32", "orders": 85, "fibers": 2, "slices": 2,
            "n_lambda": 6000, "n_slit": 64, "degree": 5, "K": K, "stamps_per_frame": stamps,
            "l2": "flushed between steps (256 MiB memset outside the timed events)",
            "parallelism": f"row bands of one frame x{world}" if band else f"independent frame per GPU x{world}"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on the headline's workload and
    config.  One step renders a bounded sample of that workload -- its first order-slices in
    full, one per host core (up to 16) -- and the line reports that sample's own time per step
    and stamps/s, the sample named in `sample` and `cpu_baseline`."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    w = W.config2()
    cores = os.cpu_count() or 1
    n = max(1, min(16, cores, len(w.model.slices)))
    sub = W.OpticalModel(w.model.det_shape, w.model.slices[:n], w.model.psf)
    stamps = sub.n_stamps
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.render(sub, w.flux_for, n_threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = statistics.median(times)
    value = stamps / t
    sample = (f"first {n} of {len(w.model.slices)} order-slices of {w.name} in full ({stamps} stamps per step), "
              f"FP64, median {t:.2f} s per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(w, w.model.slices[0].K, w.model.n_stamps, world, args.shard == "band" and world > 1),
        "sample": sample, "stamps_per_step": stamps,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    from paper_2008_05858_gb300 import binding as B
    from paper_2008_05858_gb300 import shard

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    # --shard frame: one independent full frame per rank (weak scaling); --shard band: the ranks
    # split one frame into bands of rows, halo stamps rendered by both neighbours (strong)
    band = args.shard == "band" and world > 1
    w = W.config2(seed=W.SEED_BASE + 2 + rank * 1000 if rank and not band else None)
    stamps = w.model.n_stamps  # of the whole frame, counted once
    if band:
        w, _ = shard.shard_workload_by_band(w, rank, world)
    frames_per_step = 1 if band else world
    stamps_rank = stamps / world if band else stamps  # this rank's share (halo work not counted)
    K = w.model.slices[0].K
    r = B.Renderer(dev, kernel_timing=1)
    mid = r.load_model(w.model)
    sids = r.load_spectra(w)
    plan = r.plan(mid)
    frame = r.empty_frames(mid, "f32")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(prec="mixed"):
        r.render(mid, sids, prec, "f32", out=frame, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern = {}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            for name, ms in B.e2e_kernel_times(r.ctx):
                kern.setdefault(name, []).append(ms)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = shard.reduce_over_ranks(total_ms, "max")
    ms_per_step = total_ms / args.steps
    value = stamps * frames_per_step / (ms_per_step * 1e-3)
    clocks = clk.summary()

    # plain FP64 renderer on the same frame (side by side, fewer steps: it is slow)
    fp64_ms = []
    step("fp64")
    torch.cuda.synchronize()
    for _ in range(max(1, min(3, args.steps))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step("fp64")
        b.record(stream)
        torch.cuda.synchronize()
        fp64_ms.append(a.elapsed_time(b))
    fp64_value = stamps_rank / (statistics.median(fp64_ms) * 1e-3)

    # end to end through the public API from pinned host memory
    pinned = {}
    for f, sp in w.spectra.items():
        orders = sorted(sp.flux)
        cat = torch.from_numpy(np.concatenate([np.asarray(sp.flux[o], dtype=np.float64) for o in orders]))
        pinned[f] = (orders, [len(sp.flux[o]) for o in orders], cat.pin_memory())
    h, wd = w.model.det_shape[0]
    host_frame = torch.empty((h, wd), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 8 for _, _, t in pinned.values())
    d2h = host_frame.numel() * 4

    def load_ids():
        return [_load_spectrum_ptr(B, r.ctx, f, orders, lens, flux) for f, (orders, lens, flux) in pinned.items()]

    def e2e_steps(n):
        """n steps, pipelined as a streaming caller would run them: step k's frame is rendered
        into pinned host memory (each finished band of rows copied while later bands still
        render), and while it renders step k + 1's spectra are uploaded and checked; step k's
        spectra are unloaded once its frame is on the host."""
        ids = load_ids()
        for k in range(n):
            B.e2e_render_host(r.ctx, mid, ids, B.E2E_PREC_MIXED, B.E2E_F32, [host_frame.data_ptr()], None, stream)
            nxt = load_ids() if k + 1 < n else None
            stream.synchronize()
            for i in ids:
                B.e2e_unload_spectrum(r.ctx, i)
            ids = nxt

    e2e_steps(2)
    n_e2e = max(1, min(5, args.steps))
    e2e_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_steps(n_e2e)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b) / n_e2e)
    e2e_value = shard.reduce_over_ranks(statistics.median(e2e_ms), "max")
    e2e_value = stamps * frames_per_step / (e2e_value * 1e-3)

    peaks, peak_kind = _peaks()
    mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    kr = statistics.median(kern.get("render_mixed", [float("nan")]))
    # the tiles no item overlaps are zeroed by extra CTAs of the render launch (a separate
    # launch only for a model without items); the rest merge inside the render
    km = statistics.median(kern["merge_zero"]) if "merge_zero" in kern else 0.0
    d = w.model.slices[0].degree
    ns = w.model.slices[0].n_slit
    # peaks from unit counts and the sampled clock: 128 FP32 lanes per SM; FP64 from the
    # part's nominal 1.25 TFLOP/s at 2070 MHz over 152 SMs (1.99 DFMA per clock per SM); an FMA
    # is 2 FLOP.  The FMA probe's measured rates are reported beside them.
    dfma_per_clk_sm = 1.25e12 / (2 * 152 * 2070e6)
    fp32_peak = n_sm * 128 * 2 * mhz * 1e6
    fp64_peak = n_sm * dfma_per_clk_sm * 2 * mhz * 1e6
    probe = pipe_rates(B, dev)
    a32 = fp32_flop_per_stamp(K, d) * stamps_rank / (kr * 1e-3)
    a64 = fp64_fma_per_stamp(d, ns) * 2 * stamps_rank / (kr * 1e-3)
    traffic = _load_traffic()
    roof32 = {"bound": "alu", "achieved": a32 / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
              "frac": a32 / fp32_peak, "traffic": traffic,
              "kernel": "render_mixed", "pipe": "fp32", "kernel_ms": kr,
              "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (median SM clock under load)"}
    roof64 = {"bound": "alu", "achieved": a64 / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
              "frac": a64 / fp64_peak, "traffic": traffic, "kernel": "render_mixed", "pipe": "fp64", "kernel_ms": kr,
              "peak_basis": f"{n_sm} SMs x {dfma_per_clk_sm:.2f} DFMA/clk (nominal 1.25 TFLOP/s at 2070 MHz) x 2 x "
                            f"{mhz:.0f} MHz"}
    roof32["probe_tflops"] = probe["fp32"]["tflops"]
    roof32["frac_of_probe"] = a32 / (probe["fp32"]["tflops"] * 1e12)
    roof64["probe_tflops"] = probe["fp64"]["tflops"]
    roof64["frac_of_probe"] = a64 / (probe["fp64"]["tflops"] * 1e12)
    roof = roof32 if roof32["frac"] >= roof64["frac"] else roof64
    other = roof64 if roof is roof32 else roof32
    launches_per_step = sum(1 for _ in kern)  # distinct kernels per render
    n_launch = sum(len(v) for v in kern.values())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if band else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(w, K, stamps, world, band),
        "precision": ("mixed (FP64 per-sample mapping coefficients, double-float FP32 mapping in s; "
                      "FP32 stamps from double-float edge arguments; FP32 run sums of <= 16 stamps; "
                      "exact 52-bit fixed-point item boxes; TwoSum merge of FP32 pairs)"),
        "plan": plan,
        "roofline": roof, "roofline_other_pipe": other,
        "fp64_renderer": {"value": fp64_value, "unit": UNIT, "ms_per_step": statistics.median(fp64_ms),
                          "speedup_mixed_over_fp64": statistics.median(fp64_ms) / ms_per_step},
        "kernel_ms": {"render_mixed (with the fused tile merge and the zero tiles)": kr, "merge_zero_tiles": km},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.median(e2e_ms), "steps": n_e2e,
                "note": "spectra upload + render into pinned host memory + unload per step, the next step's "
                        "upload overlapping this render"},
        "gpu_launches": n_launch,
        "launches_per_step": launches_per_step,
        "clocks": clocks, "peak_source": peak_kind, "wall_s_timed": t_wall,
        "fma_probe": probe,
    }
    line["config1"] = config1_run(B, dev, flush, cpu_baseline=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if not args.no_noise:
        line["noise"] = noise_run(B, r, mid, frame, stream, flush)
    if not args.no_photons:
        line["photon_mc"] = photon_run(B, r, mid, sids, w, stream, flush, kr + km)
    if not args.no_table:
        line["psf_table"] = table_run(B, dev, w, flush, cpu_baseline=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if not args.no_adjoint:
        line["adjoint"] = adjoint_run(B, dev, flush, cpu_baseline=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if not args.no_elliptical:
        line["elliptical"] = elliptical_run(B, dev, rank, world,
                                            cpu_baseline=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if not args.no_serving:
        line["serving"] = serving_run(B, dev)
        line["p99_latency_ms"] = line["serving"]["poisson"]["latency_ms"]["p99"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r.render(mid, sids, "mixed", "f32", out=frame, stream=stream)  # the timed step's frame
        host = frame[0].cpu().numpy()
        line["cpu_baseline"], line["accuracy"] = frame_windows_oracle(w, host)
        del host
    if rank == 0:
        print(json.dumps(line), flush=True)
    r.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def config1_run(B, dev, flush, reps=20, cpu_baseline=False):
    """The plain method's single-fiber case (one order, one fiber, 1024 x 256, 2000 x 16
    samples, degree 3, sigma 1.5, K = 7): the plain FP64 renderer and the mixed form, timed with
    CUDA events (a launch-latency-sized frame), and both compared with the oracle."""
    import torch

    w = W.config1()
    r = B.Renderer(dev)
    out = {"workload": w.name, "stamps": w.model.n_stamps, "frame": "1024x256"}
    try:
        mid = r.load_model(w.model)
        sids = r.load_spectra(w)
        st = torch.cuda.current_stream()
        frames = {}
        for prec, dt in (("fp64", "f64"), ("mixed", "f32")):
            fr = r.render(mid, sids, prec, dt, stream=st)
            ms = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                r.render(mid, sids, prec, dt, out=fr, stream=st)
                b.record(st)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            t = statistics.median(ms)
            out[prec] = {"ms_per_render": t, "value": w.model.n_stamps / (t * 1e-3), "unit": UNIT}
            frames[prec] = fr[0].double().cpu().numpy()
        out["speedup_mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    finally:
        r.close()
    if cpu_baseline:
        import oracle
        from tests.framecompare import compare, tie_boxes

        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ref = oracle.render_workload(w, n_threads=cores)[0]
        dt = time.perf_counter() - t0
        ties = tie_boxes(w.model, w.flux_for)[0]
        out["cpu_baseline"] = {"value": w.model.n_stamps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"the whole frame ({w.model.n_stamps} stamps), FP64, {dt:.2f} s"}
        out["accuracy"] = {k: _summarise([compare(frames[k], ref, ties=ties)]) for k in ("mixed", "fp64")}
        err = np.abs(frames["fp64"] - ref)
        out["accuracy"]["fp64"]["max_rel_all_pixels"] = float(np.max(err[ref > 0] / ref[ref > 0]))
    return out


def pipe_rates(B, dev, reps=3):
    """FMA rates of the FP32 and FP64 pipes, measured with the library's FMA probe (8 CTAs of
    256 threads per SM, 8 independent chains per thread), best of `reps` CUDA-event timings."""
    import torch

    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = n_sm * 8
    out = {}
    for name, fp64, iters, td in (("fp32", False, 100000, torch.float32), ("fp64", True, 2000, torch.float64)):
        sink = torch.empty(blocks * 256, dtype=td, device="cuda")
        st = torch.cuda.current_stream()
        B.e2e_fma_probe(fp64, blocks, iters, sink.data_ptr(), st)
        best = float("inf")
        n = 0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            n = B.e2e_fma_probe(fp64, blocks, iters, sink.data_ptr(), st)
            b.record(st)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        rate = n / (best * 1e-3)
        out[name] = {"fma_per_s": rate, "tflops": 2 * rate / 1e12, "ms": best, "fmas": n}
    return out


def photon_run(B, r, mid, sids, w, stream, flush, stamp_ms, reps=3):
    """The photon Monte-Carlo renderer on the full-detector model, its spectra scaled to
    1e7 ... 1e11 expected photons: photons/s, and the photon count at which it costs what
    one stamp render of the frame costs."""
    import torch

    from paper_2008_05858_gb300 import binding as Bd

    tot = sum(float(np.sum(w.flux_for(s))) * (s.lambda_hi - s.lambda_lo) / s.n_lambda * float(np.sum(s.slit_weights))
              for s in w.model.slices)
    out = r.render_photons(mid, sids, seed=7, stream=stream, want_total=False)[0]
    rows = []
    for target in (1e7, 1e8, 1e9, 1e10, 1e11):
        k = target / tot
        n_rep = reps if target < 1e11 else 1
        ids = []
        for f, sp in w.spectra.items():
            ids.append(r.load_spectrum(Bd_spec(sp, k)))
        _, n = r.render_photons(mid, ids, seed=7, out=out, stream=stream)
        ms = []
        for _ in range(n_rep):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r.render_photons(mid, ids, seed=7, out=out, stream=stream, want_total=False)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        for i in ids:
            Bd.e2e_unload_spectrum(r.ctx, i)
        t = statistics.median(ms)
        rows.append({"photons": n, "ms": t, "photons_per_s": n / (t * 1e-3)})
    # photon count at which a photon render costs one stamp render: log-log interpolation
    # between the two runs around the stamp render's time
    eq = None
    for r0, r1 in zip(rows, rows[1:]):
        if r0["ms"] <= stamp_ms <= r1["ms"]:
            f = (np.log(stamp_ms) - np.log(r0["ms"])) / (np.log(r1["ms"]) - np.log(r0["ms"]))
            eq = float(np.exp(np.log(r0["photons"]) + f * (np.log(r1["photons"]) - np.log(r0["photons"]))))
    return {"runs": rows, "stamp_render_ms": stamp_ms,
            "photons_at_equal_cost": eq,
            "note": "photon Monte-Carlo (Sec. 2.2 alternative): FP32 mapping from per-bin FP64 anchors and FP32 Box-Muller, each pixel decision bounded, FP64 redo when too close; bit-exact counts"}


def Bd_spec(sp, k):
    return W.Spectrum(sp.fiber, {o: f * k for o, f in sp.flux.items()})


def table_run(B, dev, w, flush, reps=3, cpu_baseline=False):
    """The full-detector workload with tabulated PSF maps (5 field nodes per slice, 10 samples
    per pixel over +-8 px, a 20 % comatic tail; exact per-cell phase biquadratics): mixed
    precision and the plain FP64 renderer, timed with CUDA events."""
    import torch

    m = W.with_psf_maps(w.model, oversample=10.0, half_px=8.0, coma=0.2)
    r = B.Renderer(dev)
    t0 = time.perf_counter()
    mid = r.load_model(m)
    load_s = time.perf_counter() - t0
    sids = r.load_spectra(w)
    st = torch.cuda.current_stream()
    out = {}
    for prec, n in (("mixed", reps), ("fp64", 1)):
        frames = r.render(mid, sids, prec, "f32", stream=st)
        ms = []
        for _ in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            r.render(mid, sids, prec, "f32", out=frames, stream=st)
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.median(ms)
        out[prec] = {"ms_per_render": t, "value": m.n_stamps / (t * 1e-3), "unit": UNIT}
    out["speedup_mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["model_load_s"] = load_s
    r.close()
    if cpu_baseline:
        tw = W.Workload(w.name, m, w.spectra, "f32", "mixed")
        out["cpu_baseline"], out["accuracy"] = cut_sample_oracle(B, dev, tw, m, 16, 4, ("mixed", "fp64"))
    out["workload"] = "full-detector frame (9216^2, 85 orders x 2 x 2, 6000 x 64, K=11) with tabulated PSF maps"
    return out


def noise_run(B, r, mid, frame, stream, flush, reps=5):
    """The detector-noise stage on the rendered full frame: FP32 expected electrons in, 16-bit
    ADU out (photon and dark shot noise, pixel response, read-out noise, cross-talk)."""
    import torch

    params = dict(seed=20201105, pattern_seed=17, dark_e=2.5, prnu=0.01, ron_e=3.2, xtalk=2e-4, gain=1.1,
                  bias=1000.0, saturation=65535)
    out = r.add_noise(mid, frame, "u16", stream=stream, **params)
    ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.add_noise(mid, frame, "u16", out=out, stream=stream, **params)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    px = sum(f.numel() for f in frame)
    nbytes = px * (4 + 2)
    peaks, kind = _peaks()
    hbm = peaks.get("hbm_gbs")
    return {"ms": t, "pixels": px, "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (t * 1e-3) / 1e9,
            "hbm_peak_gbs": hbm, "frac_of_hbm": (nbytes / (t * 1e-3) / 1e9 / hbm) if hbm else None,
            "peak_source": kind, "params": params,
            "note": "Philox4x32-10 draws per pixel in FP32 with error bounds (inversion, PTRS, Box-Muller, ADU rounding), FP64 only for decisions too close to call: bit-exact ADU; ALU-bound, not HBM"}


def adjoint_run(B, dev, flush, reps=10, cpu_baseline=False):
    """Calibration-fitting step on the differentiation tile (2048^2, 10 orders x 4000 x 32, K=9):
    the residual against a target rendered from coefficients shifted by up to 0.01 px, and the
    gradient of the squared residual with respect to every mapping and PSF-width coefficient by
    the adjoint kernel (e2e_render_adjoint).  Reports the adjoint alone and the whole step."""
    import torch

    w = W.config5()
    rng = np.random.default_rng(W.SEED_BASE + 5)
    shifted = w.model.copy()
    for s in shifted.slices:
        s.cx[0] += rng.uniform(-0.01, 0.01)
        s.cy[0] += rng.uniform(-0.01, 0.01)
    stamps = w.model.n_stamps
    n_grad = sum(2 * W.n_coeffs(s.degree) + 6 for s in w.model.slices)
    r = B.Renderer(dev, kernel_timing=1)
    try:
        mid, mt = r.load_model(w.model), r.load_model(shifted)
        sids = r.load_spectra(w)
        target = r.render(mt, sids)[0].double()
        frame = r.empty_frames(mid)
        stream = torch.cuda.current_stream()
        dldi = 2.0 * (r.render(mid, sids, out=frame)[0].double() - target)

        def fit_step():
            I = r.render(mid, sids, out=frame)[0]
            return r.adjoint(mid, sids, [2.0 * (I.double() - target)])

        for _ in range(3):
            fit_step()
        torch.cuda.synchronize()
        adj_ms, step_ms, kern = [], [], []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r.adjoint(mid, sids, [dldi])
            b.record(stream)
            torch.cuda.synchronize()
            adj_ms.append(a.elapsed_time(b))
            kern += [ms for name, ms in B.e2e_kernel_times(r.ctx) if name == "adjoint"]
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fit_step()
            b.record(stream)
            torch.cuda.synchronize()
            step_ms.append(a.elapsed_time(b))
        grads = [x.cpu().numpy() for x in r.adjoint(mid, sids, [dldi])]
        out = {"workload": w.name, "stamps": stamps, "gradient_entries": n_grad,
               "adjoint": {"ms": statistics.median(adj_ms), "kernel_ms": statistics.median(kern) if kern else None,
                           "value": stamps / (statistics.median(adj_ms) * 1e-3), "unit": UNIT},
               "fit_step": {"ms": statistics.median(step_ms),
                            "note": "render + residual + adjoint (the loss gradient of one fitting iteration)"}}
    finally:
        r.close()
    if cpu_baseline:
        import oracle

        cores = min(os.cpu_count() or 1, len(w.model.slices))  # the oracle runs one thread per slice
        g = dldi.cpu().numpy()
        t0 = time.perf_counter()
        ref = oracle.vjp(w.model, w.flux_for, [g], n_threads=cores)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": stamps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"the oracle's FP64 vector-Jacobian product over the whole tile "
                                         f"({stamps} stamps), {dt:.2f} s"}
        acc = {}
        for name, gg, oo in zip(("cx", "cy", "sigma_x", "sigma_y"), grads, ref):
            scale = float(np.abs(oo).max())
            err = np.abs(gg - oo)
            big = np.abs(oo) >= 1e-3 * scale
            acc[name] = {"max_abs_err_over_max": float(err.max() / scale) if scale else 0.0,
                         "max_rel_err_entries_ge_1e-3_max": float(np.max(err[big] / np.abs(oo[big]))) if big.any() else 0.0}
        acc["bound"] = "per group |g - o| <= 2e-5 max|o| + 2e-4 |o| (the adjoint tests' tolerance)"
        acc["ok"] = all(bool(np.all(np.abs(gg - oo) <= 2e-5 * np.abs(oo).max() + 2e-4 * np.abs(oo)))
                        for gg, oo in zip(grads, ref))
        out["accuracy"] = acc
    return out


def elliptical_run(B, dev, rank=0, world=1, reps=3, cpu_baseline=False):
    """The multi-detector instrument with the rotated PSF (4 x 9216^2 FP32, 30 orders per
    detector x 4 fibers x 2 slices, 8000 x 128 samples, K = 13): mixed precision on the whole
    instrument (this rank's detectors), and the plain FP64 renderer on its first order per
    detector (it is ~100x slower), both timed with CUDA events, L2 flushed between renders."""
    import torch

    from paper_2008_05858_gb300 import shard

    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for key, orders, prec, n in (("mixed", 30, "mixed", reps), ("fp64", 1, "fp64", 1)):
        w, _ = shard.shard_workload(W.config3(orders_per_detector=orders), rank, world)
        r = B.Renderer(dev)
        mid = r.load_model(w.model)
        sids = r.load_spectra(w)
        frames = r.empty_frames(mid, "f32")
        st = torch.cuda.current_stream()
        r.render(mid, sids, prec, "f32", out=frames, stream=st)
        ms = []
        for _ in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            r.render(mid, sids, prec, "f32", out=frames, stream=st)
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.median(ms)
        out[key] = {"stamps": w.model.n_stamps, "ms_per_render": t, "value": w.model.n_stamps / (t * 1e-3),
                    "unit": UNIT, "orders_per_detector": orders, "detectors": len(w.model.det_shape)}
        del frames
        r.close()
    out["speedup_mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    if cpu_baseline:
        w3 = W.config3(orders_per_detector=1)
        out["cpu_baseline"], out["accuracy"] = cut_sample_oracle(B, dev, w3, w3.model, 8, 4, ("mixed", "fp64"))
    out["workload"] = "4 x 9216^2 FP32, 30 orders/detector x 4 fibers x 2 slices, 8000 x 128 samples, deg 5, " \
                      "K=13 rotated elliptical PSF (|theta| <= 10 deg); fp64 leg on 1 order/detector"
    return out


def serving_run(B, dev, n_jobs=512, max_inflight=8, load=0.8, express_stamps=1 << 24):
    """Request stream of uneven render jobs through the serving loop (e2e_server_*).

    Three job classes (single-order 1024x256 tiles, 10-order 4096^2 tiles, full 9216^2
    frames; 40/40/20), one resident optical model and spectrum set per class.  A saturation
    run submits every job at t=0 (steady throughput); then a seeded Poisson stream arrives
    at `load` x that throughput.  Latency = completion on the device (seen by the loop) minus
    submission; frames are library-owned and released as they complete."""
    import threading

    r = B.Renderer(dev)
    classes = W.serving_classes()
    res = []
    for q, jc in enumerate(classes):
        w = jc.make(W.SEED_BASE + 40 + q)
        res.append((jc.name, r.load_model(w.model), r.load_spectra(w), w.model.n_stamps))
    rng = np.random.default_rng(W.SEED_BASE + 4)
    kinds = rng.choice(len(classes), size=n_jobs, p=[jc.share for jc in classes])
    srv = B.Server(r, max_inflight=max_inflight)

    def run(arrivals):
        rids, infos = [], [None] * n_jobs
        have = threading.Semaphore(0)

        def reaper():
            for i in range(n_jobs):
                have.acquire()
                info = srv.wait(rids[i])
                B.e2e_release_frame(r.ctx, int(info["frame_id"]))
                srv.forget(rids[i])
                infos[i] = info

        th = threading.Thread(target=reaper)
        th.start()
        t0 = time.perf_counter()
        for i in range(n_jobs):
            if arrivals is not None:
                delay = t0 + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            _, mid, sids, _ = res[kinds[i]]
            rids.append(srv.submit(mid, sids, "mixed", "f32"))
            have.release()
        th.join()
        sub = np.array([x["submit_ms"] for x in infos])
        adm = np.array([x["admit_ms"] for x in infos])
        done = np.array([x["done_ms"] for x in infos])
        span_s = (done.max() - sub.min()) * 1e-3
        lat = done - sub
        ev = sorted([(a, 1) for a in adm] + [(d, -1) for d in done])
        depth = peak = 0
        for _, dlt in ev:
            depth += dlt
            peak = max(peak, depth)
        out = {"jobs": n_jobs, "jobs_per_s": n_jobs / span_s,
               "stamps_per_s": float(sum(res[k][3] for k in kinds)) / span_s,
               "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "max": float(lat.max())},
               "queue_wait_ms_p99": float(np.percentile(adm - sub, 99)), "max_jobs_in_flight": peak,
               "by_class": {}}
        for q, (name, _, _, _) in enumerate(res):
            sel = kinds == q
            if sel.any():
                out["by_class"][name] = {
                    "jobs": int(sel.sum()), "latency_ms_p50": float(np.percentile(lat[sel], 50)),
                    "latency_ms_p99": float(np.percentile(lat[sel], 99)),
                    "device_ms_p50": float(np.median([infos[i]["device_ms"] for i in np.nonzero(sel)[0]]))}
        return out

    for q in range(len(res)):  # warm every class once
        info = srv.wait(srv.submit(res[q][1], res[q][2], "mixed", "f32"))
        B.e2e_release_frame(r.ctx, int(info["frame_id"]))
    sat = run(None)
    rate = load * sat["jobs_per_s"]
    arrivals = W.poisson_arrivals(np.random.default_rng(W.SEED_BASE + 41), n_jobs, rate)
    poi = run(arrivals)
    srv.stop()
    # the same arrivals with an express class: jobs up to express_stamps stamps are admitted
    # ahead of queued full frames and run on high-priority streams
    srv = B.Server(r, max_inflight=max_inflight, express_stamps=express_stamps)
    for q in range(len(res)):
        info = srv.wait(srv.submit(res[q][1], res[q][2], "mixed", "f32"))
        B.e2e_release_frame(r.ctx, int(info["frame_id"]))
    poi_x = run(arrivals)
    srv.stop()
    r.close()
    return {"workload": "512 jobs, 40% 1-order 1024x256 / 40% 10-order 4096^2 / 20% full 9216^2 frames, "
                        "mixed precision, f32 frames, models resident",
            "max_inflight": max_inflight, "admission": "free-HBM budget (0.9 x free at start), FIFO",
            "poisson": dict(poi, arrival_rate_jobs_per_s=rate, load=load), "saturation": sat,
            "poisson_express": dict(poi_x, express_stamps=express_stamps, arrival_rate_jobs_per_s=rate, load=load)}


def _load_spectrum_ptr(B, ctx, fiber, orders, lens, flux_tensor):
    import ctypes as C

    n = len(orders)
    oid = (C.c_int32 * n)(*orders)
    nl = (C.c_int32 * n)(*lens)
    sid = C.c_uint64()
    B._check(B.load_library().e2e_load_spectrum(C.c_void_p(ctx), fiber, n, oid, nl,
                                                C.cast(C.c_void_p(flux_tensor.data_ptr()), C.POINTER(C.c_double)),
                                                C.byref(sid)))
    return sid.value


KERNEL_SOURCES = ["paper_2008_05858_gb300/csrc/render_mixed.cu", "paper_2008_05858_gb300/csrc/render_mixed_far.cu",
                  "paper_2008_05858_gb300/csrc/render_mixed.cuh",
                  "paper_2008_05858_gb300/csrc/phi32.cuh",
                  "paper_2008_05858_gb300/csrc/mixed_common.cuh", "paper_2008_05858_gb300/csrc/merge_tile.cuh",
                  "paper_2008_05858_gb300/csrc/e2e_device.cuh", "paper_2008_05858_gb300/csrc/tail_coeffs.h"]


def _strip_comments(src: str) -> str:
    """C/C++ source without comments and blank lines (string literals in these files hold no
    comment markers), so that editing a comment does not invalidate the traffic counters."""
    import re

    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash() -> str:
    """sha256[:16] of the render kernel's source files with comments stripped (the code the
    traffic counters refer to)."""
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(_strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def _load_traffic():
    """DRAM bytes per launch of the render kernel from the committed ncu summary, or None if
    the kernel's sources changed since those counters were taken."""
    p = os.path.join(ROOT, "profiles", "render_mixed_traffic.txt")
    try:
        kv = {}
        for line in open(p):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return float(kv["traffic_bytes_per_launch_full_frame"])
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-elliptical", action="store_true")
    ap.add_argument("--no-noise", action="store_true")
    ap.add_argument("--no-photons", action="store_true")
    ap.add_argument("--no-table", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--shard", default="frame", choices=["frame", "band"],
                    help="with several GPUs: an independent frame per GPU (weak scaling) or bands of one frame (strong)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
