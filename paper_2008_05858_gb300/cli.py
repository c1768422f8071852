"""Command line: render seeded synthetic frames through the C ABI (for profiling and demos).

    python -m paper_2008_05858_gb300.cli render --config 2 --orders 12 --repeat 3
    python -m paper_2008_05858_gb300.cli render --config 5 --precision fp64 --save frame.npy
    python -m paper_2008_05858_gb300.cli aliasing        # flat-field sampling study (Fig. 4)
    python -m paper_2008_05858_gb300.cli render --config 2 --orders 12 --psf table
    python -m paper_2008_05858_gb300.cli noise --config 2 --orders 12
    python -m paper_2008_05858_gb300.cli photons --config 2 --orders 12 --photons 1e8
    python -m paper_2008_05858_gb300.cli adjoint --config 5

``--orders`` shortens the full-detector workload (config 2) to its first orders so a profiler
capture stays small; every other shape is the named configuration's.
"""
from __future__ import annotations

import argparse
import sys
import time


def _workload(args):
    from . import workloads as W

    if args.config == 2:
        return W.config2(n_orders=args.orders or 85)
    if args.config == 1:
        return W.config1()
    if args.config == 3:
        return W.config3(orders_per_detector=args.orders or 30)
    if args.config == 5:
        return W.config5()
    raise SystemExit(f"unknown config {args.config}")


def cmd_render(args) -> int:
    import numpy as np
    import torch

    from .binding import Renderer

    w = _workload(args)
    if getattr(args, "psf", "analytic") == "table":
        from . import workloads as W

        w.model = W.with_psf_maps(w.model, oversample=10.0, half_px=8.0, coma=0.2)
    r = Renderer(args.device, kernel_timing=1)
    mid = r.load_model(w.model)
    sids = r.load_spectra(w)
    dtype = args.dtype or w.out_dtype
    out = r.render(mid, sids, args.precision, dtype)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.repeat):
        r.render(mid, sids, args.precision, dtype, out=out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(args.repeat, 1)
    print(f"{w.name}: {w.model.n_stamps} stamps, {dt * 1e3:.3f} ms/render (wall), plan {r.plan(mid)}")
    if args.save:
        np.save(args.save, np.stack([o.cpu().numpy() for o in out]))
    r.close()
    return 0


def cmd_noise(args) -> int:
    import torch

    from .binding import Renderer

    w = _workload(args)
    r = Renderer(args.device, kernel_timing=1)
    mid = r.load_model(w.model)
    frame = r.render(mid, r.load_spectra(w), "mixed", "f32")
    p = dict(seed=20201105, pattern_seed=17, dark_e=2.5, prnu=0.01, ron_e=3.2, xtalk=2e-4, gain=1.1, bias=1000.0)
    out = r.add_noise(mid, frame, "u16", **p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.repeat):
        r.add_noise(mid, frame, "u16", out=out, **p)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(args.repeat, 1)
    print(f"{w.name}: noise on {sum(f.numel() for f in frame)} px, {dt * 1e3:.3f} ms (wall)")
    r.close()
    return 0


def cmd_photons(args) -> int:
    import numpy as np
    import torch

    from . import workloads as W
    from .binding import Renderer

    w = _workload(args)
    tot = sum(float(np.sum(w.flux_for(s))) * (s.lambda_hi - s.lambda_lo) / s.n_lambda * float(np.sum(s.slit_weights))
              for s in w.model.slices)
    k = args.photons / tot
    r = Renderer(args.device, kernel_timing=1)
    mid = r.load_model(w.model)
    sids = [r.load_spectrum(W.Spectrum(sp.fiber, {o: f * k for o, f in sp.flux.items()})) for sp in w.spectra.values()]
    out, n = r.render_photons(mid, sids, seed=7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.repeat):
        r.render_photons(mid, sids, seed=7, out=out, want_total=False)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(args.repeat, 1)
    print(f"{w.name}: {n} photons, {dt * 1e3:.3f} ms (wall)")
    r.close()
    return 0


def cmd_adjoint(args) -> int:
    import torch

    from .binding import Renderer

    w = _workload(args)
    r = Renderer(args.device, kernel_timing=1)
    mid = r.load_model(w.model)
    sids = r.load_spectra(w)
    frame = r.render(mid, sids, "mixed", "f32")[0]
    g = torch.Generator(device=frame.device)
    g.manual_seed(5)
    dldi = torch.randn(frame.shape, dtype=torch.float64, device=frame.device, generator=g)  # a seeded dL/dI
    grads = r.adjoint(mid, sids, [dldi])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.repeat):
        grads = r.adjoint(mid, sids, [dldi])
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(args.repeat, 1)
    n = sum(int(t.numel()) for t in grads)
    print(f"{w.name}: gradient of {n} coefficients over {w.model.n_stamps} stamps, {dt * 1e3:.3f} ms (wall)")
    r.close()
    return 0


def cmd_aliasing(args) -> int:
    import json

    from . import aliasing as A
    from .binding import Renderer

    r = Renderer(args.device)

    def render(w):
        mid = r.load_model(w.model)
        out = r.render(mid, r.load_spectra(w), "mixed", "f64")[0].cpu().numpy()
        r.unload_model(mid)
        return out

    rows = A.study(render, samples=[float(x) for x in args.samples.split(",")], sigma=args.sigma,
                   peak_e=args.peak_e)
    for row in rows:
        print(json.dumps(row))
    r.close()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="paper_2008_05858_gb300.cli")
    sub = ap.add_subparsers(dest="cmd", required=True)
    p = sub.add_parser("render", help="render a synthetic configuration")
    p.add_argument("--config", type=int, default=2)
    p.add_argument("--orders", type=int, default=0)
    p.add_argument("--repeat", type=int, default=3)
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--dtype", default=None, choices=[None, "f32", "f64"])
    p.add_argument("--device", type=int, default=0)
    p.add_argument("--save", default=None)
    p.add_argument("--psf", default="analytic", choices=["analytic", "table"])
    pn = sub.add_parser("noise", help="detector noise stage on a rendered frame")
    pp = sub.add_parser("photons", help="photon Monte-Carlo render")
    pj = sub.add_parser("adjoint", help="gradient of a frame loss (adjoint kernel) for a seeded dL/dI")
    for q in (pn, pp, pj):
        q.add_argument("--config", type=int, default=2)
        q.add_argument("--orders", type=int, default=0)
        q.add_argument("--repeat", type=int, default=3)
        q.add_argument("--device", type=int, default=0)
    pp.add_argument("--photons", type=float, default=1e8)
    pa = sub.add_parser("aliasing", help="ripple of a flat field vs wavelength samples per resolution element")
    pa.add_argument("--samples", default="0.75,1,1.25,1.5,2,3,5,10")
    pa.add_argument("--sigma", type=float, default=1.5)
    pa.add_argument("--peak-e", type=float, default=40000.0)
    pa.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    if args.cmd == "render":
        return cmd_render(args)
    if args.cmd == "aliasing":
        return cmd_aliasing(args)
    if args.cmd == "noise":
        return cmd_noise(args)
    if args.cmd == "photons":
        return cmd_photons(args)
    if args.cmd == "adjoint":
        return cmd_adjoint(args)
    return 1


if __name__ == "__main__":
    sys.exit(main())
