"""Frame comparison used by the parity tests.

Tolerances (the method's fidelity target, Sec. 1 and Sec. 2.2: the photocenter of a
resolution element must move by less than about 1e-5 px):

* per pixel: |g - o| <= REL * |o| + FLOOR * max|o| with REL = 1e-6 and FLOOR = 1e-10
  (relative per-pixel error below 1e-6; the absolute floor covers pixels more than
  ten orders of magnitude below the frame's peak, where an FP32 renderer's relative
  error is set by the FP32 representation of distances of ~5 sigma, not by the method);
* photocenter: flux-weighted centroids of fixed 16 x 16 px windows, for every window
  holding at least 1e-3 of the brightest window's flux, move by less than 1e-5 px.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

REL = 1.0e-6
FLOOR = 1.0e-10
WINDOW = 16
WINDOW_FLUX_FRACTION = 1.0e-3


def _golden_photocenter_bound() -> float:
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "accuracy_requirement.json")
    with open(here) as f:
        return float(json.load(f)["photocenter_shift_px"])


PHOTOCENTER_PX = _golden_photocenter_bound()


@dataclass
class Report:
    max_rel: float  # max |g-o|/|o| over pixels with o >= 1e-4 max
    worst_excess: float  # max over pixels of |g-o| / (REL|o| + FLOOR max|o|); <= 1 passes
    n_bad: int
    photocenter_dx: float
    photocenter_dy: float
    n_windows: int

    @property
    def ok(self) -> bool:
        return self.n_bad == 0 and self.photocenter_dx < PHOTOCENTER_PX and self.photocenter_dy < PHOTOCENTER_PX

    def __str__(self):
        return (f"max_rel={self.max_rel:.3e} worst_excess={self.worst_excess:.3f} bad={self.n_bad} "
                f"photocenter dx={self.photocenter_dx:.2e} dy={self.photocenter_dy:.2e} windows={self.n_windows}")


def window_centroids(frame: np.ndarray, win: int = WINDOW):
    """Flux, x-centroid and y-centroid of every win x win window (ragged edge windows kept)."""
    f = np.asarray(frame, dtype=np.float64)
    H, W = f.shape
    Hp, Wp = -(-H // win) * win, -(-W // win) * win
    pad = np.zeros((Hp, Wp))
    pad[:H, :W] = f
    ys, xs = np.mgrid[0:Hp, 0:Wp].astype(np.float64)
    t = pad.reshape(Hp // win, win, Wp // win, win)
    flux = t.sum(axis=(1, 3))
    mx = (pad * xs).reshape(Hp // win, win, Wp // win, win).sum(axis=(1, 3))
    my = (pad * ys).reshape(Hp // win, win, Wp // win, win).sum(axis=(1, 3))
    with np.errstate(invalid="ignore", divide="ignore"):
        return flux, mx / flux, my / flux


def compare(gpu: np.ndarray, ref: np.ndarray, rel: float = REL, floor: float = FLOOR) -> Report:
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    assert g.shape == o.shape
    peak = float(np.max(np.abs(o))) if o.size else 0.0
    err = np.abs(g - o)
    allow = rel * np.abs(o) + floor * peak
    if peak == 0.0:
        allow = np.full_like(o, 1e-300)
    excess = err / np.maximum(allow, 1e-300)
    bad = int(np.count_nonzero(err > allow))
    big = np.abs(o) >= 1e-4 * peak if peak > 0 else np.zeros_like(o, dtype=bool)
    max_rel = float(np.max(err[big] / np.abs(o[big]))) if np.any(big) else 0.0
    fg, xg, yg = window_centroids(g)
    fo, xo, yo = window_centroids(o)
    sel = fo >= WINDOW_FLUX_FRACTION * (fo.max() if fo.size else 0.0)
    sel &= fo > 0
    dx = float(np.max(np.abs(xg[sel] - xo[sel]))) if np.any(sel) else 0.0
    dy = float(np.max(np.abs(yg[sel] - yo[sel]))) if np.any(sel) else 0.0
    return Report(max_rel, float(excess.max()) if excess.size else 0.0, bad, dx, dy, int(np.count_nonzero(sel)))
