"""Frame comparison used by the parity tests.

Tolerances (the method's fidelity target, Sec. 1 and Sec. 2.2: the photocenter of a
resolution element must move by less than about 1e-5 px):

* per pixel: |g - o| <= REL * |o| + FLOOR * max|o| with REL = 1e-6 and FLOOR = 1e-10
  (relative per-pixel error below 1e-6; the absolute floor covers pixels more than
  ten orders of magnitude below the frame's peak, where an FP32 renderer's relative
  error is set by the FP32 representation of distances of ~5 sigma, not by the method);
* photocenter: flux-weighted centroids of fixed 16 x 16 px windows, for every window
  holding at least 1e-3 of the brightest window's flux, move by less than 1e-5 px.

Window flips.  A stamp's window is centred on floor(c + 1/2); where the mapped centre c lies
within rounding distance of a half-integer, two correct evaluations of c may pick windows one
pixel apart.  Such stamps are found with the oracle (window_ties) and passed to compare() as
boxes around both candidate windows; pixels failing the bound inside a box, and photocenter
windows that meet one, are reported as flips, apart from the failures, not hidden in the
tolerance.
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
    n_bad: int  # pixels failing the bound, flips excluded
    photocenter_dx: float
    photocenter_dy: float
    n_windows: int
    n_ties: int = 0  # stamps (per axis) whose centre lies within the tie margin of a pixel edge
    n_flip_px: int = 0  # pixels failing the bound inside a tie box (explained by a flip)
    n_flip_windows: int = 0  # photocenter windows over the bound that meet a tie box

    @property
    def ok(self) -> bool:
        return self.n_bad == 0 and self.photocenter_dx < PHOTOCENTER_PX and self.photocenter_dy < PHOTOCENTER_PX

    def __str__(self):
        return (f"max_rel={self.max_rel:.3e} worst_excess={self.worst_excess:.3f} bad={self.n_bad} "
                f"photocenter dx={self.photocenter_dx:.2e} dy={self.photocenter_dy:.2e} windows={self.n_windows} "
                f"ties={self.n_ties} flip_px={self.n_flip_px} flip_windows={self.n_flip_windows}")


TIE_MARGIN = 1e-9  # px: far above the ~1e-12 px rounding of the mapping at 9216 px


def tie_boxes(model, flux_of, margin: float = TIE_MARGIN):
    """Per detector, the boxes (x0, x1, y0, y1), half-open, that hold both candidate windows of
    every stamp whose centre lies within `margin` px of a pixel edge (oracle.window_ties)."""
    import oracle

    boxes = {d: [] for d in range(len(model.det_shape))}
    for i, det, j, k, axis in oracle.window_ties(model, flux_of, margin):
        s = model.slices[i]
        xc, yc, _, _, _ = oracle.map_stamp(s, flux_of(s), j, k)
        i0 = int(np.floor(xc + 0.5)) - s.K // 2
        r0 = int(np.floor(yc + 0.5)) - s.K // 2
        boxes[det].append((i0 - 1, i0 + s.K + 1, r0 - 1, r0 + s.K + 1))
    return boxes


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


def compare(gpu: np.ndarray, ref: np.ndarray, rel: float = REL, floor: float = FLOOR, ties=None) -> Report:
    """ties: boxes (x0, x1, y0, y1) of this frame from tie_boxes (None: no stamp is near a tie)."""
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    assert g.shape == o.shape
    peak = float(np.max(np.abs(o))) if o.size else 0.0
    err = np.abs(g - o)
    allow = rel * np.abs(o) + floor * peak
    if peak == 0.0:
        allow = np.full_like(o, 1e-300)
    excess = err / np.maximum(allow, 1e-300)
    over = err > allow
    flip = np.zeros_like(over)
    for x0, x1, y0, y1 in ties or ():
        flip[max(y0, 0):max(y1, 0), max(x0, 0):max(x1, 0)] = True
    bad = int(np.count_nonzero(over & ~flip))
    n_flip_px = int(np.count_nonzero(over & flip))
    big = np.abs(o) >= 1e-4 * peak if peak > 0 else np.zeros_like(o, dtype=bool)
    max_rel = float(np.max(err[big] / np.abs(o[big]))) if np.any(big) else 0.0
    fg, xg, yg = window_centroids(g)
    fo, xo, yo = window_centroids(o)
    sel = fo >= WINDOW_FLUX_FRACTION * (fo.max() if fo.size else 0.0)
    sel &= fo > 0
    fw = window_centroids(flip.astype(np.float64))[0] > 0 if flip.size else np.zeros_like(sel)
    shift = np.maximum(np.abs(xg - xo), np.abs(yg - yo))
    n_flip_windows = int(np.count_nonzero(sel & fw & (shift >= PHOTOCENTER_PX)))
    sel &= ~(fw & (shift >= PHOTOCENTER_PX))
    dx = float(np.max(np.abs(xg[sel] - xo[sel]))) if np.any(sel) else 0.0
    dy = float(np.max(np.abs(yg[sel] - yo[sel]))) if np.any(sel) else 0.0
    return Report(max_rel, float(excess.max()) if excess.size else 0.0, bad, dx, dy, int(np.count_nonzero(sel)),
                  len(ties or ()), n_flip_px, n_flip_windows)
