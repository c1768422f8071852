"""Partition of a render across GPUs: one process per GPU, no data-path collective.

Detectors are independent frames (each order-slice belongs to one detector and deposits
nothing on another), so a multi-detector instrument shards by detector: rank r renders the
detectors d with d % world == r, as a model of its own.  One large frame shards by bands of
rows: rank r renders every stamp of the model into a frame holding only its band, and the
stamps whose windows cross a band edge are rendered by both neighbours, each keeping its own
rows (the frame edge rule drops the others), so the bands concatenate to the whole frame with
the halo compute duplicated and no exchange.  A single-detector workload otherwise runs one
independent frame per rank (weak scaling).  The only cross-rank traffic is the timing
reduction of the benchmark (max over ranks) and the stamp count (sum).
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

from .workloads import OpticalModel, Workload


def detectors_of_rank(n_det: int, rank: int, world: int) -> List[int]:
    """Detectors rank `rank` of `world` renders (round robin)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return [d for d in range(n_det) if d % world == rank]


def shard_model(model: OpticalModel, rank: int, world: int) -> Tuple[OpticalModel, List[int]]:
    """The sub-model of the detectors of this rank (renumbered 0..n-1) and their global indices."""
    dets = detectors_of_rank(len(model.det_shape), rank, world)
    local = {d: i for i, d in enumerate(dets)}
    slices = [dataclasses.replace(s.copy(), detector=local[s.detector]) for s in model.slices if s.detector in local]
    return OpticalModel([model.det_shape[d] for d in dets], slices, model.psf), dets


def shard_workload(w: Workload, rank: int, world: int) -> Tuple[Workload, List[int]]:
    """A workload restricted to this rank's detectors (spectra are shared, read-only)."""
    m, dets = shard_model(w.model, rank, world)
    return dataclasses.replace(w, model=m, name=f"{w.name}[rank {rank}/{world}]"), dets


def band_rows(height: int, rank: int, world: int) -> Tuple[int, int]:
    """Rows [y0, y1) of band `rank` of `world` near-equal contiguous bands of `height` rows."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    if height < world:
        raise ValueError(f"{height} rows cannot make {world} non-empty bands")
    return height * rank // world, height * (rank + 1) // world


def shard_model_by_band(model: OpticalModel, rank: int, world: int) -> Tuple[OpticalModel, List[Tuple[int, int]]]:
    """This rank's band of every detector as a model of its own, and each band's rows [y0, y1)
    in the full frame.  Detector d keeps the rows band_rows(H_d, rank, world); every slice of
    it moves up by y0 (the constant term of its y mapping, an exact subtraction for the usual
    positive centres), so row r of the band frame is row y0 + r of the full frame.  All
    slices are kept: the planner drops the work whose windows miss the band."""
    rows = [band_rows(h, rank, world) for h, _ in model.det_shape]
    shapes = [(y1 - y0, w) for (y0, y1), (_, w) in zip(rows, model.det_shape)]
    slices = []
    for s in model.slices:
        t = s.copy()
        t.cy[0] -= rows[s.detector][0]  # coefficient (a, b) = (0, 0)
        slices.append(t)
    return OpticalModel(shapes, slices, model.psf), rows


def shard_workload_by_band(w: Workload, rank: int, world: int) -> Tuple[Workload, List[Tuple[int, int]]]:
    """A workload whose frames are this rank's bands (spectra are shared, read-only)."""
    m, rows = shard_model_by_band(w.model, rank, world)
    return dataclasses.replace(w, model=m, name=f"{w.name}[band {rank}/{world}]"), rows


def assemble_bands(bands: List[List["object"]], rows: List[List[Tuple[int, int]]], shapes: List[Tuple[int, int]]):
    """Whole frames (numpy) from every rank's band frames: bands[r][d] holds rows rows[r][d] of
    detector d.  Checks that the bands tile each frame exactly once."""
    import numpy as np

    out = []
    for d, (h, wd) in enumerate(shapes):
        f = np.zeros((h, wd), dtype=np.asarray(bands[0][d]).dtype)
        covered = 0
        for r in range(len(bands)):
            y0, y1 = rows[r][d]
            if y0 != covered:
                raise ValueError(f"detector {d}: band {r} starts at row {y0}, expected {covered}")
            f[y0:y1] = np.asarray(bands[r][d])
            covered = y1
        if covered != h:
            raise ValueError(f"detector {d}: bands cover {covered} of {h} rows")
        out.append(f)
    return out


def reduce_over_ranks(value: float, op: str = "max") -> float:
    """Max (timing) or sum (work) of a scalar over the ranks of the default process group;
    the value itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
