"""Partition of a render across GPUs: one process per GPU, no data-path collective.

Detectors are independent frames (each order-slice belongs to one detector and deposits
nothing on another), so a multi-detector instrument shards by detector: rank r renders the
detectors d with d % world == r, as a model of its own.  A single-detector workload runs one
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
