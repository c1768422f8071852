"""Multi-process sharding on CPU (gloo, world size 2): each rank renders its detectors (or its
band of rows of every detector) with the oracle, rank 0 gathers them and checks the union
equals the whole-instrument render; the timing and work reductions match max / sum over the
ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2008_05858_gb300 import shard
        from paper_2008_05858_gb300 import workloads as W

        w = W.small_config(seed=401, n_detectors=3, n_lambda=120, n_slit=8, orders=1)
        sub, dets = shard.shard_workload(w, rank, world)
        frames = oracle.render_workload(sub, n_threads=1) if sub.model.slices else [
            np.zeros(s) for s in sub.model.det_shape]
        got = {d: f for d, f in zip(dets, frames)}
        gathered = [None] * world
        dist.all_gather_object(gathered, got)
        tmax = shard.reduce_over_ranks(10.0 + rank, "max")
        nsum = shard.reduce_over_ranks(sub.model.n_stamps, "sum")
        if rank == 0:
            full = oracle.render_workload(w, n_threads=1)
            merged = {}
            for g in gathered:
                merged.update(g)
            ok = sorted(merged) == list(range(len(full))) and all(
                np.array_equal(merged[d], full[d]) for d in range(len(full)))
            ok = ok and tmax == 10.0 + world - 1 and nsum == w.model.n_stamps
            with open(out_path, "w") as f:
                f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_detector_shards_reassemble_the_frame(tmp_path):
    out = tmp_path / "result.txt"
    mp.spawn(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    assert out.read_text() == "ok"


def test_detectors_of_rank_partition():
    from paper_2008_05858_gb300.shard import detectors_of_rank

    for n in range(0, 9):
        for world in range(1, 5):
            parts = [detectors_of_rank(n, r, world) for r in range(world)]
            assert sorted(d for p in parts for d in p) == list(range(n))
    with pytest.raises(ValueError):
        detectors_of_rank(3, 2, 2)


def _band_worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2008_05858_gb300 import shard
        from paper_2008_05858_gb300 import workloads as W

        # two detectors of 150 rows, three orders each: traces cross the band edge
        w = W.small_config(seed=402, n_detectors=2, height=150, n_lambda=90, n_slit=6, orders=3, trace_pitch=12.0)
        sub, rows = shard.shard_workload_by_band(w, rank, world)
        frames = oracle.render_workload(sub, n_threads=1)
        gathered = [None] * world
        dist.all_gather_object(gathered, (rows, frames))
        if rank == 0:
            full = oracle.render_workload(w, n_threads=1)
            got = shard.assemble_bands([g[1] for g in gathered], [g[0] for g in gathered], w.model.det_shape)
            # the same stamps; only the rounding of the shifted y mapping differs
            ok = all(np.all(np.abs(a - b) <= 1e-11 * np.abs(b) + 1e-14 * np.abs(b).max()) for a, b in zip(got, full))
            ok = ok and all(np.abs(b).max() > 0 for b in full)
            with open(out_path, "w") as f:
                f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_band_shards_reassemble_the_frame(tmp_path):
    out = tmp_path / "result.txt"
    mp.spawn(_band_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    assert out.read_text() == "ok"


def test_band_rows_partition_and_assembly_checks():
    from paper_2008_05858_gb300.shard import assemble_bands, band_rows

    for h in (1, 2, 7, 32, 1000, 9216):
        for world in range(1, 9):
            if h < world:
                with pytest.raises(ValueError):
                    band_rows(h, 0, world)
                continue
            parts = [band_rows(h, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == h
            assert all(a[1] == b[0] and a[1] > a[0] for a, b in zip(parts, parts[1:]))
    z = [[np.zeros((2, 3))], [np.zeros((2, 3))]]
    with pytest.raises(ValueError):  # a gap between the bands
        assemble_bands(z, [[(0, 2)], [(3, 5)]], [(5, 3)])
    with pytest.raises(ValueError):  # the bands stop short of the frame
        assemble_bands(z, [[(0, 2)], [(2, 4)]], [(5, 3)])
