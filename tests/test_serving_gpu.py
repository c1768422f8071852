"""Serving loop (e2e_server_*): continuous batching over streams, admission by a memory
budget, results identical alone and in the mix, cancellation and wait timeouts."""
import numpy as np
import pytest

from paper_2008_05858_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def renderer():
    from paper_2008_05858_gb300.binding import Renderer

    r = Renderer(0)
    yield r
    r.close()


def _models(r, heavy=False):
    ws = [W.small_config(seed=200 + i, width=300 + 40 * i, height=160, n_lambda=300 + 37 * i,
                         n_slit=16 + 8 * (i % 3)) for i in range(4)]
    if heavy:  # a few-millisecond job, so that the small ones arrive while it runs
        ws.append(W.config2(n_orders=8))
    ids = []
    for w in ws:
        ids.append((r.load_model(w.model), r.load_spectra(w), w))
    return ids


def test_each_result_is_identical_alone_and_in_the_mix(renderer):
    from paper_2008_05858_gb300.binding import Server

    ms = _models(renderer, heavy=True)
    alone = []
    for mid, sids, w in ms:
        f = renderer.render(mid, sids, "mixed", "f32")
        torch.cuda.synchronize()
        alone.append([t.clone() for t in f])
    srv = Server(renderer, max_inflight=3)
    outs, rids = [], []
    for rep in range(3):  # 15 jobs, arriving while others run
        for q, (mid, sids, w) in enumerate(ms):
            out = renderer.empty_frames(mid, "f32")
            rids.append(srv.submit(mid, sids, "mixed", "f32", out=out))
            outs.append((q, out))
    infos = [srv.wait(r) for r in rids]
    srv.stop()
    for (q, out), info in zip(outs, infos):
        assert info["status"] == 0
        for a, b in zip(out, alone[q]):
            assert torch.equal(a, b)
    # the loop overlapped jobs on the device: some job was admitted before another finished
    spans = sorted((i["admit_ms"], i["done_ms"]) for i in infos)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))


def test_admission_by_budget_and_refusal(renderer):
    from paper_2008_05858_gb300.binding import Server, E2EError, E2E_ETOOBIG

    ms = _models(renderer)
    need = [renderer.plan(mid)["scratch_bytes"] for mid, _, _ in ms]
    budget = max(need) + (64 << 10) + 16  # room for one job at a time
    assert max(need) + min(need) + (128 << 10) > budget
    srv = Server(renderer, max_inflight=4, budget_bytes=budget)
    rids = [srv.submit(mid, sids, "mixed", "f32", out=renderer.empty_frames(mid)) for mid, sids, _ in ms]
    infos = [srv.wait(r) for r in rids]
    spans = sorted((i["admit_ms"], i["done_ms"]) for i in infos)
    for k in range(len(spans) - 1):  # never two in flight at once
        assert spans[k + 1][0] >= spans[k][1]
    big = W.config5()
    bid = renderer.load_model(big.model)
    bs = renderer.load_spectra(big)
    assert renderer.plan(bid)["scratch_bytes"] > budget
    with pytest.raises(E2EError) as e:
        srv.submit(bid, bs, "mixed", "f32")
    assert e.value.code == E2E_ETOOBIG
    srv.stop()


def test_cancel_timeout_and_library_frames(renderer):
    from paper_2008_05858_gb300 import binding as B

    w = W.config2(n_orders=8)
    mid = renderer.load_model(w.model)
    sids = renderer.load_spectra(w)
    srv = B.Server(renderer, max_inflight=1)
    slow = srv.submit(mid, sids, "fp64", "f32")      # library-owned frame, ~tens of ms
    queued = srv.submit(mid, sids, "mixed", "f32")   # waits for the single slot
    srv.cancel(queued)
    with pytest.raises(B.E2EError) as e:
        srv.wait(slow, timeout_ms=0)
    assert e.value.code == B.E2E_ETIMEOUT
    info = srv.wait(slow)
    assert info["status"] == 0 and info["frame_id"] != 0
    with pytest.raises(B.E2EError) as e:
        srv.wait(queued)
    assert e.value.code == B.E2E_ECANCELLED
    h, wd = w.model.det_shape[0]
    host = np.zeros((h, wd), dtype=np.float32)
    B.e2e_fetch_frame(renderer.ctx, int(info["frame_id"]), 0, host.ctypes.data, False, host.nbytes)
    torch.cuda.synchronize()
    ref = renderer.render(mid, sids, "fp64", "f32")[0].cpu().numpy()
    assert np.array_equal(host, ref) or np.allclose(host, ref, rtol=1e-6, atol=0)
    B.e2e_release_frame(renderer.ctx, int(info["frame_id"]))
    srv.stop()


def test_express_jobs_overtake_queued_frames(renderer):
    from paper_2008_05858_gb300 import binding as B

    heavy = W.config2(n_orders=8)
    hid = renderer.load_model(heavy.model)
    hs = renderer.load_spectra(heavy)
    small = W.small_config(seed=230)
    sid = renderer.load_model(small.model)
    ss = renderer.load_spectra(small)
    srv = B.Server(renderer, max_inflight=1, express_stamps=1 << 20)
    outs = [renderer.empty_frames(hid) for _ in range(3)]
    h = [srv.submit(hid, hs, "fp64", "f32", out=o) for o in outs]  # ~50 ms each, one slot
    s_out = renderer.empty_frames(sid)
    x = srv.submit(sid, ss, "mixed", "f32", out=s_out)
    infos = [srv.wait(r) for r in h]
    xi = srv.wait(x)
    srv.stop()
    assert xi["status"] == 0 and all(i["status"] == 0 for i in infos)
    assert xi["admit_ms"] <= infos[1]["admit_ms"]  # ahead of the frames queued before it
    ref = renderer.render(sid, ss, "mixed", "f32")
    torch.cuda.synchronize()
    assert torch.equal(ref[0], s_out[0])


def test_failed_job_leaves_other_jobs_and_the_model_intact(renderer):
    # A job that passes submission but fails when it is launched (its destination pitch is
    # below the frame width, which the render checks) reports its error and frees its slot
    # and budget; the jobs queued around it and the resident model are not affected.
    from paper_2008_05858_gb300.binding import E2E_EINVAL, E2EError, Server

    ms = _models(renderer)
    alone = []
    for mid, sids, w in ms:
        f = renderer.render(mid, sids, "mixed", "f32")
        torch.cuda.synchronize()
        alone.append([t.clone() for t in f])
    srv = Server(renderer, max_inflight=2)
    outs, rids, bad = [], [], []
    for q, (mid, sids, w) in enumerate(ms):
        out = renderer.empty_frames(mid, "f32")
        rids.append(srv.submit(mid, sids, "mixed", "f32", out=out))
        outs.append((q, out))
        h, wd = w.model.det_shape[0]
        narrow = [torch.empty(h * wd, device="cuda").as_strided((h, wd), (wd - 1, 1))]
        bad.append(srv.submit(mid, sids, "mixed", "f32", out=narrow))
    for b in bad:
        with pytest.raises(E2EError) as e:
            srv.wait(b)
        assert e.value.code == E2E_EINVAL
    infos = [srv.wait(r) for r in rids]
    srv.stop()
    for (q, out), info in zip(outs, infos):
        assert info["status"] == 0
        for a, b in zip(out, alone[q]):
            assert torch.equal(a, b)
    for (mid, sids, w), ref in zip(ms, alone):  # the models still render the same frames
        again = renderer.render(mid, sids, "mixed", "f32")
        torch.cuda.synchronize()
        for a, b in zip(again, ref):
            assert torch.equal(a, b)
