"""The continuous-batching request loop (adgi_server_*).

Requests of several volumes are submitted at once and run on several CUDA
streams, so their updates are in flight together; each volume's results must
still be those of the same frames run on a lone volume with adgi_update:
integer outputs identical, atlases within the parity tolerances (1e-3
relative for irradiance, 1e-4 for the depth moments).  Admission holds a
volume back until the memory budget has room for it.
"""
import time

import numpy as np
import pytest

from paper_2301_05125_gb300 import scenegen as S

from _helpers import DEP_RTOL, IRR_RTOL, gpu_volume, rel_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adgi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05125_gb300 import adgi as A
    from paper_2301_05125_gb300 import build

    build.build()
    A.load()
    return A


def _workloads():
    return [S.box_room(1), S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40),
            S.small_city(6, n_boxes=500, dims=(6, 4, 5), rays_avg=24),
            S.small_city(7, n_boxes=700, dims=(7, 3, 6), rays_avg=32)]


def _submit(srv, vid, w, f):
    mv = w.dyn_at(f) if (w.dyn_at is not None and w.dyn_count) else None
    return srv.submit(vid, f, w.seed, w.lights_at(f), w.sky, move_first=w.dyn_first, move_verts=mv)


def _alone(adgi, w, frames, **over):
    v = gpu_volume(adgi, w, **over)
    for f in range(frames):
        if w.dyn_at is not None and w.dyn_count:
            v.move_vertices(w.dyn_first, w.dyn_at(f))
        v.update(f, w.seed, w.lights_at(f), w.sky)
    v.stats()
    return v


def _same(a, b, tag):
    np.testing.assert_array_equal(a.W(), b.W(), err_msg=tag)
    np.testing.assert_array_equal(a.n(), b.n(), err_msg=tag)
    np.testing.assert_array_equal(a.pilot_hit(), b.pilot_hit(), err_msg=tag)
    np.testing.assert_array_equal(a.main_hit()[:, 0], b.main_hit()[:, 0], err_msg=tag)
    np.testing.assert_array_equal(a.dep_n(), b.dep_n(), err_msg=tag)
    rel_check(a.irr(), b.irr(), IRR_RTOL, tag + " irr")
    rel_check(a.dep_moments(), b.dep_moments(), DEP_RTOL, tag + " dep")


@pytest.mark.parametrize("graph", [True, False])
def test_results_in_the_mix_equal_results_alone(adgi, graph):
    ws = _workloads()
    fp16 = [0, 0, 1, 2]
    frames = 5
    srv = adgi.Server(streams=3, hbm_budget_bytes=8 << 30, graph=graph)
    vids = []
    for w, h in zip(ws, fp16):
        vd = dict(w.volume)
        vd["atlas_fp16"] = h
        vids.append(srv.add_volume(w.verts, w.idx, w.albedo, **vd))
    rid = {}
    for f in range(frames):
        for vid, w in zip(vids, ws):
            rid[_submit(srv, vid, w, f)] = (vid, f)
    srv.drain(300.0)
    res = srv.poll()
    assert len(res) == len(rid)
    assert all(r.status == 0 for r in res), [(r.request_id, r.status) for r in res if r.status]
    by_vol = {}
    for r in res:
        assert rid[r.request_id][0] == r.volume
        assert r.t_submit_s <= r.t_start_s <= r.t_done_s
        by_vol.setdefault(r.volume, []).append(r)
    for vid, rs in by_vol.items():  # one volume's requests run in submission order
        rs.sort(key=lambda r: r.request_id)
        assert all(a.t_done_s <= b.t_start_s for a, b in zip(rs, rs[1:]))
    # requests of different volumes were in flight at the same time
    iv = sorted((r.t_start_s, r.t_done_s, r.volume) for r in res)
    assert any(b[0] < a[1] and a[2] != b[2] for a, b in zip(iv, iv[1:]))
    for vid, w, h in zip(vids, ws, fp16):
        served = srv.volume(vid)
        alone = _alone(adgi, w, frames, atlas_fp16=h)
        _same(served, alone, "%s fp16=%d graph=%s" % (w.name, h, graph))
        alone.close()
    srv.close()


def test_admission_waits_for_memory(adgi):
    w = S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40)
    probe = adgi.Server(streams=1, hbm_budget_bytes=8 << 30)
    probe.add_volume(w.verts, w.idx, w.albedo, **w.volume)
    _submit(probe, 0, w, 0)
    probe.drain(120.0)
    footprint = probe.info()["used_bytes"]
    probe.close()
    assert footprint > 0
    srv = adgi.Server(streams=2, hbm_budget_bytes=int(footprint * 1.5))
    a = srv.add_volume(w.verts, w.idx, w.albedo, **w.volume)
    b = srv.add_volume(w.verts, w.idx, w.albedo, **w.volume)
    for f in range(2):
        _submit(srv, a, w, f)
        _submit(srv, b, w, f)
    done = []
    t_end = time.time() + 120.0
    while len(done) < 2 and time.time() < t_end:  # volume a's two requests
        done += srv.poll()
        time.sleep(0.01)
    assert sorted(r.volume for r in done) == [a, a]
    info = srv.info()
    assert info["resident"] == 1 and info["waiting"] == 1 and info["used_bytes"] <= footprint * 1.5
    alone = _alone(adgi, w, 2)
    _same(srv.volume(a), alone, "admitted first")
    srv.remove_volume(a)  # frees the memory: b is admitted and its queued requests run
    srv.drain(120.0)
    done = srv.poll()
    assert sorted(r.volume for r in done) == [b, b] and all(r.status == 0 for r in done)
    _same(srv.volume(b), alone, "admitted after release")
    alone.close()
    srv.close()


def test_coalescing_keeps_the_newest_frame(adgi):
    w = S.small_city(6, n_boxes=500, dims=(6, 4, 5), rays_avg=24)
    srv = adgi.Server(streams=1, hbm_budget_bytes=8 << 30, coalesce=True)
    vid = srv.add_volume(w.verts, w.idx, w.albedo, **w.volume)
    ids = [_submit(srv, vid, w, f) for f in range(6)]
    srv.drain(120.0)
    res = {r.request_id: r for r in srv.poll()}
    assert sorted(res) == ids
    assert res[ids[-1]].status == 0  # the newest request is never dropped
    assert all(r.status in (0, 1) for r in res.values())
    assert all(r.rays == 0 for r in res.values() if r.status == 1)
    srv.close()


def test_drain_times_out_and_the_server_recovers(adgi):
    # failure detection on the host: a drain whose time limit runs out while
    # requests are still queued returns TIMEOUT (nothing on the device
    # waits); the server keeps running, a later drain completes, and the
    # volume ends as the same frames alone leave it
    w = S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40)
    srv = adgi.Server(streams=1, hbm_budget_bytes=8 << 30, coalesce=False)
    vid = srv.add_volume(w.verts, w.idx, w.albedo, **w.volume)
    ids = [_submit(srv, vid, w, f) for f in range(8)]
    with pytest.raises(adgi.AdgiError) as e:
        srv.drain(0.0)
    assert e.value.code == -6
    srv.drain(120.0)
    res = srv.poll()
    assert sorted(r.request_id for r in res) == ids and all(r.status == 0 for r in res)
    alone = _alone(adgi, w, 8)
    _same(srv.volume(vid), alone, "after a timed-out drain")
    alone.close()
    srv.close()


def test_server_rejects_bad_calls(adgi):
    with pytest.raises(adgi.AdgiError):
        adgi.Server(streams=0)
    srv = adgi.Server(streams=2, hbm_budget_bytes=1 << 20)
    w = S.box_room(1)
    with pytest.raises(adgi.AdgiError) as e:  # larger than the whole budget
        srv.add_volume(w.verts, w.idx, w.albedo, **w.volume)
    assert e.value.code == -3
    with pytest.raises(adgi.AdgiError):
        srv.submit(7, 0, 1, w.lights_at(0))
    srv.close()
