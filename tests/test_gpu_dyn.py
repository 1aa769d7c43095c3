"""GPU parity of the dynamic Metropolis chains over virtual proxies
(sampler = 1, dyn_ratio > 0) against the CPU oracle.

Both sides take every decision in exact FP32 or integers, so with alpha = 0
(the static guide f_s) and the dynamic target (integer q_d maxima) the
static and dynamic chains, the marks, the traced cells, the ray lists and
all hits agree bit for bit; radiance and atlases are within the parity
tolerances (1e-3 relative irradiance, 1e-4 relative depth moments).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S

from _helpers import DEP_RTOL, IRR_RTOL, gpu_volume, mh_compare, oracle_volume, rel_check

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


def _dyn_compare(A, gv, ov, tag):
    np.testing.assert_array_equal(gv.qd(), ov.qd(), err_msg=tag + " q_d")
    mh_compare(A, gv, ov, tag)
    g, u = gv.dyn_chains()
    og, ou = ov.dyn_chain_state()
    np.testing.assert_array_equal(g.view(np.uint32), og.view(np.uint32), err_msg=tag + " dynamic chain positions")
    np.testing.assert_array_equal(u.view(np.uint32), ou.view(np.uint32), err_msg=tag + " dynamic chain directions")
    q, d, cell = gv.dyn_samples()
    oq, od, ocell = ov.dyn_samples()
    np.testing.assert_array_equal(q, oq, err_msg=tag + " dynamic sample proxies")
    np.testing.assert_array_equal(d.view(np.uint32), od.view(np.uint32), err_msg=tag + " dynamic sample directions")
    np.testing.assert_array_equal(cell, ocell, err_msg=tag + " dynamic cells")
    s = ov.dyn_sizes()
    cells = 8 * s["proxies"]
    first = np.full(cells, 0xFFFFFFFF, np.uint64)
    pos = np.flatnonzero(ocell >= 0)
    cu, fi = np.unique(ocell[pos], return_index=True)
    first[cu] = pos[fi]
    np.testing.assert_array_equal(gv.dyn_first().astype(np.uint64), first, err_msg=tag + " marks")
    marks, traced = ov.dyn_marks()
    incl = np.zeros(cells, np.uint8)
    incl[marks[:traced]] = 1
    np.testing.assert_array_equal(gv.dyn_incl(), incl, err_msg=tag + " traced cells")
    R = ov.dyn_rays()
    np.testing.assert_array_equal(gv.dyn_off(), R["off"], err_msg=tag + " dynamic ray offsets")
    n = s["rays"]
    h = gv.dyn_hit()[:n]
    np.testing.assert_array_equal(A.hit_tri(h), R["tri"], err_msg=tag + " dynamic tri")
    m = R["tri"] >= 0
    np.testing.assert_array_equal(A.hit_t(h)[m], R["t"][m], err_msg=tag + " dynamic t")
    if n:
        rel_check(gv.dyn_rec()[:n, :3], R["rad"], IRR_RTOL, tag + " dynamic radiance")
        rel_check(gv.dyn_rec()[:n, 3], R["dep"], DEP_RTOL, tag + " dynamic depth")
    return n, traced, len(marks)


def _room_volumes(adgi, over):
    w = S.box_room(1)
    vol = dict(w.volume, dims=(4, 4, 4), spacing=(7.0 / 3,) * 3, origin=(0.5, 0.5, 0.5), rays_avg=48,
               rays_max=128, tr_theta=8)
    vol.update(over)
    w2 = S.Workload(w.name, w.seed, w.verts, w.idx, w.albedo, vol, w.frames, w.sky, w.lights_at)
    return w2, gpu_volume(adgi, w2), oracle_volume(O, w2)


@pytest.mark.parametrize("ratio,hd", [(4, 0.91), (1, 0.0)])
def test_dyn_room_light_toggling(adgi, ratio, hd):
    # the light is off on the second frame of every pair: a change each pair
    w, gv, ov = _room_volumes(adgi, dict(sampler=1, alpha=0.0, dyn_ratio=ratio, hysteresis_dyn=hd))
    on = w.lights_at(0)
    seen = []
    for f in range(6):
        lights = on if f % 2 == 0 else []
        gv.update(f, 9, lights, w.sky)
        ov.update(f, 9, lights, w.sky)
        seen.append(_dyn_compare(adgi, gv, ov, "room r=%d frame %d" % (ratio, f)))
    assert any(n > 0 for n, _, _ in seen)  # dynamic rays were traced
    if ratio == 4:
        assert any(0 < t < m for _, t, m in seen)  # and the budget cap bound
    st = gv.stats()
    assert st.rays_per_update == 8 * gv.P + 2 * ov.mh_samples + seen[-1][0]
    gv.close()


def test_dyn_small_city_moving_occluders(adgi):
    # 9 x 5 x 7 probes: proxies clipped at the grid end; moving gates
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    over = dict(sampler=1, alpha=0.0, dyn_ratio=4, hysteresis_dyn=0.91)
    gv, ov = gpu_volume(adgi, w, **over), oracle_volume(O, w, **over)
    total = 0
    for f in range(6):
        dv = w.dyn_at(f)
        gv.move_vertices(w.dyn_first, dv)
        ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky)
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        total += _dyn_compare(adgi, gv, ov, "city frame %d" % f)[0]
    assert total > 0
    gv.close()


def test_dyn_graph_equals_plain(adgi):
    w, plain, _ = _room_volumes(adgi, dict(sampler=1, alpha=1.0, dyn_ratio=4))
    _, graph, _ = _room_volumes(adgi, dict(sampler=1, alpha=1.0, dyn_ratio=4))
    on = w.lights_at(0)
    for f in range(6):
        lights = on if f % 2 == 0 else []
        plain.update(f, 9, lights, w.sky)
        graph.update_graph(f, 9, lights, w.sky)
    np.testing.assert_array_equal(graph.dyn_incl(), plain.dyn_incl())
    np.testing.assert_array_equal(graph.irr(), plain.irr())
    np.testing.assert_array_equal(graph.dep(), plain.dep())
    plain.close()
    graph.close()


def test_dyn_rejects_bad_calls(adgi):
    w = S.box_room(1)
    with pytest.raises(adgi.AdgiError):  # the dynamic chains belong to the Metropolis mode
        gpu_volume(adgi, w, sampler=0, dyn_ratio=4)
    with pytest.raises(adgi.AdgiError):
        gpu_volume(adgi, w, sampler=1, dyn_ratio=-1)
    with pytest.raises(adgi.AdgiError):
        gpu_volume(adgi, w, sampler=1, dyn_ratio=4, hysteresis_dyn=1.0)
    v = gpu_volume(adgi, w, sampler=1)
    with pytest.raises(adgi.AdgiError):  # no dynamic state without the dynamic chains
        v.dyn_off()
    v.close()
