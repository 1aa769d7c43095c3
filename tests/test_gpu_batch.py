"""Graph-captured, batched and autotuned updates give the results of the plain
update (same kernels; only the launch mechanism and block shapes differ).

Integer outputs (allocation, heuristics, hits, counts) must be identical;
float atlases may differ only by the order of shared-memory additions in the
blend (a few ulps), checked at 1e-5 relative.
"""
import numpy as np
import pytest

from paper_2301_05125_gb300 import scenegen as S

from _helpers import gpu_volume, rel_check

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


def _same(a, b, tag):
    np.testing.assert_array_equal(a.W(), b.W(), err_msg=tag)
    np.testing.assert_array_equal(a.n(), b.n(), err_msg=tag)
    np.testing.assert_array_equal(a.trv(), b.trv(), err_msg=tag)
    np.testing.assert_array_equal(a.main_hit()[:, 0], b.main_hit()[:, 0], err_msg=tag)
    np.testing.assert_array_equal(a.pilot_hit(), b.pilot_hit(), err_msg=tag)
    np.testing.assert_array_equal(a.dep_n(), b.dep_n(), err_msg=tag)
    rel_check(a.irr(), b.irr(), 1e-5, tag + " irr")
    rel_check(a.dep_moments(), b.dep_moments(), 1e-5, tag + " dep")


def _step(v, w, f, mode):
    if w.dyn_at is not None and w.dyn_count:
        v.move_vertices(w.dyn_first, w.dyn_at(f))
    getattr(v, mode)(f, w.seed, w.lights_at(f), w.sky)


def test_graph_update_matches_plain(adgi):
    w = S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40)
    a, b = gpu_volume(adgi, w), gpu_volume(adgi, w)
    for f in range(6):
        _step(a, w, f, "update")
        _step(b, w, f, "update_graph")
        a.stats()
        b.stats()
        _same(a, b, "graph frame %d" % f)


def test_batch_matches_individual(adgi):
    ws = [S.box_room(1), S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40),
          S.small_city(6, n_boxes=500, dims=(6, 4, 5), rays_avg=24)]
    ref = [gpu_volume(adgi, w) for w in ws]
    bat = [gpu_volume(adgi, w, atlas_fp16=0) for w in ws]
    stream = torch.cuda.Stream()
    B = adgi.Batch(bat, stream.cuda_stream)
    for f in range(6):
        frames = []
        for v, w in zip(bat, ws):
            if w.dyn_at is not None and w.dyn_count:
                v.move_vertices(w.dyn_first, w.dyn_at(f))
            frames.append(adgi.make_frame(f, w.seed, w.lights_at(f), w.sky))
        B.update(frames)
        stream.synchronize()
        for v, w in zip(ref, ws):
            _step(v, w, f, "update")
        for i in range(len(ws)):
            bat[i].stats()
            _same(ref[i], bat[i], "batch vol %d frame %d" % (i, f))
    B.close()


def test_autotune_keeps_results(adgi):
    w = S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40)
    a, b = gpu_volume(adgi, w), gpu_volume(adgi, w)
    _step(a, w, 0, "update")
    _step(b, w, 0, "update")
    t = b.autotune(0, w.seed, w.lights_at(0), w.sky, reps=2)
    assert t.trace_block in (64, 128, 256) and t.blend_block in (32, 64, 128)
    assert t.ms_trace > 0 and t.ms_shade > 0 and t.ms_blend > 0
    _same(a, b, "after autotune")
    for f in range(1, 5):
        _step(a, w, f, "update")
        _step(b, w, f, "update")
        _same(a, b, "autotuned frame %d" % f)
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_set_tuning(b.h, adgi.adgi_tuning(100, 128, 0, 128))
