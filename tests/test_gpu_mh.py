"""GPU parity of the Metropolis sampler (sampler = 1) against the CPU oracle.

The chains' decisions are exact FP32 on both sides, so wherever both read the
same guide they follow the same path bit for bit: with alpha = 0 the guide
is f_s = q_c q_v / 1023^2 (bit-exact heuristics), and with alpha > 0 the
test writes the same FP32 atlas into both before each frame.  Checked per
frame: chain states, samples (probe, direction), the grouping by probe, the
+w and -w hits (bit-exact), the +w radiance (1e-3 relative) and the
atlases (counts exact, irradiance 1e-3, depth moments 1e-4 relative).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S

from _helpers import IRR_RTOL, gpu_volume, mh_compare as _compare, oracle_volume, rel_check

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


def _run(A, w, frames, over, camera=None, atlas=None, moving=False, what=""):
    gv = gpu_volume(A, w, **over)
    ov = oracle_volume(O, w, **over)
    for f in range(frames):
        if atlas is not None:  # the same FP32 atlas on both sides: the guide reads identical values
            gi, gd, gn, oi, on, od = atlas(gv, f)
            gv.write_atlas(gi, gd, gn)
            ov.set_atlas(oi, on, od, gn)
        if moving:
            dv = w.dyn_at(f)
            gv.move_vertices(w.dyn_first, dv)
            ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky, camera=camera)
        ov.update(f, w.seed, w.lights_at(f), w.sky, camera=camera)
        _compare(A, gv, ov, "%s frame %d" % (what, f))
    return gv, ov


def test_mh_alpha0_small_city(adgi):
    # 9 x 5 x 7 probes (ragged against every block size), moving occluders
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    gv, _ = _run(adgi, w, 4, dict(sampler=1, alpha=0.0), moving=True, what="alpha 0 city")
    st = gv.stats()
    assert st.rays_per_update == 8 * gv.P + 2 * (40 - 8) * gv.P
    c = adgi.adgi_count_traversal(gv.h, adgi.make_frame(3, w.seed, w.lights_at(3), w.sky))
    assert all(x > 0 for x in c), c  # pilots, then the samples' +w/-w rays and the +w shadow rays
    gv.close()


def _fold(a, T):
    """every tile's border texels from their octahedral fold partners (the
    oracle's border copy applied to texel ids), as the library keeps them"""
    ids, _ = O.border_copy(np.arange(T * T, dtype=np.float64).reshape(T, T, 1), np.zeros((T, T), np.uint8), T - 2)
    src = ids[..., 0].astype(np.int64)
    return a[:, src // T, src % T]


def _random_atlas(seed):
    def make(gv, f):
        rng = np.random.default_rng(seed + f)
        P, Ti, Td = gv.P, gv.Ti, gv.Td
        irr = rng.uniform(0.0, 0.8, (P, Ti, Ti, 4)).astype(np.float32)
        irr[rng.random((P, Ti, Ti)) < 0.3, :3] = 0.0
        irr[..., 3] = rng.integers(0, 40, (P, Ti, Ti)).astype(np.float32)
        irr = _fold(irr, Ti)
        mean = rng.uniform(0.5, 10.0, (P, Td, Td)).astype(np.float32)
        var = rng.uniform(0.0, 2.0, (P, Td, Td)).astype(np.float32)
        dep = _fold(np.stack([mean, var], axis=-1), Td)
        mean, var = dep[..., 0], dep[..., 1]
        dn = _fold(rng.integers(0, 40, (P, Td, Td)).astype(np.uint8), Td)
        od = np.stack([mean.astype(np.float64), var.astype(np.float64) + mean.astype(np.float64) ** 2], axis=-1)
        return irr, dep, dn, irr[..., :3].astype(np.float64), irr[..., 3].astype(np.uint8), od
    return make


def _empty_atlas(gv):
    P, Ti, Td = gv.P, gv.Ti, gv.Td
    z = np.zeros
    return (z((P, Ti, Ti, 4), np.float32), z((P, Td, Td, 2), np.float32), z((P, Td, Td), np.uint8),
            z((P, Ti, Ti, 3)), z((P, Ti, Ti), np.uint8), z((P, Td, Td, 2)))


@pytest.mark.parametrize("alpha", [1.0, 3.0])
def test_mh_alpha_with_written_atlas_and_camera(adgi, alpha):
    w = S.small_city(6, n_boxes=500, dims=(7, 4, 6), rays_avg=32)
    cam = ((0.0, 6.0, 0.0), 10.0)
    gv, _ = _run(adgi, w, 4, dict(sampler=1, alpha=alpha), camera=cam, atlas=_random_atlas(11),
                 what="alpha %g" % alpha)
    gv.close()


def test_mh_room_chains_run_on(adgi):
    # the chains carry their state across frames; the room's closed walls
    # give every q_v a value, so the guide is positive everywhere
    w = S.box_room(1)
    gv, _ = _run(adgi, w, w.frames, dict(sampler=1, alpha=0.5), what="room")
    gv.close()


def test_mh_pilots_only(adgi):
    # rays_avg = 8: no adaptive samples, the pilots alone are blended
    w = S.box_room(2)
    over = dict(sampler=1, alpha=1.0, rays_avg=8, rays_min=8, rays_max=8)
    gv, _ = _run(adgi, w, 3, over, what="pilots only")
    assert gv.mh_order().size == 0 and np.all(gv.mh_off() == 0)
    gv.close()


def test_mh_graph_and_batch_equal_plain(adgi):
    w = S.small_city(5, n_boxes=600, dims=(6, 4, 5), rays_avg=24)
    over = dict(sampler=1, alpha=1.0)
    plain = gpu_volume(adgi, w, **over)
    graph = gpu_volume(adgi, w, **over)
    batched = gpu_volume(adgi, w, **over)
    other = gpu_volume(adgi, w)
    stream = torch.cuda.Stream()
    batch = adgi.Batch([batched, other], stream.cuda_stream)
    for f in range(4):
        plain.update(f, w.seed, w.lights_at(f), w.sky)
        graph.update_graph(f, w.seed, w.lights_at(f), w.sky)
        batch.update([adgi.make_frame(f, w.seed, w.lights_at(f), w.sky) for _ in range(2)])
    stream.synchronize()
    for v, tag in ((graph, "graph"), (batched, "batch")):
        np.testing.assert_array_equal(v.mh_samples()[0], plain.mh_samples()[0], err_msg=tag)
        np.testing.assert_array_equal(v.mh_order(), plain.mh_order(), err_msg=tag)
        np.testing.assert_array_equal(v.irr(), plain.irr(), err_msg=tag)
        np.testing.assert_array_equal(v.dep(), plain.dep(), err_msg=tag)
    batch.close()
    for v in (plain, graph, batched, other):
        v.close()


def test_mh_rejects_bad_calls(adgi):
    w = S.box_room(1)
    with pytest.raises(adgi.AdgiError):
        gpu_volume(adgi, w, sampler=1, atlas_fp16=3)
    with pytest.raises(adgi.AdgiError):
        gpu_volume(adgi, w, sampler=1, alpha=-1.0)
    with pytest.raises(adgi.AdgiError):
        gpu_volume(adgi, w, sampler=2)
    v = gpu_volume(adgi, w, sampler=1)
    v.update(0, w.seed, w.lights_at(0), w.sky)
    with pytest.raises(adgi.AdgiError):
        v.autotune(0, w.seed, w.lights_at(0), w.sky)
    v.close()
    plain = gpu_volume(adgi, w)
    with pytest.raises(adgi.AdgiError):  # no Metropolis state without the sampler
        plain.mh_order()
    plain.close()


def test_mh_fp16_atlases(adgi):
    # half atlases: the guide reads the rounded cache; the chains' integer
    # decisions at alpha = 0 do not depend on it.  The multi-bounce term of
    # the radiance and the atlases carry half rounding: the bounds of the
    # FP16 parity tests (maxima 6e-3 relative)
    w = S.small_city(7, n_boxes=700, dims=(7, 3, 6), rays_avg=32)
    over = dict(sampler=1, alpha=0.0, atlas_fp16=1)
    gv = gpu_volume(adgi, w, **over)
    ov = oracle_volume(O, w, **over)
    for f in range(3):
        gv.update(f, w.seed, w.lights_at(f), w.sky)
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        _compare(adgi, gv, ov, "fp16 frame %d" % f, check_atlas=False, rad_rtol=6e-3)
        gi = gv.irr()
        np.testing.assert_array_equal(gi[..., 3].astype(np.int64), ov.irr_n().astype(np.int64))
        rel_check(gi[..., :3], ov.irr(), 6e-3, "fp16 irradiance atlas")
    gv.close()


def test_mh_tunnel_city_full_size_two_frames(adgi):
    """The bench workload (16384 probes, 4.06M samples, each with a +w and a
    -w ray, moving occluders) on both sides for two frames with alpha = 1:
    frame 0 reads the empty atlas on both sides; before frame 1 the same
    seeded atlas is written into both."""
    w = S.tunnel_city(1)
    over = dict(sampler=1, alpha=1.0)
    make = _random_atlas(21)
    gv, _ = _run(adgi, w, 2, over, atlas=lambda v, f: make(v, f) if f else _empty_atlas(v), moving=True,
                 what="tunnel")
    gv.close()
