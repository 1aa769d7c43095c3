"""GPU parity of the DDGI cosine-gather blend (blend_mode = 1) against the
oracle: allocation, hits and the per-texel ray counts (the rays with
n . w > 0, an exact FP32 test on both sides) bit-exact; irradiance within
1e-3 and depth moments within 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S

from _helpers import gpu_volume, oracle_volume, rel_check
from test_gpu_parity import _compare_update

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


@pytest.mark.parametrize("scene", ["room", "city"])
def test_cosine_gather_matches_oracle(adgi, scene):
    if scene == "room":
        w = S.box_room(1)
    else:
        w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    gv, ov = gpu_volume(adgi, w, blend_mode=1), oracle_volume(O, w, blend_mode=1)
    for f in range(4):
        if w.dyn_at is not None and w.dyn_count:
            dv = w.dyn_at(f)
            gv.move_vertices(w.dyn_first, dv)
            ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky)
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        _compare_update(gv, ov, f, what="cosine gather " + scene)
    gv.close()


def test_cosine_gather_with_clip_volumes_and_fp16(adgi):
    w = S.small_city(5, n_boxes=600, dims=(6, 4, 5), rays_avg=24)
    from test_gpu_clip import view_proj

    gv = gpu_volume(adgi, w, blend_mode=1, atlas_fp16=1)
    ov = oracle_volume(O, w, blend_mode=1)
    for f in range(4):
        eye = (-30.0 + 5.0 * f, 12.0, -5.0)
        cam = (eye, 30.0, view_proj(eye, (0.0, 6.0, 0.0)))
        gv.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        ov.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        np.testing.assert_array_equal(gv.cls(), ov.cls())
        gi = gv.irr()
        np.testing.assert_array_equal(gi[..., 3].astype(np.int64), ov.irr_n().astype(np.int64))
        rel_check(gi[..., :3], ov.irr(), 6e-3, "fp16 cosine-gather irradiance")  # half storage (FP16 bounds)
    gv.close()


def test_cosine_gather_rejects_bad_modes(adgi):
    w = S.box_room(1)
    for over in (dict(blend_mode=2), dict(blend_mode=1, sampler=1), dict(blend_mode=1, atlas_fp16=3)):
        with pytest.raises(adgi.AdgiError):
            gpu_volume(adgi, w, **over)
