"""GPU parity of the camera clip volumes (Fig. TrCam(b)) against the oracle.

With a view-projection matrix, every probe is classified per frame as V_in,
V_out - V_in or outside; pilots, heuristics, allocation, samples and the
count catch-up follow the class.  The classification, allocation and every
hit are bit-exact; radiance and atlases are within the parity tolerances.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S

from _helpers import gpu_volume, mh_compare, oracle_volume
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


def view_proj(eye, target, fov_deg=60.0, near=0.5, far=500.0):
    """row-major OpenGL-style look-at times perspective, FP32"""
    eye, target = np.asarray(eye, np.float64), np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, [0.0, 1.0, 0.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = r, u, -f
    V[:3, 3] = -V[:3, :3] @ eye
    t = 1.0 / np.tan(np.radians(fov_deg) / 2)
    Pm = np.zeros((4, 4))
    Pm[0, 0], Pm[1, 1] = t, t
    Pm[2, 2], Pm[2, 3] = -(far + near) / (far - near), -2 * far * near / (far - near)
    Pm[3, 2] = -1.0
    return (Pm @ V).astype(np.float32)


def _camera(f):
    # a camera sweeping past the city: the clip volumes change every frame
    eye = (-50.0 + 6.0 * f, 14.0, -10.0 + 3.0 * f)
    target = (0.0, 6.0, 5.0 * np.sin(f))
    return (eye, 38.0, view_proj(eye, target))


def test_clip_volumes_allocation_mode(adgi):
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    gv, ov = gpu_volume(adgi, w), oracle_volume(O, w)
    seen = set()
    for f in range(8):
        cam = _camera(f)
        dv = w.dyn_at(f)
        gv.move_vertices(w.dyn_first, dv)
        ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        ov.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        np.testing.assert_array_equal(gv.cls(), ov.cls(), err_msg="clip volumes, frame %d" % f)
        seen |= set(np.unique(ov.cls()).tolist())
        _compare_update(gv, ov, f, what="clip")
        cls = ov.cls()
        assert (gv.n()[cls == 0] == 0).all() and (gv.n()[cls == 1] == 8).all()
    assert seen == {0, 1, 2}  # every class occurred
    gv.close()


def test_clip_volumes_metropolis_dynamic(adgi):
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    over = dict(sampler=1, alpha=0.0, dyn_ratio=4, hysteresis_dyn=0.91)
    gv, ov = gpu_volume(adgi, w, **over), oracle_volume(O, w, **over)
    for f in range(6):
        cam = _camera(f)
        dv = w.dyn_at(f)
        gv.move_vertices(w.dyn_first, dv)
        ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        ov.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        np.testing.assert_array_equal(gv.cls(), ov.cls(), err_msg="clip volumes, frame %d" % f)
        np.testing.assert_array_equal(gv.qd(), ov.qd(), err_msg="q_d, frame %d" % f)
        mh_compare(adgi, gv, ov, "clip metropolis frame %d" % f)
        np.testing.assert_array_equal(gv.dyn_off(), ov.dyn_rays()["off"], err_msg="dynamic rays, frame %d" % f)
    gv.close()


def test_clip_volumes_packed_sky_bit_exact(adgi):
    # sky only: every sample is the FP32 sky, so the codes (and the count
    # catch-up of V_out - V_in) agree bit for bit
    w = S.box_room(1)
    vd = dict(w.volume)
    vd.update(dims=(5, 4, 3), rays_avg=40, atlas_fp16=3)
    g = adgi.Volume(**vd)
    empty = (np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.float32))
    g.set_scene(*empty)
    o = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], vd["irr_interior"], vd["depth_interior"],
                       vd["rays_avg"], vd["rays_min"], vd["rays_max"], vd["hysteresis"], vd["depth_max"],
                       vd["tr_theta"], packed=True)
    o.set_scene(*empty)
    seen_catch_up = False
    for f in range(30):
        sky = (0.3 + 0.01 * f, 1.7 - 0.02 * f, 0.05 * f)
        cam = None
        if f >= 24:  # after the counts pass 16, a camera that leaves part of the grid in V_out - V_in
            eye = (-6.0 + f - 24, 4.0, 4.0)
            cam = (eye, 100.0, view_proj(eye, (4.0, 4.0, 4.0), fov_deg=50.0))
        g.update(f, 7, [], sky, camera=cam)
        o.update(f, 7, [], sky, camera=cam)
        g.stats()
        np.testing.assert_array_equal(g.cls(), o.cls(), err_msg="clip volumes, frame %d" % f)
        np.testing.assert_array_equal(g.irr(), o.irr_packed(), err_msg="irradiance codes, frame %d" % f)
        np.testing.assert_array_equal(g.dep(), o.dep_packed(), err_msg="visibility codes, frame %d" % f)
        seen_catch_up |= bool((o.cls() == 1).any())
    assert seen_catch_up
    g.close()
    o.close()
