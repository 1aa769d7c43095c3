"""The persistent batched tick (one cooperative kernel launch per tick, grid
barriers between the update's phases) against the plain per-volume update.

The tick runs the plain update's device bodies in the same order, so every
output must be identical, floating point included: allocation, heuristics,
hits, ray records and atlases.  The plain update is pinned to the FP64
oracle by the parity tests, so this carries that parity over.  Also: the
grid-wide allocation over many chunks (a ragged last chunk, clip volumes),
and the bounded barrier waits: a barrier that no block arrives at makes the
tick return ADGI_ERR_TIMEOUT, and the next tick runs normally.
"""
import numpy as np
import pytest

from paper_2301_05125_gb300 import scenegen as S

from _helpers import gpu_volume

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
    eye = (-50.0 + 6.0 * f, 14.0, -10.0 + 3.0 * f)
    return (eye, 38.0, view_proj(eye, (0.0, 6.0, 5.0 * np.sin(f))))


def _identical(a, b, tag):
    for name in ("W", "n", "off", "qv", "qr", "trv", "trr", "cls", "pilot_hit", "pilot_lum", "dep_n", "irr", "dep"):
        np.testing.assert_array_equal(getattr(a, name)(), getattr(b, name)(), err_msg="%s %s" % (tag, name))
    R = int(a.off()[-1])
    np.testing.assert_array_equal(a.main_hit()[:R], b.main_hit()[:R], err_msg=tag + " main hits")
    np.testing.assert_array_equal(a.main_rec()[:R], b.main_rec()[:R], err_msg=tag + " main records")


def _run(adgi, ws, frames, cams=None, fp16=None):
    cams = cams or [None] * len(ws)
    fp16 = fp16 or [0] * len(ws)
    ref = [gpu_volume(adgi, w, atlas_fp16=h) for w, h in zip(ws, fp16)]
    tic = [gpu_volume(adgi, w, atlas_fp16=h) for w, h in zip(ws, fp16)]
    stream = torch.cuda.Stream()
    T = adgi.Tick(tic, stream.cuda_stream)
    for f in range(frames):
        fr = []
        for k, (v, r, w) in enumerate(zip(tic, ref, ws)):
            cam = cams[k](f) if cams[k] else None
            if w.dyn_at is not None and w.dyn_count:
                v.move_vertices(w.dyn_first, w.dyn_at(f))
                r.move_vertices(w.dyn_first, w.dyn_at(f))
            fr.append(adgi.make_frame(f, w.seed, w.lights_at(f), w.sky, cam))
            r.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        T.update(fr)
        assert T.sync() == 0, adgi.load().adgi_last_error()
        for k in range(len(ws)):
            sr, st = ref[k].stats(), tic[k].stats()  # raise on a device anomaly flag
            assert sr.shadow_rays == st.shadow_rays and sr.frames == st.frames
            _identical(ref[k], tic[k], "tick vol %d frame %d" % (k, f))
    info = T.info()
    T.close()
    for v in ref + tic:
        v.close()
    return info


def test_tick_matches_plain_update(adgi):
    ws = [S.box_room(1), S.small_city(5, n_boxes=900, dims=(9, 5, 7), rays_avg=40),
          S.small_city(6, n_boxes=500, dims=(6, 4, 5), rays_avg=24), S.small_city(7, n_boxes=700)]
    info = _run(adgi, ws, 6, cams=[None, None, None, _camera], fp16=[0, 0, 1, 0])
    assert info["grid_blocks"] > 0 and info["chunks"] == len(ws)


def test_tick_grid_allocation_many_chunks(adgi):
    # 63 x 31 x 65 = 126,945 probes: 62 allocation chunks, the last one ragged
    big = S._city(3, 1500, 320, (63, 31, 65), (-126.0, 1.0, -126.0), (4.0, 4.0, 4.0), 16, 8, 64, 4, "big")
    small = S.small_city(5, n_boxes=400, dims=(7, 3, 5), rays_avg=32)
    info = _run(adgi, [big, small], 3, cams=[_camera, None])
    assert info["chunks"] == 62 + 1


def test_tick_wait_gives_up(adgi):
    ws = [S.box_room(1), S.small_city(5, n_boxes=400, dims=(7, 3, 5), rays_avg=32)]
    vols = [gpu_volume(adgi, w) for w in ws]
    stream = torch.cuda.Stream()
    T = adgi.Tick(vols, stream.cuda_stream)
    fr = [adgi.make_frame(0, w.seed, w.lights_at(0), w.sky) for w in ws]
    T.update(fr)
    assert T.sync() == 0
    # barriers that no block arrives at: after the pilot shadow rays, in the
    # allocation's first pass, at or after the allocation's end; each wait
    # gives up after 20 ms
    for stall in (3, 8, 11):
        T.set_wait(20_000_000, stall)
        T.update(fr)
        assert T.sync() == -6  # ADGI_ERR_TIMEOUT
        assert "barrier" in adgi.load().adgi_last_error().decode()
    # the context stays usable: a normal tick afterwards
    T.set_wait(2_000_000_000, -1)
    for f in range(1, 3):
        T.update([adgi.make_frame(f, w.seed, w.lights_at(f), w.sky) for w in ws])
        assert T.sync() == 0
    torch.cuda.synchronize()
    T.close()
    for v in vols:
        v.close()


def test_tick_rejects_other_modes(adgi):
    w = S.small_city(5, n_boxes=300, dims=(5, 3, 4), rays_avg=24)
    a = gpu_volume(adgi, w)
    m = gpu_volume(adgi, w, sampler=1)
    with pytest.raises(adgi.AdgiError):
        adgi.Tick([a, m])
    with pytest.raises(adgi.AdgiError):
        adgi.Tick([a, a])
    a.close()
    m.close()
