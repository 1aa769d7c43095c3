"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact: ray allocation, heuristics, pilot luminance, hit indices and t,
texel counts.  Tolerances (tests/_helpers.py): irradiance 1e-3 relative,
depth moments 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S

from _helpers import DEP_RTOL, IRR_RTOL, diag_path, gpu_volume, oracle_volume, rel_check

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


def _dump_rays(gv, ov, frame, what):
    def dump(rows):
        R = int(ov.off()[-1])
        np.savez(diag_path("fail_%s_f%d.npz" % (what.replace(" ", "_"), frame)), rows=rows[:64],
                 gpu_rec=gv.main_rec()[:R][rows[:64]], ora_rad=ov.main_rad()[rows[:64]],
                 ora_dep=ov.main_dep()[rows[:64]], tri=ov.main_tri()[rows[:64]], t=ov.main_t()[rows[:64]],
                 off=ov.off(), n=ov.n())
    return dump


def _compare_update(gv, ov, frame, check_atlas=True, what=""):
    tag = "%s frame %d" % (what, frame)
    gv.stats()  # raises if a device-side anomaly flag was set
    np.testing.assert_array_equal(gv.W(), ov.W(), err_msg=tag + " W")
    np.testing.assert_array_equal(gv.n(), ov.n(), err_msg=tag + " n")
    np.testing.assert_array_equal(gv.off(), ov.off(), err_msg=tag + " off")
    np.testing.assert_array_equal(gv.qv(), ov.qv(), err_msg=tag + " qv")
    np.testing.assert_array_equal(gv.qr(), ov.qr(), err_msg=tag + " qr")
    np.testing.assert_array_equal(gv.trv(), ov.trv(), err_msg=tag + " trv")
    np.testing.assert_array_equal(gv.trr(), ov.trr(), err_msg=tag + " trr")
    ph = gv.pilot_hit()
    from paper_2301_05125_gb300 import adgi as A

    np.testing.assert_array_equal(A.hit_tri(ph), ov.pilot_tri(), err_msg=tag + " pilot tri")
    hitm = ov.pilot_tri() >= 0
    np.testing.assert_array_equal(A.hit_t(ph)[hitm], ov.pilot_t()[hitm], err_msg=tag + " pilot t")
    np.testing.assert_array_equal(gv.pilot_lum(), ov.pilot_lum().astype(np.float32), err_msg=tag + " pilot lum")
    R = int(ov.off()[-1])
    mh = gv.main_hit()[:R]
    np.testing.assert_array_equal(A.hit_tri(mh), ov.main_tri(), err_msg=tag + " main tri")
    hm = ov.main_tri() >= 0
    np.testing.assert_array_equal(A.hit_t(mh)[hm], ov.main_t()[hm], err_msg=tag + " main t")
    rel_check(gv.main_rec()[:R, :3], ov.main_rad(), IRR_RTOL, tag + " main radiance",
              dump=_dump_rays(gv, ov, frame, what))
    rel_check(gv.main_rec()[:R, 3], ov.main_dep(), DEP_RTOL, tag + " main depth")
    if check_atlas:
        gi, oi = gv.irr(), ov.irr()
        np.testing.assert_array_equal(gi[..., 3].astype(np.int64), ov.irr_n().astype(np.int64),
                                      err_msg=tag + " irr counts")
        np.testing.assert_array_equal(gv.dep_n(), ov.dep_n(), err_msg=tag + " depth counts")
        e_i = rel_check(gi[..., :3], oi, IRR_RTOL, tag + " irradiance atlas")
        e_d = rel_check(gv.dep_moments(), ov.dep(), DEP_RTOL, tag + " depth atlas")
        return e_i, e_d
    return None


# ------------------------------------------------------------------ allocation
# 196608 is the largest grid of the 8-CTA cluster kernel, 196609 the smallest
# of the one-block kernel
@pytest.mark.parametrize("P", [1, 7, 64, 1000, 1025, 16384, 24576, 131072, 196608, 196609, 200000])
def test_allocation_bit_exact(adgi, P):
    rng = np.random.default_rng(P)
    cases = [
        (rng.integers(0, 1 << 24, P), 64, 8, 256),
        (rng.integers(0, 3, P), 64, 4, 512),
        (np.where(rng.random(P) < 0.01, rng.integers(1, 1 << 24, P), 0), 256, 8, 1024),
        (np.zeros(P, np.int64), 33, 8, 40),
        (np.full(P, 5), 9, 8, 9),
        (rng.integers(0, 2, P) * ((1 << 24) - 1), 100, 16, 101),
        (rng.integers(0, 1 << 32, P, dtype=np.uint64), 64, 8, 256),  # weights beyond what the heuristics make
    ]
    dev = torch.device("cuda")
    for W, avg, rmin, rmax in cases:
        W = W.astype(np.uint32)
        n_ref, off_ref = O.allocate(W, avg, rmin, rmax)
        Wd = torch.from_numpy(W.view(np.int32)).to(dev)
        nd = torch.empty(P, dtype=torch.int32, device=dev)
        od = torch.empty(P + 1, dtype=torch.int32, device=dev)
        adgi.adgi_allocate_rays(Wd, avg, rmin, rmax, nd, od, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(nd.cpu().numpy().view(np.uint32), n_ref)
        np.testing.assert_array_equal(od.cpu().numpy().view(np.uint32), off_ref)


def test_allocation_large_then_smaller_then_large(adgi):
    # the cluster kernel's shared memory grows with P (8 B a probe): a grid
    # above 49,152 probes, then a smaller one also above it, then the larger
    # again must all match the oracle (the kernel's shared-memory limit is
    # never lowered by the smaller grid)
    dev = torch.device("cuda")
    rng = np.random.default_rng(21)
    for P in (131072, 60000, 131072, 50000, 196608):
        W = rng.integers(0, 1 << 24, P).astype(np.uint32)
        n_ref, off_ref = O.allocate(W, 64, 8, 256)
        Wd = torch.from_numpy(W.view(np.int32)).to(dev)
        nd = torch.empty(P, dtype=torch.int32, device=dev)
        od = torch.empty(P + 1, dtype=torch.int32, device=dev)
        adgi.adgi_allocate_rays(Wd, 64, 8, 256, nd, od, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(nd.cpu().numpy().view(np.uint32), n_ref, err_msg="P=%d" % P)
        np.testing.assert_array_equal(od.cpu().numpy().view(np.uint32), off_ref, err_msg="P=%d" % P)


def test_graph_of_large_volume_replays_after_smaller_capture(adgi):
    # two volumes above 49,152 probes (cluster allocation with more than
    # 48 KB of shared memory): the larger one's captured update graph is
    # replayed after the smaller one was captured, and must still equal
    # plain updates of an identical volume
    w = S.box_room(1)
    big = dict(origin=(0.2, 0.2, 0.2), spacing=(7.6 / 63, 7.6 / 31, 7.6 / 63), dims=(64, 32, 64), rays_avg=9,
               rays_min=8, rays_max=24)
    small = dict(big, dims=(60, 25, 40), spacing=(7.6 / 59, 7.6 / 24, 7.6 / 39))
    g_big = gpu_volume(adgi, w, **big)
    p_big = gpu_volume(adgi, w, **big)
    g_small = gpu_volume(adgi, w, **small)
    wsum = 0
    for f in range(5):
        lights = w.lights_at(f)
        g_big.update_graph(f, w.seed, lights, w.sky)
        g_small.update_graph(f, w.seed, lights, w.sky)
        p_big.update(f, w.seed, lights, w.sky)
        torch.cuda.synchronize()
        g_big.stats()
        np.testing.assert_array_equal(g_big.W(), p_big.W(), err_msg="frame %d W" % f)
        np.testing.assert_array_equal(g_big.n(), p_big.n(), err_msg="frame %d n" % f)
        np.testing.assert_array_equal(g_big.main_hit(), p_big.main_hit(), err_msg="frame %d hits" % f)
        np.testing.assert_array_equal(g_big.irr(), p_big.irr(), err_msg="frame %d irradiance" % f)
        wsum += int(p_big.W().astype(np.int64).sum())
    assert wsum > 0  # some allocation was not uniform
    for v in (g_big, p_big, g_small):
        v.close()


def test_allocation_rejects_impossible_budget(adgi):
    dev = torch.device("cuda")
    W = torch.zeros(10, dtype=torch.int32, device=dev)
    n = torch.empty(10, dtype=torch.int32, device=dev)
    off = torch.empty(11, dtype=torch.int32, device=dev)
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_allocate_rays(W, 300, 8, 256, n, off)


# ------------------------------------------------------------------ tracing
def _trace_case(adgi, w, O_, D, use_bvh):
    gv = gpu_volume(adgi, w)
    dev = torch.device("cuda")
    o = torch.from_numpy(O_).to(dev)
    d = torch.from_numpy(D).to(dev)
    n = O_.shape[0]
    t = torch.empty(n, dtype=torch.float32, device=dev)
    tri = torch.empty(n, dtype=torch.int32, device=dev)
    adgi.adgi_trace_closest(gv.h, o, d, 1e-4, float("inf"), t, tri)
    torch.cuda.synchronize()
    t_ref, tri_ref, det_ref = O.trace_closest(w.verts, w.idx, O_, D, 1e-4, np.inf, use_bvh=use_bvh)
    h = np.stack([tri.cpu().numpy(), t.cpu().numpy().view(np.int32)], 1)
    np.testing.assert_array_equal(adgi.hit_tri(h), tri_ref)
    np.testing.assert_array_equal(t.cpu().numpy(), t_ref)
    hit = tri_ref >= 0
    np.testing.assert_array_equal(adgi.hit_back(h)[hit], (det_ref < 0)[hit])
    gv.close()


def test_trace_room_bit_exact_vs_brute_force(adgi):
    rng = np.random.default_rng(11)
    w = S.box_room(1)
    n = 200000
    O_ = rng.uniform(0.1, 7.9, (n, 3)).astype(np.float32)
    D = rng.normal(size=(n, 3)).astype(np.float32)
    # rays aimed exactly at box edges and corners stress watertightness
    tgt = w.verts[rng.integers(0, len(w.verts), n // 4)]
    D[: n // 4] = (tgt - O_[: n // 4]).astype(np.float32)
    _trace_case(adgi, w, O_, D, use_bvh=False)


def test_trace_city_bit_exact_vs_oracle(adgi):
    rng = np.random.default_rng(12)
    w = S.small_city(3, n_boxes=2000)
    n = 100000
    O_ = rng.uniform(-40, 40, (n, 3)).astype(np.float32)
    O_[:, 1] = rng.uniform(0.5, 30, n)
    D = rng.normal(size=(n, 3)).astype(np.float32)
    _trace_case(adgi, w, O_, D, use_bvh=True)


def test_trace_axis_aligned_directions(adgi):
    # directions with exact zero components (axis-aligned rays, rays in a
    # coordinate plane, signed zeros): 1/0 in the box test must not reject boxes
    rng = np.random.default_rng(14)
    w = S.small_city(3, n_boxes=2000)
    n = 60000
    O_ = rng.uniform(-40, 40, (n, 3)).astype(np.float32)
    O_[:, 1] = rng.uniform(0.5, 30, n)
    D = rng.normal(size=(n, 3)).astype(np.float32)
    ax = rng.integers(0, 3, n)
    D[np.arange(n) % 3 == 0, :] = 0.0  # axis-aligned: keep one component
    keep = np.arange(n) % 3 == 0
    D[keep, ax[keep]] = np.where(rng.random(keep.sum()) < 0.5, -1.0, 1.0)
    one = np.arange(n) % 3 == 1  # one component zero (+0 or -0)
    D[one, ax[one]] = np.where(rng.random(one.sum()) < 0.5, 0.0, -0.0)
    _trace_case(adgi, w, O_, D, use_bvh=True)


def test_update_axis_aligned_sun(adgi):
    # a sun straight down: every shadow ray points straight up (two zero
    # direction components)
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    sun = [(1, (0.0, -1.0, 0.0), (2.0, 2.0, 2.0))]
    gv = gpu_volume(adgi, w)
    ov = oracle_volume(O, w)
    for f in range(2):
        gv.update(f, w.seed, sun, w.sky)
        ov.update(f, w.seed, sun, w.sky)
        _compare_update(gv, ov, f, what="axis-aligned sun")
    gv.close()


def test_trace_degenerate_scenes(adgi):
    rng = np.random.default_rng(13)
    O_ = rng.uniform(-1, 1, (5000, 3)).astype(np.float32)
    D = rng.normal(size=(5000, 3)).astype(np.float32)
    one = S.Workload("one", 0, np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32),
                     np.array([[0, 1, 2]], np.int32), np.ones((1, 3), np.float32), S.box_room(1).volume, 1,
                     (0, 0, 0), lambda f: [])
    _trace_case(adgi, one, O_, D, use_bvh=False)
    # duplicated triangles: ties must resolve to the smaller index
    dup = S.Workload("dup", 0, one.verts, np.repeat(one.idx, 5, 0), np.ones((5, 3), np.float32),
                     S.box_room(1).volume, 1, (0, 0, 0), lambda f: [])
    _trace_case(adgi, dup, O_, D, use_bvh=False)


# ------------------------------------------------------------------ full update
def test_update_room_bit_exact_and_within_tolerance(adgi):
    w = S.box_room(1)
    gv = gpu_volume(adgi, w)
    ov = oracle_volume(O, w)
    for f in range(w.frames):
        gv.update(f, w.seed, w.lights_at(f), w.sky)
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        _compare_update(gv, ov, f, what="room")
    rng = np.random.default_rng(3)
    pos = rng.uniform(0.5, 7.5, (4000, 3)).astype(np.float32)
    nrm = rng.normal(size=(4000, 3)).astype(np.float32)
    rel_check(gv.query(pos, nrm), ov.query(pos, nrm), IRR_RTOL, "room query")
    gv.close()


def test_update_small_city_ragged(adgi):
    # 9 x 5 x 7 probes (ragged against every block size), moving occluders
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    gv = gpu_volume(adgi, w)
    ov = oracle_volume(O, w)
    for f in range(4):
        dv = w.dyn_at(f)
        gv.move_vertices(w.dyn_first, dv)
        ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky)
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        _compare_update(gv, ov, f, what="small city")
    rng = np.random.default_rng(5)
    pos = rng.uniform(-40, 40, (4000, 3)).astype(np.float32)
    pos[:, 1] = rng.uniform(0, 40, 4000)
    nrm = rng.normal(size=(4000, 3)).astype(np.float32)
    rel_check(gv.query(pos, nrm), ov.query(pos, nrm), IRR_RTOL, "city query")
    gv.close()


@pytest.mark.parametrize("case", ["pilots_only", "uniform_forced", "empty_scene", "theta1_camera", "minimal_grid",
                                  "tiles_8_16", "tiles_5_9", "tiles_1_1"])
def test_update_edge_cases(adgi, case):
    w = S.box_room(2)
    over = {}
    cam = None
    if case == "pilots_only":
        over = dict(rays_avg=8, rays_min=8, rays_max=8)
    elif case == "uniform_forced":
        over = dict(rays_avg=32, rays_min=32, rays_max=32)
    elif case == "empty_scene":
        w = S.Workload("empty", 1, np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32),
                       np.zeros((0, 3), np.float32), w.volume, 3, (0.3, 0.5, 0.9), lambda f: [])
    elif case == "theta1_camera":
        over = dict(tr_theta=1)
        cam = ((2.0, 3.0, 2.5), 1.5)
    elif case == "minimal_grid":
        over = dict(dims=(2, 2, 2), spacing=(4.0, 4.0, 4.0), rays_avg=100, rays_max=300)
    elif case == "tiles_8_16":  # the 8 x 8 / 16 x 16 interiors of the DDGI paper
        over = dict(irr_interior=8, depth_interior=16)
    elif case == "tiles_5_9":  # odd tiles, and texel runs split across 32-sample passes
        over = dict(irr_interior=5, depth_interior=9, rays_avg=120, rays_max=300)
    elif case == "tiles_1_1":  # one texel per tile: every sample in one run, counts above 255
        over = dict(irr_interior=1, depth_interior=1, rays_avg=290, rays_min=290, rays_max=300)
    gv = gpu_volume(adgi, w, **over)
    ov = oracle_volume(O, w, **over)
    for f in range(4):
        gv.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        ov.update(f, w.seed, w.lights_at(f), w.sky, camera=cam)
        _compare_update(gv, ov, f, what=case)
    gv.close()


def test_update_rejects_bad_calls(adgi):
    w = S.box_room(1)
    v = adgi.Volume(**w.volume)
    with pytest.raises(adgi.AdgiError) as e:
        v.update(0, 1, [])
    assert e.value.code == -4  # no scene
    v.set_scene(w.verts, w.idx, w.albedo)
    with pytest.raises(adgi.AdgiError):
        v.move_vertices(len(w.verts) - 1, np.zeros((2, 3), np.float32))
    bad = w.idx.copy()
    bad[0, 0] = len(w.verts)
    with pytest.raises(adgi.AdgiError):
        v.set_scene(w.verts, bad, w.albedo)
    v.close()


# ------------------------------------------------------------------ full size
def test_tunnel_city_full_size_two_frames(adgi):
    """The bench workload (16384 probes, 4.19M rays/update, ~200k triangles,
    moving occluders) on both sides for two frames: allocation, heuristics and
    every hit bit-exact; atlases within tolerance."""
    w = S.tunnel_city(1)
    gv = gpu_volume(adgi, w)
    ov = oracle_volume(O, w)
    for f in range(2):
        dv = w.dyn_at(f)
        gv.move_vertices(w.dyn_first, dv)
        ov.move_vertices(w.dyn_first, dv)
        gv.update(f, w.seed, w.lights_at(f), w.sky)
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        _compare_update(gv, ov, f, what="tunnel")
    gv.close()


# ------------------------------------------------------------------ stand-alone BVH build
@pytest.mark.parametrize("scene", ["room", "city", "one", "two"])
def test_build_bvh_matches_volume_bvh(adgi, scene):
    if scene == "room":
        w = S.box_room(1)
    elif scene == "city":
        w = S.small_city(6, n_boxes=1500)
    else:
        nt = 1 if scene == "one" else 2
        v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
        w = S.Workload(scene, 0, v, np.array([[0, 1, 2], [1, 2, 3]], np.int32)[:nt], np.ones((nt, 3), np.float32),
                       S.box_room(1).volume, 1, (0, 0, 0), lambda f: [])
    gv = gpu_volume(adgi, w)
    # moving every vertex (to where it is) makes every triangle part of the
    # moving set, whose BVH is the linear one adgi_build_bvh builds
    gv.move_vertices(0, w.verts)
    dev = torch.device("cuda")
    nt = w.n_tris
    V = torch.from_numpy(w.verts).to(dev)
    I = torch.from_numpy(w.idx).to(dev)
    nodes = torch.zeros(max(nt - 1, 1) * 16, dtype=torch.int32, device=dev)
    tris = torch.zeros(nt * 12, dtype=torch.float32, device=dev)
    adgi.adgi_build_bvh(V, I, adgi.scene_eps(w.verts), nodes, tris, torch.cuda.current_stream().cuda_stream)
    ref_nodes = gv.state("MOVING_BVH_NODES", np.int32)
    ref_tris = gv.state("MOVING_BVH_TRIS", np.int32)
    if nt > 1:
        np.testing.assert_array_equal(nodes.cpu().numpy(), ref_nodes)
    np.testing.assert_array_equal(tris.cpu().numpy().view(np.int32), ref_tris)
    # triangles in BVH order are a permutation of the input, tagged with their index
    t = tris.cpu().numpy().reshape(nt, 3, 4)
    orig = t[:, 0, 3].view(np.int32)
    assert sorted(orig.tolist()) == list(range(nt))
    np.testing.assert_array_equal(t[:, :, :3], w.verts[w.idx[orig]])
    gv.close()


def test_moving_bvh_after_static_part(adgi):
    """With static and moving triangles, the moving part is built after the
    static part's nodes and triangles and its references relocated; the
    state reader gives it back in the layout of a stand-alone build of the
    moving triangles (those touching a moved vertex, in index order)."""
    w = S.small_city(3, n_boxes=400, dims=(6, 4, 5), rays_avg=24)
    gv = gpu_volume(adgi, w)
    dv = w.dyn_at(1)
    gv.move_vertices(w.dyn_first, dv)
    gv.update(0, w.seed, w.lights_at(0), w.sky)
    verts = w.verts.copy()
    verts[w.dyn_first:w.dyn_first + len(dv)] = dv
    moved = np.zeros(len(verts), bool)
    moved[w.dyn_first:w.dyn_first + len(dv)] = True
    mov = np.flatnonzero(moved[w.idx].any(axis=1))
    assert 1 < len(mov) < w.n_tris  # both parts hold triangles
    dev = torch.device("cuda")
    nt = len(mov)
    nodes = torch.zeros((nt - 1) * 16, dtype=torch.int32, device=dev)
    tris = torch.zeros(nt * 12, dtype=torch.float32, device=dev)
    adgi.adgi_build_bvh(torch.from_numpy(verts).to(dev), torch.from_numpy(np.ascontiguousarray(w.idx[mov])).to(dev),
                        adgi.scene_eps(w.verts), nodes, tris, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gv.state("MOVING_BVH_NODES", np.int32), nodes.cpu().numpy())
    got = gv.state("MOVING_BVH_TRIS", np.float32).reshape(nt, 3, 4)
    ref = tris.cpu().numpy().reshape(nt, 3, 4)
    np.testing.assert_array_equal(got[:, :, :3], ref[:, :, :3])
    # the volume tags each triangle with its scene index, the stand-alone build with its list position
    np.testing.assert_array_equal(got[:, 0, 3].view(np.int32), mov[ref[:, 0, 3].view(np.int32)])
    gv.close()


def _morton_keys(tv):
    """63-bit Morton codes of triangles (vertices tv[n, 3, 3]) in their
    centroid bounds, with the builder's FP32 steps"""
    f = np.float32
    c = ((tv[:, 0] + tv[:, 1]) + tv[:, 2]) * f(1.0 / 3.0)
    lo, hi = c.min(0), c.max(0)
    ext = np.maximum(hi - lo, f(1e-30))
    q = np.clip((c - lo) / ext * f(2097152.0), f(0), f(2097151.0)).astype(np.uint64)
    key = np.zeros(len(tv), np.uint64)
    for b in range(21):
        for k in range(3):
            key |= ((q[:, k] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 2 - k)
    return key


@pytest.mark.parametrize("nt", [5, 1500, 2048, 2049, 30000])
def test_build_order_is_stable_morton_order(adgi, nt):
    # below 2,049 triangles one block sorts (bitonic, by key then index),
    # above it the radix passes do: both must give the stable key order
    rng = np.random.default_rng(nt)
    verts = rng.uniform(-50, 50, (3 * nt, 3)).astype(np.float32)
    verts[: 3 * nt // 2] = np.round(verts[: 3 * nt // 2] / 8.0) * 8.0  # repeated centroids: equal keys
    idx = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    dev = torch.device("cuda")
    nodes = torch.zeros(max(nt - 1, 1) * 16, dtype=torch.int32, device=dev)
    tris = torch.zeros(nt * 12, dtype=torch.float32, device=dev)
    adgi.adgi_build_bvh(torch.from_numpy(verts).to(dev), torch.from_numpy(idx).to(dev), adgi.scene_eps(verts), nodes,
                        tris, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t = tris.cpu().numpy().reshape(nt, 3, 4)
    orig = t[:, 0, 3].view(np.int32)
    assert sorted(orig.tolist()) == list(range(nt))
    key = _morton_keys(verts.reshape(nt, 3, 3))[orig]
    k0, k1 = key[:-1], key[1:]
    assert np.all((k0 < k1) | ((k0 == k1) & (orig[:-1] < orig[1:]))), "not the stable Morton order"
    assert (k0 == k1).any() or nt < 100  # the ties were exercised


def test_build_bvh_rejects_bad_index(adgi):
    dev = torch.device("cuda")
    w = S.box_room(1)
    idx = w.idx.copy()
    idx[5, 1] = len(w.verts) + 3
    nodes = torch.zeros((w.n_tris - 1) * 16, dtype=torch.int32, device=dev)
    tris = torch.zeros(w.n_tris * 12, dtype=torch.float32, device=dev)
    with pytest.raises(adgi.AdgiError) as e:
        adgi.adgi_build_bvh(torch.from_numpy(w.verts).to(dev), torch.from_numpy(idx).to(dev), 1e-4, nodes, tris)
    assert e.value.code == -1 and "index" in str(e.value)
