"""Thin ctypes binding of the C ABI in include/adgi.h.

Argument marshalling only: every step of the update runs in the CUDA kernels
of libadgi.so.  There is no fallback: if the library is missing or fails to
load, every call raises.  PyTorch is used only to hand over device memory
(tensor data pointers) and streams.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libadgi.so")

ADGI_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "OVER_BUDGET", -4: "NO_SCENE", -5: "CUDA", -6: "TIMEOUT"}

STATE = dict(W=0, N=1, OFF=2, QV=3, QR=4, TRV=5, TRR=6, PILOT_HIT=7, PILOT_REC=8, PILOT_LUM=9, MAIN_HIT=10,
             MAIN_REC=11, IRR=12, DEP=13, DEP_N=14, ROT=15, BVH_NODES=16, BVH_TRIS=17, MOVING_BVH_NODES=18,
             MOVING_BVH_TRIS=19, MH_CHAINS=20, MH_SAMPLES=21, MH_ORDER=22, MH_OFF=23, MH_HIT_NEG=24,
             QD=25, DYN_CHAINS=26, DYN_SAMPLES=27, DYN_CELLS=28, DYN_FIRST=29, DYN_INCL=30, DYN_OFF=31, DYN_HIT=32,
             DYN_REC=33, CLS=34, DEP_MOMENTS=35, G=36)


class AdgiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("adgi error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class adgi_volume_desc(C.Structure):
    _fields_ = [
        ("origin", C.c_float * 3),
        ("spacing", C.c_float * 3),
        ("dims", C.c_int32 * 3),
        ("irr_interior", C.c_int32),
        ("depth_interior", C.c_int32),
        ("rays_avg", C.c_int32),
        ("rays_min", C.c_int32),
        ("rays_max", C.c_int32),
        ("hysteresis", C.c_float),
        ("depth_max", C.c_float),
        ("atlas_fp16", C.c_int32),
        ("tr_theta", C.c_int32),
        ("sampler", C.c_int32),
        ("alpha", C.c_float),
        ("dyn_ratio", C.c_int32),
        ("hysteresis_dyn", C.c_float),
        ("blend_mode", C.c_int32),
        ("cheb_var_floor_rel", C.c_float),
    ]


class adgi_light(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos_or_dir", C.c_float * 3), ("rgb", C.c_float * 3)]


class adgi_frame(C.Structure):
    _fields_ = [
        ("frame", C.c_uint64),
        ("seed", C.c_uint64),
        ("lights", C.POINTER(adgi_light)),
        ("n_lights", C.c_int32),
        ("sky_rgb", C.c_float * 3),
        ("has_camera", C.c_int32),
        ("cam_pos", C.c_float * 3),
        ("cam_k", C.c_float),
        ("has_clip", C.c_int32),
        ("view_proj", C.c_float * 16),
    ]


class adgi_tuning(C.Structure):
    _fields_ = [("trace_block", C.c_int32), ("shade_block", C.c_int32), ("shadow_blocks_per_sm", C.c_int32),
                ("blend_block", C.c_int32), ("ms_trace", C.c_float), ("ms_shade", C.c_float), ("ms_blend", C.c_float)]


class adgi_result(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("volume", C.c_int32), ("status", C.c_int32), ("t_submit_s", C.c_double),
                ("t_start_s", C.c_double), ("t_done_s", C.c_double), ("rays", C.c_uint64)]


SERVER_COALESCE = 1
SERVER_NO_GRAPH = 2


class adgi_stats(C.Structure):
    _fields_ = [
        ("frames", C.c_uint64),
        ("rays_per_update", C.c_uint64),
        ("pilot_rays", C.c_uint64),
        ("shadow_rays", C.c_uint64),
        ("bvh_nodes", C.c_uint32),
        ("n_tris", C.c_uint32),
        ("device_bytes", C.c_uint64),
        ("ms_last_update", C.c_float),
        ("ms_phase", C.c_float * 8),
        ("kernels_launched", C.c_uint64),
        ("ms_shadow", C.c_float * 2),
        ("ms_blend_plan", C.c_float),
    ]


PHASES = ["bvh", "pilot_trace", "pilot_shade", "heuristics", "allocation", "trace", "shade", "blend"]


EXPORTED = ["adgi_create_volume", "adgi_set_scene", "adgi_move_vertices", "adgi_update", "adgi_query_irradiance",
            "adgi_get_stats", "adgi_destroy", "adgi_set_stream", "adgi_enable_timing", "adgi_state_bytes",
            "adgi_read_state", "adgi_write_atlas", "adgi_trace_closest", "adgi_count_traversal", "adgi_build_bvh",
            "adgi_build_bvh_noalloc", "adgi_allocate_rays", "adgi_update_graph", "adgi_batch_create",
            "adgi_batch_update", "adgi_batch_destroy", "adgi_autotune", "adgi_set_tuning", "adgi_get_tuning",
            "adgi_server_create", "adgi_server_add_volume", "adgi_server_submit", "adgi_server_poll",
            "adgi_server_drain", "adgi_server_volume", "adgi_server_remove_volume", "adgi_server_info",
            "adgi_server_destroy", "adgi_update_slab", "adgi_slab_copy", "adgi_slab_bytes", "adgi_inject_alloc_failure",
            "adgi_tick_create", "adgi_tick_update", "adgi_tick_sync", "adgi_tick_set_wait", "adgi_tick_info",
            "adgi_tick_phase_ns", "adgi_tick_destroy", "adgi_last_error"]

BVH_NOALLOC_MAX_TRIS = 32768

_lib = None


def load(path: str = LIB_PATH):
    """Load libadgi.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libadgi.so not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
    L.adgi_create_volume.argtypes = [C.POINTER(adgi_volume_desc), vp, C.POINTER(vp)]
    L.adgi_set_scene.argtypes = [vp, vp, i32, vp, i32, vp, i32]
    L.adgi_move_vertices.argtypes = [vp, i32, i32, vp, i32]
    L.adgi_update.argtypes = [vp, C.POINTER(adgi_frame)]
    L.adgi_query_irradiance.argtypes = [vp, vp, vp, i32, vp, i32]
    L.adgi_get_stats.argtypes = [vp, C.POINTER(adgi_stats)]
    L.adgi_destroy.argtypes = [vp]
    L.adgi_set_stream.argtypes = [vp, vp]
    L.adgi_enable_timing.argtypes = [vp, i32]
    L.adgi_state_bytes.argtypes = [vp, i32, C.POINTER(u64)]
    L.adgi_read_state.argtypes = [vp, i32, vp, u64]
    L.adgi_write_atlas.argtypes = [vp, vp, vp, vp]
    L.adgi_trace_closest.argtypes = [vp, vp, vp, i32, C.c_float, C.c_float, vp, vp]
    L.adgi_allocate_rays.argtypes = [vp, i32, i32, i32, i32, vp, vp, vp]
    L.adgi_count_traversal.argtypes = [vp, C.POINTER(adgi_frame), C.POINTER(C.c_uint64)]
    L.adgi_build_bvh.argtypes = [vp, i32, vp, i32, C.c_float, vp, vp, vp]
    L.adgi_build_bvh_noalloc.argtypes = [vp, i32, vp, i32, C.c_float, vp, vp, vp]
    L.adgi_update_graph.argtypes = [vp, C.POINTER(adgi_frame)]
    L.adgi_batch_create.argtypes = [C.POINTER(vp), i32, vp, C.POINTER(vp)]
    L.adgi_batch_update.argtypes = [vp, C.POINTER(adgi_frame)]
    L.adgi_batch_destroy.argtypes = [vp]
    L.adgi_tick_create.argtypes = [C.POINTER(vp), i32, vp, C.POINTER(vp)]
    L.adgi_tick_update.argtypes = [vp, C.POINTER(adgi_frame)]
    L.adgi_tick_sync.argtypes = [vp]
    L.adgi_tick_set_wait.argtypes = [vp, u64, i32]
    L.adgi_tick_info.argtypes = [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.adgi_tick_phase_ns.argtypes = [vp, C.POINTER(C.c_uint64), i32]
    L.adgi_tick_destroy.argtypes = [vp]
    L.adgi_autotune.argtypes = [vp, C.POINTER(adgi_frame), i32, C.POINTER(adgi_tuning)]
    L.adgi_set_tuning.argtypes = [vp, C.POINTER(adgi_tuning)]
    L.adgi_get_tuning.argtypes = [vp, C.POINTER(adgi_tuning)]
    L.adgi_server_create.argtypes = [i32, u64, i32, C.POINTER(vp)]
    L.adgi_server_add_volume.argtypes = [vp, C.POINTER(adgi_volume_desc), vp, i32, vp, i32, vp, C.POINTER(i32)]
    L.adgi_server_submit.argtypes = [vp, i32, C.POINTER(adgi_frame), i32, i32, vp, C.POINTER(u64)]
    L.adgi_server_poll.argtypes = [vp, C.POINTER(adgi_result), i32, C.POINTER(i32)]
    L.adgi_server_drain.argtypes = [vp, C.c_double]
    L.adgi_server_volume.argtypes = [vp, i32, C.POINTER(vp)]
    L.adgi_server_remove_volume.argtypes = [vp, i32]
    L.adgi_server_info.argtypes = [vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(i32), C.POINTER(i32)]
    L.adgi_server_destroy.argtypes = [vp]
    L.adgi_update_slab.argtypes = [vp, C.POINTER(adgi_frame), i32, i32, i32]
    L.adgi_slab_copy.argtypes = [vp, i32, i32, i32, vp, i32]
    L.adgi_slab_bytes.argtypes = [vp, i32, i32, i32, C.POINTER(u64)]
    L.adgi_inject_alloc_failure.argtypes = [i32]
    L.adgi_last_error.restype = C.c_char_p
    for name in EXPORTED[:-1]:
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc):
    if rc != ADGI_OK:
        raise AdgiError(rc, load().adgi_last_error().decode(errors="replace"))


def _ptr(x):
    """data pointer of a numpy array or a torch tensor (device or host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _is_dev(x):
    return not isinstance(x, np.ndarray) and getattr(x, "is_cuda", False)


# ------------------------------------------------------------ C-ABI, same names
def adgi_create_volume(desc: adgi_volume_desc, stream=None):
    h = C.c_void_p()
    _check(load().adgi_create_volume(C.byref(desc), stream, C.byref(h)))
    return h


def adgi_set_scene(vol, verts, idx, albedo):
    on_dev = _is_dev(verts)
    nv = int(verts.shape[0]) if verts.ndim == 2 else int(verts.shape[0] // 3)
    nt = int(idx.shape[0]) if idx.ndim == 2 else int(idx.shape[0] // 3)
    _check(load().adgi_set_scene(vol, _ptr(verts), nv, _ptr(idx), nt, _ptr(albedo), int(on_dev)))


def adgi_move_vertices(vol, first, verts):
    on_dev = _is_dev(verts)
    n = int(verts.shape[0]) if verts.ndim == 2 else int(verts.shape[0] // 3)
    _check(load().adgi_move_vertices(vol, int(first), n, _ptr(verts), int(on_dev)))


def adgi_update(vol, frame: adgi_frame):
    _check(load().adgi_update(vol, C.byref(frame)))


def adgi_query_irradiance(vol, pos, nrm, out):
    on_dev = _is_dev(pos)
    n = int(pos.shape[0]) if pos.ndim == 2 else int(pos.shape[0] // 3)
    _check(load().adgi_query_irradiance(vol, _ptr(pos), _ptr(nrm), n, _ptr(out), int(on_dev)))


def adgi_get_stats(vol) -> adgi_stats:
    st = adgi_stats()
    _check(load().adgi_get_stats(vol, C.byref(st)))
    return st


def adgi_destroy(vol):
    _check(load().adgi_destroy(vol))


def adgi_set_stream(vol, stream):
    _check(load().adgi_set_stream(vol, stream))


def adgi_enable_timing(vol, enable=True):
    _check(load().adgi_enable_timing(vol, int(bool(enable))))


def adgi_state_bytes(vol, which) -> int:
    b = C.c_uint64()
    _check(load().adgi_state_bytes(vol, STATE[which] if isinstance(which, str) else int(which), C.byref(b)))
    return int(b.value)


def adgi_read_state(vol, which, dtype) -> np.ndarray:
    nb = adgi_state_bytes(vol, which)
    out = np.empty(nb // np.dtype(dtype).itemsize, dtype)
    _check(load().adgi_read_state(vol, STATE[which] if isinstance(which, str) else int(which), out.ctypes.data, nb))
    return out


def adgi_write_atlas(vol, irr=None, dep=None, dep_n=None):
    keep = [np.ascontiguousarray(a) if a is not None else None for a in (irr, dep, dep_n)]
    _check(load().adgi_write_atlas(vol, *[_ptr(a) for a in keep]))


def adgi_trace_closest(vol, o, d, tmin, tmax, t_out, tri_out):
    n = int(o.shape[0]) if o.ndim == 2 else int(o.shape[0] // 3)
    _check(load().adgi_trace_closest(vol, _ptr(o), _ptr(d), n, float(tmin), float(tmax), _ptr(t_out), _ptr(tri_out)))


def adgi_count_traversal(vol, frame: adgi_frame):
    out = (C.c_uint64 * 12)()
    _check(load().adgi_count_traversal(vol, C.byref(frame), out))
    return [int(x) for x in out]


def adgi_build_bvh(verts, idx, eps, nodes_out, tris_out, stream=None):
    nv = int(verts.shape[0]) if verts.ndim == 2 else int(verts.shape[0] // 3)
    nt = int(idx.shape[0]) if idx.ndim == 2 else int(idx.shape[0] // 3)
    _check(load().adgi_build_bvh(_ptr(verts), nv, _ptr(idx), nt, float(eps), _ptr(nodes_out), _ptr(tris_out), stream))


def adgi_build_bvh_noalloc(verts, idx, eps, nodes_out, tris_out, stream=None, n_tris=None):
    """adgi_build_bvh with its scratch in the library's fixed device array
    (no allocation; at most BVH_NOALLOC_MAX_TRIS triangles; calls must not
    overlap on the GPU)."""
    nv = int(verts.shape[0]) if verts.ndim == 2 else int(verts.shape[0] // 3)
    nt = n_tris if n_tris is not None else (int(idx.shape[0]) if idx.ndim == 2 else int(idx.shape[0] // 3))
    _check(load().adgi_build_bvh_noalloc(_ptr(verts), nv, _ptr(idx), nt, float(eps), _ptr(nodes_out),
                                         _ptr(tris_out), stream))


def scene_eps(verts):
    """The box enlargement adgi_set_scene uses for these vertices."""
    v = np.asarray(verts, np.float64).reshape(-1, 3)
    if v.size == 0:
        return float(np.float32(1e-30))
    ext = float((v.max(0) - v.min(0)).max())
    mag = float(np.abs(v).max())
    return float(np.float32(1e-5 * max(ext, mag) + 1e-30))


def adgi_allocate_rays(W, rays_avg, rays_min, rays_max, n_out, off_out, stream=None):
    _check(load().adgi_allocate_rays(_ptr(W), int(W.shape[0]), int(rays_avg), int(rays_min), int(rays_max),
                                     _ptr(n_out), _ptr(off_out), stream))


def adgi_update_graph(vol, frame: adgi_frame):
    _check(load().adgi_update_graph(vol, C.byref(frame)))


def adgi_batch_create(vols, stream=None):
    arr = (C.c_void_p * len(vols))(*[v.value if isinstance(v, C.c_void_p) else v for v in vols])
    h = C.c_void_p()
    _check(load().adgi_batch_create(arr, len(vols), stream, C.byref(h)))
    return h


def adgi_batch_update(batch, frames):
    arr = (adgi_frame * len(frames))(*frames)
    _check(load().adgi_batch_update(batch, arr))


def adgi_batch_destroy(batch):
    _check(load().adgi_batch_destroy(batch))


def adgi_tick_create(vols, stream=None):
    arr = (C.c_void_p * len(vols))(*[v.value if isinstance(v, C.c_void_p) else v for v in vols])
    h = C.c_void_p()
    _check(load().adgi_tick_create(arr, len(vols), stream, C.byref(h)))
    return h


def adgi_tick_update(tick, frames):
    arr = (adgi_frame * len(frames))(*frames)
    _check(load().adgi_tick_update(tick, arr))


def adgi_tick_sync(tick) -> int:
    """ADGI_OK, or the negative error code (ADGI_ERR_TIMEOUT: a barrier wait gave up)."""
    return int(load().adgi_tick_sync(tick))


def adgi_tick_set_wait(tick, limit_ns, stall_barrier=-1):
    _check(load().adgi_tick_set_wait(tick, int(limit_ns), int(stall_barrier)))


def adgi_tick_info(tick):
    g, sm, ch = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(load().adgi_tick_info(tick, C.byref(g), C.byref(sm), C.byref(ch)))
    return {"grid_blocks": g.value, "smem_bytes": sm.value, "chunks": ch.value}


def adgi_tick_phase_ns(tick, n=64):
    out = (C.c_uint64 * n)()
    _check(load().adgi_tick_phase_ns(tick, out, n))
    return [int(x) for x in out]


def adgi_tick_destroy(tick):
    _check(load().adgi_tick_destroy(tick))


def adgi_autotune(vol, frame: adgi_frame, reps=3) -> adgi_tuning:
    t = adgi_tuning()
    _check(load().adgi_autotune(vol, C.byref(frame), int(reps), C.byref(t)))
    return t


def adgi_set_tuning(vol, t: adgi_tuning):
    _check(load().adgi_set_tuning(vol, C.byref(t)))


def adgi_get_tuning(vol) -> adgi_tuning:
    t = adgi_tuning()
    _check(load().adgi_get_tuning(vol, C.byref(t)))
    return t


def adgi_server_create(streams, hbm_budget_bytes, flags=0):
    h = C.c_void_p()
    _check(load().adgi_server_create(int(streams), int(hbm_budget_bytes), int(flags), C.byref(h)))
    return h


def adgi_server_add_volume(server, desc: adgi_volume_desc, verts, idx, albedo) -> int:
    verts = np.ascontiguousarray(verts, np.float32)
    idx = np.ascontiguousarray(idx, np.int32)
    albedo = np.ascontiguousarray(albedo, np.float32)
    vid = C.c_int32()
    _check(load().adgi_server_add_volume(server, C.byref(desc), _ptr(verts), verts.size // 3, _ptr(idx),
                                         idx.size // 3, _ptr(albedo), C.byref(vid)))
    return int(vid.value)


def adgi_server_submit(server, volume, frame: adgi_frame, move_first=0, move_verts=None) -> int:
    rid = C.c_uint64()
    mv = None if move_verts is None else np.ascontiguousarray(move_verts, np.float32)
    _check(load().adgi_server_submit(server, int(volume), C.byref(frame), int(move_first),
                                     0 if mv is None else mv.size // 3, _ptr(mv), C.byref(rid)))
    return int(rid.value)


_poll_bufs = {}


def adgi_server_poll(server, max_results=4096):
    buf = _poll_bufs.get(max_results)
    if buf is None:
        buf = _poll_bufs[max_results] = (adgi_result * max_results)()
    n = C.c_int32()
    _check(load().adgi_server_poll(server, buf, max_results, C.byref(n)))
    return [adgi_result.from_buffer_copy(buf[i]) for i in range(n.value)]


def adgi_server_drain(server, timeout_s=600.0):
    _check(load().adgi_server_drain(server, float(timeout_s)))


def adgi_server_volume(server, volume):
    h = C.c_void_p()
    _check(load().adgi_server_volume(server, int(volume), C.byref(h)))
    return h


def adgi_server_remove_volume(server, volume):
    _check(load().adgi_server_remove_volume(server, int(volume)))


def adgi_server_info(server):
    used, sup = C.c_uint64(), C.c_uint64()
    res, wait = C.c_int32(), C.c_int32()
    _check(load().adgi_server_info(server, C.byref(used), C.byref(sup), C.byref(res), C.byref(wait)))
    return dict(used_bytes=int(used.value), superseded=int(sup.value), resident=int(res.value),
                waiting=int(wait.value))


def adgi_server_destroy(server):
    _check(load().adgi_server_destroy(server))


def adgi_update_slab(vol, frame: adgi_frame, step, p0, p1):
    _check(load().adgi_update_slab(vol, C.byref(frame), int(step), int(p0), int(p1)))


def adgi_slab_copy(vol, which, p0, p1, dev_buf, into):
    _check(load().adgi_slab_copy(vol, STATE[which] if isinstance(which, str) else int(which), int(p0), int(p1),
                                 _ptr(dev_buf), int(into)))


def adgi_slab_bytes(vol, which, p0, p1) -> int:
    b = C.c_uint64()
    _check(load().adgi_slab_bytes(vol, STATE[which] if isinstance(which, str) else int(which), int(p0), int(p1),
                                  C.byref(b)))
    return int(b.value)


def adgi_inject_alloc_failure(n):
    _check(load().adgi_inject_alloc_failure(int(n)))


def adgi_last_error() -> str:
    return load().adgi_last_error().decode(errors="replace")


# ------------------------------------------------------------ convenience
def make_desc(origin, spacing, dims, irr_interior=6, depth_interior=14, rays_avg=64, rays_min=8, rays_max=256,
              hysteresis=0.97, depth_max=0.0, atlas_fp16=0, tr_theta=16, sampler=0,
              alpha=1.0, dyn_ratio=0, hysteresis_dyn=0.91, blend_mode=0,
              cheb_var_floor_rel=0.0) -> adgi_volume_desc:
    d = adgi_volume_desc()
    d.origin[:] = [float(x) for x in origin]
    d.spacing[:] = [float(x) for x in spacing]
    d.dims[:] = [int(x) for x in dims]
    d.irr_interior, d.depth_interior = int(irr_interior), int(depth_interior)
    d.rays_avg, d.rays_min, d.rays_max = int(rays_avg), int(rays_min), int(rays_max)
    d.hysteresis = float(hysteresis)
    d.depth_max = float(depth_max)
    d.atlas_fp16 = int(atlas_fp16)
    d.tr_theta = int(tr_theta)
    d.sampler = int(sampler)
    d.alpha = float(alpha)
    d.dyn_ratio = int(dyn_ratio)
    d.hysteresis_dyn = float(hysteresis_dyn)
    d.blend_mode = int(blend_mode)
    d.cheb_var_floor_rel = float(cheb_var_floor_rel)
    return d


def make_frame(frame, seed, lights, sky=(0.0, 0.0, 0.0), camera=None) -> adgi_frame:
    arr = (adgi_light * max(1, len(lights)))()
    for i, (kind, v, rgb) in enumerate(lights):
        arr[i].kind = int(kind)
        arr[i].pos_or_dir[:] = [float(x) for x in v]
        arr[i].rgb[:] = [float(x) for x in rgb]
    f = adgi_frame()
    f.frame = int(frame)
    f.seed = int(seed)
    f.lights = C.cast(arr, C.POINTER(adgi_light))
    f.n_lights = len(lights)
    f.sky_rgb[:] = [float(x) for x in sky]
    if camera is not None:
        f.has_camera = 1
        f.cam_pos[:] = [float(x) for x in camera[0]]
        f.cam_k = float(camera[1])
        if len(camera) > 2 and camera[2] is not None:  # (pos, k, row-major 4x4 view-projection)
            f.has_clip = 1
            f.view_proj[:] = [float(x) for x in np.asarray(camera[2], np.float32).reshape(16)]
    f._keep = arr
    return f


class Volume:
    """Owning wrapper of an adgi_volume handle."""

    def __init__(self, stream=None, **desc):
        self.desc = make_desc(**desc)
        self.h = adgi_create_volume(self.desc, stream)
        d = self.desc
        self.P = d.dims[0] * d.dims[1] * d.dims[2]
        self.Ti, self.Td = d.irr_interior + 2, d.depth_interior + 2
        self.fp16 = bool(d.atlas_fp16)

    @classmethod
    def borrow(cls, h, desc):
        """view of a handle owned elsewhere (a server volume): never destroyed here"""
        v = cls.__new__(cls)
        v.desc, v.h, v._borrowed = desc, h, True
        v.P = desc.dims[0] * desc.dims[1] * desc.dims[2]
        v.Ti, v.Td = desc.irr_interior + 2, desc.depth_interior + 2
        v.fp16 = bool(desc.atlas_fp16)
        return v

    def close(self):
        if self.h and not getattr(self, "_borrowed", False):
            adgi_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scene(self, verts, idx, albedo):
        if isinstance(verts, np.ndarray):
            verts = np.ascontiguousarray(verts, np.float32)
            idx = np.ascontiguousarray(idx, np.int32)
            albedo = np.ascontiguousarray(albedo, np.float32)
        adgi_set_scene(self.h, verts, idx, albedo)

    def move_vertices(self, first, verts):
        if isinstance(verts, np.ndarray):
            verts = np.ascontiguousarray(verts, np.float32)
        adgi_move_vertices(self.h, first, verts)

    def update(self, frame, seed, lights, sky=(0, 0, 0), camera=None):
        adgi_update(self.h, make_frame(frame, seed, lights, sky, camera))

    def update_graph(self, frame, seed, lights, sky=(0, 0, 0), camera=None):
        adgi_update_graph(self.h, make_frame(frame, seed, lights, sky, camera))

    def autotune(self, frame, seed, lights, sky=(0, 0, 0), reps=3):
        return adgi_autotune(self.h, make_frame(frame, seed, lights, sky), reps)

    def query(self, pos, nrm, out=None):
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, np.float32)
            nrm = np.ascontiguousarray(nrm, np.float32)
            out = np.empty_like(pos) if out is None else out
        adgi_query_irradiance(self.h, pos, nrm, out)
        return out

    def stats(self):
        return adgi_get_stats(self.h)

    def state(self, which, dtype):
        return adgi_read_state(self.h, which, dtype)

    # typed readers
    def W(self):
        return self.state("W", np.uint32)

    def n(self):
        return self.state("N", np.uint32)

    def off(self):
        return self.state("OFF", np.uint32)

    def qv(self):
        return self.state("QV", np.uint16).reshape(self.P, 8)

    def qr(self):
        return self.state("QR", np.uint16).reshape(self.P, 8)

    def trv(self):
        return self.state("TRV", np.uint16).reshape(self.P, 8)

    def trr(self):
        return self.state("TRR", np.uint16).reshape(self.P, 8)

    def pilot_hit(self):
        return self.state("PILOT_HIT", np.int32).reshape(self.P, 8, 2)

    def pilot_rec(self):
        return self.state("PILOT_REC", np.float32).reshape(self.P, 8, 4)

    def pilot_lum(self):
        return self.state("PILOT_LUM", np.float32).reshape(self.P, 8)

    def main_hit(self):
        return self.state("MAIN_HIT", np.int32).reshape(-1, 2)

    def main_rec(self):
        return self.state("MAIN_REC", np.float32).reshape(-1, 4)

    # Metropolis volumes (sampler = 1)
    def mh_chains(self):
        """chain states: (g float32[C, 3], u float32[C, 2])"""
        a = self.state("MH_CHAINS", np.float32).reshape(2, -1, 4)
        return a[0, :, :3].copy(), np.stack([a[0, :, 3], a[1, :, 0]], axis=1)

    def mh_samples(self):
        """the last update's samples in chain order: (probe int32[B], direction float32[B, 3])"""
        a = self.state("MH_SAMPLES", np.float32).reshape(-1, 4)
        return a[:, 3].copy().view(np.int32), a[:, :3].copy()

    def mh_order(self):
        return self.state("MH_ORDER", np.uint32)

    def mh_off(self):
        return self.state("MH_OFF", np.uint32)

    def mh_hit_neg(self):
        return self.state("MH_HIT_NEG", np.int32).reshape(-1, 2)

    def qd(self):
        return self.state("QD", np.uint32).reshape(self.P, 8)

    def cls(self):
        return self.state("CLS", np.uint8)

    # dynamic chains (dyn_ratio > 0)
    def dyn_chains(self):
        a = self.state("DYN_CHAINS", np.float32).reshape(2, -1, 4)
        return a[0, :, :3].copy(), np.stack([a[0, :, 3], a[1, :, 0]], axis=1)

    def dyn_samples(self):
        """(proxy int32[Bd], direction float32[Bd, 3], cell int32[Bd])"""
        a = self.state("DYN_SAMPLES", np.float32).reshape(-1, 4)
        return a[:, 3].copy().view(np.int32), a[:, :3].copy(), self.state("DYN_CELLS", np.int32)

    def dyn_first(self):
        return self.state("DYN_FIRST", np.uint32)

    def dyn_incl(self):
        return self.state("DYN_INCL", np.uint8)

    def dyn_off(self):
        return self.state("DYN_OFF", np.uint32)

    def dyn_hit(self):
        return self.state("DYN_HIT", np.int32).reshape(-1, 2)

    def dyn_rec(self):
        return self.state("DYN_REC", np.float32).reshape(-1, 4)

    @property
    def packed(self):
        return int(self.desc.atlas_fp16) == 3

    def irr(self):
        """irradiance atlas as float32 {r, g, b, count}; packed volumes: the
        raw 32-bit codes (R bits 0-8, G 9-17, B 18-25, count 26-31)"""
        if self.packed:
            return self.state("IRR", np.uint32).reshape(self.P, self.Ti, self.Ti)
        dt = np.float16 if self.fp16 else np.float32
        return self.state("IRR", dt).reshape(self.P, self.Ti, self.Ti, 4).astype(np.float32)

    def dep(self):
        """depth atlas as float32 {mean, variance}; packed volumes: the raw
        32-bit codes (mean bits 0-12, mean square 13-25, count 26-31)"""
        if self.packed:
            return self.state("DEP", np.uint32).reshape(self.P, self.Td, self.Td)
        dt = np.float16 if self.fp16 else np.float32
        return self.state("DEP", dt).reshape(self.P, self.Td, self.Td, 2).astype(np.float32)

    def dep_moments(self):
        """depth atlas as the moments {mean, mean^2} (the library stores
        {mean, variance}; the C ABI forms mean^2 in FP64)."""
        return self.state("DEP_MOMENTS", np.float64).reshape(self.P, self.Td, self.Td, 2)

    def dep_n(self):
        return self.state("DEP_N", np.uint8).reshape(self.P, self.Td, self.Td)

    def rotation(self):
        return self.state("ROT", np.float32).reshape(3, 3)

    def write_atlas(self, irr=None, dep=None, dep_n=None):
        dt = np.float16 if self.fp16 else np.float32
        adgi_write_atlas(self.h, None if irr is None else np.ascontiguousarray(irr, dt),
                         None if dep is None else np.ascontiguousarray(dep, dt),
                         None if dep_n is None else np.ascontiguousarray(dep_n, np.uint8))


class Server:
    """Owning wrapper of an adgi_server (continuous-batching request loop)."""

    def __init__(self, streams=4, hbm_budget_bytes=120 << 30, coalesce=False, graph=True):
        flags = (SERVER_COALESCE if coalesce else 0) | (0 if graph else SERVER_NO_GRAPH)
        self.h = adgi_server_create(streams, hbm_budget_bytes, flags)
        self.descs = {}

    def add_volume(self, verts, idx, albedo, **desc):
        d = make_desc(**desc)
        vid = adgi_server_add_volume(self.h, d, verts, idx, albedo)
        self.descs[vid] = d
        return vid

    def submit(self, volume, frame, seed, lights, sky=(0, 0, 0), camera=None, move_first=0, move_verts=None):
        return adgi_server_submit(self.h, volume, make_frame(frame, seed, lights, sky, camera), move_first,
                                  move_verts)

    def poll(self, max_results=4096):
        return adgi_server_poll(self.h, max_results)

    def drain(self, timeout_s=600.0):
        adgi_server_drain(self.h, timeout_s)

    def volume(self, vid):
        """a non-owning Volume view of an admitted, idle volume"""
        return Volume.borrow(adgi_server_volume(self.h, vid), self.descs[vid])

    def remove_volume(self, vid):
        adgi_server_remove_volume(self.h, vid)

    def info(self):
        return adgi_server_info(self.h)

    def close(self):
        if self.h:
            adgi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper of an adgi_batch: one graph launch per tick for all volumes."""

    def __init__(self, volumes, stream=None):
        self.volumes = list(volumes)
        self.h = adgi_batch_create([v.h for v in self.volumes], stream)

    def update(self, frames):
        """frames: list of adgi_frame (make_frame), one per volume."""
        self._keep = frames
        adgi_batch_update(self.h, frames)

    def close(self):
        if self.h:
            adgi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tick:
    """Owning wrapper of an adgi_tick: one persistent kernel launch per tick for all volumes."""

    def __init__(self, volumes, stream=None):
        self.volumes = list(volumes)
        self.h = adgi_tick_create([v.h for v in self.volumes], stream)

    def update(self, frames):
        """frames: list of adgi_frame (make_frame), one per volume."""
        self._keep = frames
        adgi_tick_update(self.h, frames)

    def sync(self) -> int:
        return adgi_tick_sync(self.h)

    def set_wait(self, limit_ns, stall_barrier=-1):
        adgi_tick_set_wait(self.h, limit_ns, stall_barrier)

    def info(self):
        return adgi_tick_info(self.h)

    def phase_ns(self, n=64):
        """ns from the tick's start to the completion of each grid barrier (last tick)"""
        return adgi_tick_phase_ns(self.h, n)

    def close(self):
        if self.h:
            adgi_tick_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hit_tri(hit):
    """triangle index of packed hits (-1 on a miss), back-face bit removed."""
    x = hit[..., 0].astype(np.int64) & 0xFFFFFFFF
    return np.where(x == 0xFFFFFFFF, -1, x & 0x7FFFFFFF).astype(np.int64)


def hit_back(hit):
    x = hit[..., 0].astype(np.int64) & 0xFFFFFFFF
    return (x != 0xFFFFFFFF) & ((x & 0x80000000) != 0)


def hit_t(hit):
    return hit[..., 1].astype(np.int32).view(np.float32)
