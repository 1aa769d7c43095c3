"""ctypes wrapper of the C oracle (test infrastructure only).

Every function here forwards to ``adgi_oracle.c``; the arithmetic lives there
and follows the paper's sections cited in that file's header.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcDesc(C.Structure):
    _fields_ = [
        ("origin", C.c_float * 3),
        ("spacing", C.c_float * 3),
        ("dims", C.c_int * 3),
        ("n_irr", C.c_int),
        ("n_dep", C.c_int),
        ("avg", C.c_int),
        ("rmin", C.c_int),
        ("rmax", C.c_int),
        ("hyst", C.c_float),
        ("depth_max", C.c_float),
        ("theta", C.c_int),
        ("packed", C.c_int),
        ("sampler", C.c_int),
        ("alpha", C.c_float),
        ("blend_mode", C.c_int),
        ("dyn_ratio", C.c_int),
        ("hyst_dyn", C.c_float),
        ("var_rel", C.c_float),
    ]


class OrcLight(C.Structure):
    _fields_ = [("kind", C.c_int), ("v", C.c_float * 3), ("rgb", C.c_float * 3)]


class OrcFrame(C.Structure):
    _fields_ = [
        ("frame", C.c_uint64),
        ("seed", C.c_uint64),
        ("lights", C.POINTER(OrcLight)),
        ("n_lights", C.c_int),
        ("sky", C.c_float * 3),
        ("has_camera", C.c_int),
        ("cam", C.c_float * 3),
        ("cam_k", C.c_float),
        ("has_clip", C.c_int),
        ("clip", C.c_float * 16),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        f32p = C.POINTER(C.c_float)
        f64p = C.POINTER(C.c_double)
        i32p = C.POINTER(C.c_int)
        u32p = C.POINTER(C.c_uint32)
        u16p = C.POINTER(C.c_uint16)
        u8p = C.POINTER(C.c_uint8)
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_pilot_dir.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, f32p]
        L.orc_frame_rotation.argtypes = [C.c_uint64, C.c_uint64, f32p]
        L.orc_sf_points.argtypes = [C.c_int, f32p]
        L.orc_oct_encode.argtypes = [f64p, f64p]
        L.orc_oct_decode.argtypes = [f64p, f64p]
        L.orc_texel_of_dir.argtypes = [f32p, C.c_int]
        L.orc_texel_of_dir.restype = C.c_int
        L.orc_intersect_tri.argtypes = [f32p, f32p, f32p, f32p, f32p, f32p, f32p]
        L.orc_intersect_tri.restype = C.c_int
        L.orc_trace_closest.argtypes = [f32p, C.c_int, i32p, C.c_int, C.c_int, f32p, f32p, C.c_float, C.c_float,
                                        C.c_int, f32p, i32p, f32p]
        L.orc_trace_any.argtypes = [f32p, C.c_int, i32p, C.c_int, C.c_int, f32p, f32p, C.c_float, C.c_float,
                                    C.c_int, u8p]
        L.orc_allocate.argtypes = [u32p, C.c_int, C.c_int, C.c_int, C.c_int, u32p, u32p]
        L.orc_allocate.restype = C.c_int
        L.orc_luts.argtypes = [C.c_double, u16p, u16p]
        L.orc_create.argtypes = [C.POINTER(OrcDesc), C.c_int]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_set_scene.argtypes = [vp, f32p, C.c_int, i32p, C.c_int, f32p]
        L.orc_set_scene.restype = C.c_int
        L.orc_move_vertices.argtypes = [vp, C.c_int, C.c_int, f32p]
        L.orc_move_vertices.restype = C.c_int
        L.orc_update.argtypes = [vp, C.POINTER(OrcFrame)]
        L.orc_update.restype = C.c_int
        L.orc_trace_shade_probes.argtypes = [vp, C.POINTER(OrcFrame), i32p, C.c_int]
        L.orc_trace_shade_probes.restype = C.c_longlong
        L.orc_set_threads.argtypes = [vp, C.c_int]
        for fn in ("orc_slab_begin", "orc_slab_weights", "orc_slab_finish"):
            getattr(L, fn).argtypes = [vp, C.POINTER(OrcFrame), C.c_int, C.c_int]
            getattr(L, fn).restype = C.c_int
        L.orc_slab_slice.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, C.c_int]
        L.orc_slab_slice.restype = C.c_longlong
        L.orc_query.argtypes = [vp, C.c_int, f32p, f32p, f64p]
        L.orc_num_probes.argtypes = [vp]
        L.orc_num_probes.restype = C.c_int
        L.orc_num_main_rays.argtypes = [vp]
        L.orc_num_main_rays.restype = C.c_longlong
        for name, rt in [("orc_irr", f64p), ("orc_irr_n", u8p), ("orc_dep", f64p), ("orc_dep_n", u8p),
                         ("orc_W", u32p), ("orc_n", u32p), ("orc_off", u32p), ("orc_qv", u16p), ("orc_qr", u16p),
                         ("orc_trv", u16p), ("orc_trr", u16p), ("orc_pil_t", f32p), ("orc_pil_tri", i32p),
                         ("orc_pil_lum", f32p), ("orc_pil_dir", f32p), ("orc_pil_rad", f64p), ("orc_pil_dep", f64p),
                         ("orc_m_t", f32p), ("orc_m_tri", i32p), ("orc_m_rad", f64p), ("orc_m_dep", f64p),
                         ("orc_rot", f32p)]:
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = rt
        L.orc_probe_pos.argtypes = [vp, C.c_int, f32p]
        L.orc_main_dir.argtypes = [vp, C.c_int, C.c_int, f32p]
        L.orc_voxel_diag.argtypes = [vp]
        L.orc_voxel_diag.restype = C.c_double
        L.orc_depth_max.argtypes = [vp]
        L.orc_depth_max.restype = C.c_float
        L.orc_tmin.argtypes = [vp]
        L.orc_tmin.restype = C.c_float
        L.orc_set_atlas.argtypes = [vp, f64p, u8p, f64p, u8p]
        L.orc_border_copy.argtypes = [f64p, u8p, C.c_int, C.c_int]
        L.orc_change_from_pilots.argtypes = [vp, C.POINTER(OrcFrame), f32p, i32p, f32p]
        L.orc_codec_enc.argtypes = [C.c_int, C.c_float]
        L.orc_codec_enc.restype = C.c_uint32
        L.orc_codec_dec.argtypes = [C.c_int, C.c_uint32]
        L.orc_codec_dec.restype = C.c_float
        L.orc_codec_mav.argtypes = [C.c_float, C.c_float, C.c_uint32]
        L.orc_codec_mav.restype = C.c_float
        for name in ("orc_irr_packed", "orc_dep_packed"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = u32p
        L.orc_cage_diag.argtypes = [vp]
        L.orc_cage_diag.restype = C.c_float
        L.orc_blend_packed_records.argtypes = [vp, C.c_int, C.c_int, f64p, f64p, f64p, f64p]
        L.orc_mh_normal_quantile.argtypes = [C.c_int]
        L.orc_mh_normal_quantile.restype = C.c_float
        L.orc_mh_exp.argtypes = [C.c_int]
        L.orc_mh_exp.restype = C.c_float
        for name in ("orc_mh_samples", "orc_mh_chains"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = C.c_longlong
        for name, rt in [("orc_mh_chain_g", f32p), ("orc_mh_chain_u", f32p), ("orc_mh_probe", i32p),
                         ("orc_mh_dir", f32p), ("orc_mh_tri", i32p), ("orc_mh_t", f32p), ("orc_mh_t_neg", f32p),
                         ("orc_mh_tri_neg", i32p), ("orc_mh_rad", f64p), ("orc_mh_dep", f64p)]:
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = rt
        L.orc_cls.argtypes = [vp]
        L.orc_cls.restype = C.POINTER(C.c_uint8)
        L.orc_allocate_masked.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int,
                                          C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_qd.argtypes = [vp]
        L.orc_qd.restype = C.POINTER(C.c_uint32)
        L.orc_dyn_sizes.argtypes = [vp, C.POINTER(C.c_longlong)]
        for name, rt in [("orc_dyn_chain_g", f32p), ("orc_dyn_chain_u", f32p), ("orc_dyn_proxy", i32p),
                         ("orc_dyn_dir", f32p), ("orc_dyn_cell", i32p), ("orc_dyn_marks", i32p),
                         ("orc_dyn_off", C.POINTER(C.c_uint32)), ("orc_dyn_ray_probe", i32p),
                         ("orc_dyn_ray_key", i32p), ("orc_dyn_t", f32p), ("orc_dyn_tri", i32p),
                         ("orc_dyn_rad", f64p), ("orc_dyn_dep", f64p), ("orc_dyn_tex", i32p),
                         ("orc_dyn_tex_dir", f32p)]:
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = rt
        L.orc_dyn_ntex.argtypes = [vp, C.c_int]
        L.orc_dyn_ntex.restype = C.c_int
        L.orc_texel_centre_dir.argtypes = [C.c_int, C.c_int, C.c_int, f32p]
        L.orc_mh_guide.argtypes = [vp, C.POINTER(OrcFrame), f32p, f32p]
        L.orc_mh_guide.restype = C.c_float
        L.orc_mh_run_table.argtypes = [i32p, f32p, C.c_int, C.c_int, C.c_int, C.c_uint64, f64p]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------- primitives
def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def pilot_dir(seed: int, frame: int, probe: int, octant: int) -> np.ndarray:
    out = np.zeros(3, np.float32)
    lib().orc_pilot_dir(seed, frame, probe, octant, _p(out, C.c_float))
    return out


# packed atlas codec: which = 0 (9-bit irradiance), 1 (8-bit irradiance),
# 2 (13-bit mean distance), 3 (13-bit mean squared distance)
CODEC_BITS = (9, 8, 13, 13)


def codec_enc(which: int, v: float) -> int:
    return int(lib().orc_codec_enc(int(which), float(v)))


def codec_dec(which: int, k: int) -> float:
    return float(lib().orc_codec_dec(int(which), int(k)))


def codec_table(which: int) -> np.ndarray:
    """decoded value of every code (FP32)"""
    return np.array([codec_dec(which, k) for k in range(1 << CODEC_BITS[which])], np.float32)


def mh_normal_quantile(i: int) -> float:
    return float(lib().orc_mh_normal_quantile(int(i)))


def mh_run_table(dims, table, chains, frames, skip, seed=1):
    """chains on a fixed piecewise-constant guide table[probe, octant];
    sample counts per (probe, octant) of frames >= skip"""
    d = np.ascontiguousarray(dims, np.int32)
    t = _f32(table).reshape(-1)
    out = np.zeros(t.shape[0], np.float64)
    lib().orc_mh_run_table(_p(d, C.c_int), _p(t, C.c_float), int(chains), int(frames), int(skip), int(seed),
                           _p(out, C.c_double))
    return out.reshape(-1, 8)


def allocate_masked(W, cls, avg, rmin, rmax):
    """the allocation restricted to the clip volumes (cls per probe: 2, 1, 0)"""
    W = np.ascontiguousarray(W, np.uint32)
    cls = np.ascontiguousarray(cls, np.uint8)
    P = len(W)
    n = np.zeros(P, np.uint32)
    off = np.zeros(P + 1, np.uint32)
    rc = lib().orc_allocate_masked(_p(W, C.c_uint32), _p(cls, C.c_uint8), P, int(avg), int(rmin), int(rmax),
                                   _p(n, C.c_uint32), _p(off, C.c_uint32))
    if rc:
        raise ValueError("invalid allocation arguments")
    return n, off


def texel_centre_dir(cx: int, cy: int, n: int) -> np.ndarray:
    """FP32 direction through the centre of interior texel (cx, cy) of an n x n octahedral grid"""
    w = np.zeros(3, np.float32)
    lib().orc_texel_centre_dir(int(cx), int(cy), int(n), _p(w, C.c_float))
    return w


def mh_exp(k: int) -> float:
    return float(lib().orc_mh_exp(int(k)))


def codec_mav(o: float, v: float, n: int) -> float:
    return float(lib().orc_codec_mav(float(o), float(v), int(n)))


def frame_rotation(seed: int, frame: int) -> np.ndarray:
    out = np.zeros(9, np.float32)
    lib().orc_frame_rotation(seed, frame, _p(out, C.c_float))
    return out.reshape(3, 3)


def sf_points(m: int) -> np.ndarray:
    out = np.zeros((m, 3), np.float32)
    lib().orc_sf_points(m, _p(out, C.c_float))
    return out


def oct_encode(w) -> np.ndarray:
    w = np.ascontiguousarray(w, np.float64)
    out = np.zeros(2, np.float64)
    lib().orc_oct_encode(_p(w, C.c_double), _p(out, C.c_double))
    return out


def oct_decode(p) -> np.ndarray:
    p = np.ascontiguousarray(p, np.float64)
    out = np.zeros(3, np.float64)
    lib().orc_oct_decode(_p(p, C.c_double), _p(out, C.c_double))
    return out


def texel_of_dir(w, n: int) -> int:
    w = _f32(w)
    return int(lib().orc_texel_of_dir(_p(w, C.c_float), n))


def intersect_tri(o, d, A, B, Cv):
    o, d, A, B, Cv = (_f32(x) for x in (o, d, A, B, Cv))
    t = C.c_float(0)
    det = C.c_float(0)
    r = lib().orc_intersect_tri(_p(o, C.c_float), _p(d, C.c_float), _p(A, C.c_float), _p(B, C.c_float),
                                _p(Cv, C.c_float), C.byref(t), C.byref(det))
    return bool(r), t.value, det.value


def trace_closest(V, I, O, D, tmin, tmax, use_bvh=True):
    V = _f32(V).reshape(-1, 3)
    I = np.ascontiguousarray(I, np.int32).reshape(-1, 3)
    O = _f32(O).reshape(-1, 3)
    D = _f32(D).reshape(-1, 3)
    n = O.shape[0]
    t = np.zeros(n, np.float32)
    tri = np.zeros(n, np.int32)
    det = np.zeros(n, np.float32)
    lib().orc_trace_closest(_p(V, C.c_float), V.shape[0], _p(I, C.c_int), I.shape[0], n, _p(O, C.c_float),
                            _p(D, C.c_float), C.c_float(tmin), C.c_float(tmax), int(use_bvh), _p(t, C.c_float),
                            _p(tri, C.c_int), _p(det, C.c_float))
    return t, tri, det


def trace_any(V, I, O, D, tlo, thi, use_bvh=True):
    V = _f32(V).reshape(-1, 3)
    I = np.ascontiguousarray(I, np.int32).reshape(-1, 3)
    O = _f32(O).reshape(-1, 3)
    D = _f32(D).reshape(-1, 3)
    n = O.shape[0]
    out = np.zeros(n, np.uint8)
    lib().orc_trace_any(_p(V, C.c_float), V.shape[0], _p(I, C.c_int), I.shape[0], n, _p(O, C.c_float),
                        _p(D, C.c_float), C.c_float(tlo), C.c_float(thi), int(use_bvh), _p(out, C.c_uint8))
    return out.astype(bool)


def allocate(W, avg, rmin, rmax):
    W = np.ascontiguousarray(W, np.uint32)
    P = W.shape[0]
    n = np.zeros(P, np.uint32)
    off = np.zeros(P + 1, np.uint32)
    r = lib().orc_allocate(_p(W, C.c_uint32), P, avg, rmin, rmax, _p(n, C.c_uint32), _p(off, C.c_uint32))
    if r != 0:
        raise ValueError("allocation budget cannot be met")
    return n, off


def luts(s: float):
    lv = np.zeros(4096, np.uint16)
    lc = np.zeros(4096, np.uint16)
    lib().orc_luts(C.c_double(s), _p(lv, C.c_uint16), _p(lc, C.c_uint16))
    return lv, lc


def border_copy(tile, cnt, n):
    tile = np.ascontiguousarray(tile, np.float64).copy()
    cnt = np.ascontiguousarray(cnt, np.uint8).copy()
    ch = tile.shape[-1]
    lib().orc_border_copy(_p(tile, C.c_double), _p(cnt, C.c_uint8), n, ch)
    return tile, cnt


# ---------------------------------------------------------------- volume
def make_frame(frame, seed, lights, sky=(0.0, 0.0, 0.0), camera=None):
    """lights: list of (kind, (x,y,z), (r,g,b)); camera: None, (pos, k), or
    (pos, k, M) with M the row-major 4x4 view-projection matrix of the clip
    volumes (Fig. TrCam(b))."""
    arr = (OrcLight * max(1, len(lights)))()
    for i, (kind, v, rgb) in enumerate(lights):
        arr[i].kind = int(kind)
        arr[i].v[:] = [float(x) for x in v]
        arr[i].rgb[:] = [float(x) for x in rgb]
    fr = OrcFrame()
    fr.frame = int(frame)
    fr.seed = int(seed)
    fr.lights = C.cast(arr, C.POINTER(OrcLight))
    fr.n_lights = len(lights)
    fr.sky[:] = [float(x) for x in sky]
    if camera is not None:
        fr.has_camera = 1
        fr.cam[:] = [float(x) for x in camera[0]]
        fr.cam_k = float(camera[1])
        if len(camera) > 2 and camera[2] is not None:
            fr.has_clip = 1
            fr.clip[:] = [float(x) for x in np.asarray(camera[2], np.float32).reshape(16)]
    fr._keep = arr
    return fr


class OracleVolume:
    """FP64 oracle volume with the same five-call shape as the C-ABI."""

    def __init__(self, origin, spacing, dims, n_irr=6, n_dep=14, rays_avg=64, rays_min=8, rays_max=256,
                 hysteresis=0.97, depth_max=0.0, theta=16, threads=None, packed=False, sampler=0, alpha=1.0,
                 dyn_ratio=0, hyst_dyn=0.91, blend_mode=0, cheb_var_floor_rel=0.0):
        d = OrcDesc()
        d.origin[:] = [float(x) for x in origin]
        d.spacing[:] = [float(x) for x in spacing]
        d.dims[:] = [int(x) for x in dims]
        d.n_irr, d.n_dep = int(n_irr), int(n_dep)
        d.avg, d.rmin, d.rmax = int(rays_avg), int(rays_min), int(rays_max)
        d.hyst = float(hysteresis)
        d.depth_max = float(depth_max)
        d.theta = int(theta)
        d.packed = int(bool(packed))
        self.packed = bool(packed)
        d.sampler = int(sampler)
        d.alpha = float(alpha)
        d.blend_mode = int(blend_mode)
        d.dyn_ratio = int(dyn_ratio)
        d.hyst_dyn = float(hyst_dyn)
        d.var_rel = float(cheb_var_floor_rel)
        self.desc = d
        if threads is None:
            threads = os.cpu_count() or 1
        self.h = lib().orc_create(C.byref(d), int(threads))
        if not self.h:
            raise ValueError("invalid volume description")
        self.P = int(dims[0]) * int(dims[1]) * int(dims[2])
        self.Ti, self.Td = n_irr + 2, n_dep + 2
        self.n_irr, self.n_dep = n_irr, n_dep

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scene(self, verts, idx, albedo):
        V = _f32(verts).reshape(-1, 3)
        I = np.ascontiguousarray(idx, np.int32).reshape(-1, 3)
        A = _f32(albedo).reshape(-1, 3)
        self._scene = (V, I, A)
        r = lib().orc_set_scene(self.h, _p(V, C.c_float), V.shape[0], _p(I, C.c_int), I.shape[0], _p(A, C.c_float))
        if r:
            raise ValueError("bad scene")

    def move_vertices(self, first, verts):
        V = _f32(verts).reshape(-1, 3)
        r = lib().orc_move_vertices(self.h, int(first), V.shape[0], _p(V, C.c_float))
        if r:
            raise ValueError("bad vertex range")

    def update(self, frame, seed, lights, sky=(0, 0, 0), camera=None):
        fr = make_frame(frame, seed, lights, sky, camera)
        r = lib().orc_update(self.h, C.byref(fr))
        if r:
            raise RuntimeError("oracle update failed")

    # ---- probe-slab split (one rank's share of an update; see orc_slab_*)
    SLAB = {"TRV": (0, np.uint16, 8), "TRR": (1, np.uint16, 8), "W": (2, np.uint32, 1), "IRR": (3, np.float64, None),
            "IRR_N": (4, np.uint8, None), "DEP": (5, np.float64, None), "DEP_N": (6, np.uint8, None)}

    def _slab_call(self, fn, frame, seed, lights, p0, p1, sky, camera):
        self._fr = make_frame(frame, seed, lights, sky, camera)
        if getattr(lib(), fn)(self.h, C.byref(self._fr), int(p0), int(p1)):
            raise ValueError(fn + " failed")

    def slab_begin(self, frame, seed, lights, p0, p1, sky=(0, 0, 0), camera=None):
        self._slab_call("orc_slab_begin", frame, seed, lights, p0, p1, sky, camera)

    def slab_weights(self, frame, seed, lights, p0, p1, sky=(0, 0, 0), camera=None):
        self._slab_call("orc_slab_weights", frame, seed, lights, p0, p1, sky, camera)

    def slab_finish(self, frame, seed, lights, p0, p1, sky=(0, 0, 0), camera=None):
        self._slab_call("orc_slab_finish", frame, seed, lights, p0, p1, sky, camera)

    def _slab_elems(self, which):
        code, dt, per = self.SLAB[which]
        if per is None:
            per = {"IRR": self.Ti * self.Ti * 3, "IRR_N": self.Ti * self.Ti, "DEP": self.Td * self.Td * 2,
                   "DEP_N": self.Td * self.Td}[which]
        return code, dt, per

    def slab_get(self, which, p0, p1):
        code, dt, per = self._slab_elems(which)
        out = np.empty((p1 - p0) * per, dt)
        if lib().orc_slab_slice(self.h, code, int(p0), int(p1), out.ctypes.data, 0) != out.nbytes:
            raise ValueError("bad slice")
        return out

    def slab_set(self, which, p0, p1, data):
        code, dt, per = self._slab_elems(which)
        a = np.ascontiguousarray(data, dt).reshape(-1)
        if a.size != (p1 - p0) * per or lib().orc_slab_slice(self.h, code, int(p0), int(p1), a.ctypes.data, 1) != a.nbytes:
            raise ValueError("bad slice")

    def set_threads(self, n):
        """threads for the later phases (timing only: results do not depend on it)"""
        lib().orc_set_threads(self.h, int(n))

    def trace_shade_probes(self, frame, seed, lights, probes, sky=(0, 0, 0)):
        fr = make_frame(frame, seed, lights, sky)
        pr = np.ascontiguousarray(probes, np.int32)
        return int(lib().orc_trace_shade_probes(self.h, C.byref(fr), _p(pr, C.c_int), pr.shape[0]))

    def change_from_pilots(self, frame, pilot_t, pilot_tri, pilot_lum, camera=None, seed=0):
        fr = make_frame(frame, seed, [], (0, 0, 0), camera)
        t = _f32(pilot_t).reshape(-1)
        tri = np.ascontiguousarray(pilot_tri, np.int32).reshape(-1)
        lum = _f32(pilot_lum).reshape(-1)
        lib().orc_change_from_pilots(self.h, C.byref(fr), _p(t, C.c_float), _p(tri, C.c_int), _p(lum, C.c_float))

    def query(self, pos, nrm):
        pos = _f32(pos).reshape(-1, 3)
        nrm = _f32(nrm).reshape(-1, 3)
        out = np.zeros((pos.shape[0], 3), np.float64)
        lib().orc_query(self.h, pos.shape[0], _p(pos, C.c_float), _p(nrm, C.c_float), _p(out, C.c_double))
        return out

    def _arr(self, name, count, dtype, shape=None):
        ptr = getattr(lib(), name)(self.h)
        a = np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True)
        return a.reshape(shape) if shape is not None else a

    @property
    def n_main(self):
        return int(lib().orc_num_main_rays(self.h))

    def irr(self):
        return self._arr("orc_irr", self.P * self.Ti * self.Ti * 3, np.float64, (self.P, self.Ti, self.Ti, 3))

    def irr_n(self):
        return self._arr("orc_irr_n", self.P * self.Ti * self.Ti, np.uint8, (self.P, self.Ti, self.Ti))

    def dep(self):
        return self._arr("orc_dep", self.P * self.Td * self.Td * 2, np.float64, (self.P, self.Td, self.Td, 2))

    def dep_n(self):
        return self._arr("orc_dep_n", self.P * self.Td * self.Td, np.uint8, (self.P, self.Td, self.Td))

    def irr_packed(self):
        """packed irradiance codes (R bits 0-8, G 9-17, B 18-25, N 26-31)"""
        return self._arr("orc_irr_packed", self.P * self.Ti * self.Ti, np.uint32, (self.P, self.Ti, self.Ti))

    def dep_packed(self):
        """packed visibility codes (mean 0-12, mean square 13-25, N 26-31)"""
        return self._arr("orc_dep_packed", self.P * self.Td * self.Td, np.uint32, (self.P, self.Td, self.Td))

    @property
    def cage_diag(self):
        return float(lib().orc_cage_diag(self.h))

    def blend_packed_records(self, p, use_pilots, pil_rad=None, pil_dep=None, m_rad=None, m_dep=None):
        def ptr(a):
            return None if a is None else _p(np.ascontiguousarray(a, np.float64), C.c_double)
        keep = [None if a is None else np.ascontiguousarray(a, np.float64) for a in (pil_rad, pil_dep, m_rad, m_dep)]
        lib().orc_blend_packed_records(self.h, int(p), int(bool(use_pilots)),
                                       *[None if a is None else _p(a, C.c_double) for a in keep])

    # Metropolis sampler (sampler=1): this frame's samples
    @property
    def mh_samples(self):
        return int(lib().orc_mh_samples(self.h))

    @property
    def mh_chains(self):
        return int(lib().orc_mh_chains(self.h))

    def mh_probe(self):
        return self._arr("orc_mh_probe", self.mh_samples, np.int32)

    def mh_dir(self):
        return self._arr("orc_mh_dir", self.mh_samples * 3, np.float32, (self.mh_samples, 3))

    def mh_tri(self):
        return self._arr("orc_mh_tri", self.mh_samples, np.int32)

    def mh_t(self):
        return self._arr("orc_mh_t", self.mh_samples, np.float32)

    def mh_t_neg(self):
        return self._arr("orc_mh_t_neg", self.mh_samples, np.float32)

    def mh_tri_neg(self):
        return self._arr("orc_mh_tri_neg", self.mh_samples, np.int32)

    def mh_rad(self):
        return self._arr("orc_mh_rad", self.mh_samples * 3, np.float64, (self.mh_samples, 3))

    def mh_dep(self):
        return self._arr("orc_mh_dep", self.mh_samples, np.float64)

    def cls(self):
        """clip volume of each probe this frame: 2 V_in, 1 V_out - V_in, 0 outside"""
        return self._arr("orc_cls", self.P, np.uint8)

    def qd(self):
        """per (probe, octant) dynamic weight q_d of the last update"""
        return self._arr("orc_qd", self.P * 8, np.uint32, (self.P, 8))

    # dynamic chains (dyn_ratio > 0)
    def dyn_sizes(self):
        """dict: chains, samples, ray budget, rays this frame, marked cells, traced cells, proxies"""
        out = (C.c_longlong * 8)()
        lib().orc_dyn_sizes(self.h, out)
        return dict(zip(("chains", "samples", "budget", "rays", "marked", "traced", "proxies"), [int(x) for x in out]))

    def dyn_chain_state(self):
        n = self.dyn_sizes()["chains"]
        return (self._arr("orc_dyn_chain_g", n * 3, np.float32, (n, 3)),
                self._arr("orc_dyn_chain_u", n * 2, np.float32, (n, 2)))

    def dyn_samples(self):
        """(proxy int32[Bd], direction float32[Bd, 3], cell int32[Bd] (-1: target 0))"""
        n = self.dyn_sizes()["samples"]
        return (self._arr("orc_dyn_proxy", n, np.int32), self._arr("orc_dyn_dir", n * 3, np.float32, (n, 3)),
                self._arr("orc_dyn_cell", n, np.int32))

    def dyn_marks(self):
        """marked cells in first-sample order, and how many of them were traced"""
        s = self.dyn_sizes()
        return self._arr("orc_dyn_marks", s["marked"], np.int32), s["traced"]

    def dyn_rays(self):
        """dict of this frame's dynamic rays grouped by probe"""
        n = self.dyn_sizes()["rays"]
        return {"off": self._arr("orc_dyn_off", self.P + 1, np.uint32),
                "probe": self._arr("orc_dyn_ray_probe", n, np.int32), "key": self._arr("orc_dyn_ray_key", n, np.int32),
                "t": self._arr("orc_dyn_t", n, np.float32), "tri": self._arr("orc_dyn_tri", n, np.int32),
                "rad": self._arr("orc_dyn_rad", n * 3, np.float64, (n, 3)), "dep": self._arr("orc_dyn_dep", n, np.float64)}

    def dyn_texels(self):
        """per octant: (tile texel indices, centre directions) of the irradiance texels whose centre lies in it"""
        nn = self.n_irr * self.n_irr
        t = self._arr("orc_dyn_tex", 8 * nn, np.int32, (8, nn))
        d = self._arr("orc_dyn_tex_dir", 8 * nn * 3, np.float32, (8, nn, 3))
        out = []
        for o in range(8):
            k = int(lib().orc_dyn_ntex(self.h, o))
            out.append((t[o, :k].copy(), d[o, :k].copy()))
        return out

    def mh_chain_state(self):
        C_ = self.mh_chains
        return (self._arr("orc_mh_chain_g", C_ * 3, np.float32, (C_, 3)),
                self._arr("orc_mh_chain_u", C_ * 2, np.float32, (C_, 2)))

    def mh_guide(self, frame, g, u, camera=None, seed=0):
        fr = make_frame(frame, seed, [], (0, 0, 0), camera)
        g = _f32(g).reshape(3)
        u = _f32(u).reshape(2)
        return float(lib().orc_mh_guide(self.h, C.byref(fr), _p(g, C.c_float), _p(u, C.c_float)))

    def W(self):
        return self._arr("orc_W", self.P, np.uint32)

    def n(self):
        return self._arr("orc_n", self.P, np.uint32)

    def off(self):
        return self._arr("orc_off", self.P + 1, np.uint32)

    def qv(self):
        return self._arr("orc_qv", self.P * 8, np.uint16, (self.P, 8))

    def qr(self):
        return self._arr("orc_qr", self.P * 8, np.uint16, (self.P, 8))

    def trv(self):
        return self._arr("orc_trv", self.P * 8, np.uint16, (self.P, 8))

    def trr(self):
        return self._arr("orc_trr", self.P * 8, np.uint16, (self.P, 8))

    def pilot_t(self):
        return self._arr("orc_pil_t", self.P * 8, np.float32, (self.P, 8))

    def pilot_tri(self):
        return self._arr("orc_pil_tri", self.P * 8, np.int32, (self.P, 8))

    def pilot_lum(self):
        return self._arr("orc_pil_lum", self.P * 8, np.float32, (self.P, 8))

    def pilot_dir(self):
        return self._arr("orc_pil_dir", self.P * 24, np.float32, (self.P, 8, 3))

    def pilot_rad(self):
        return self._arr("orc_pil_rad", self.P * 24, np.float64, (self.P, 8, 3))

    def pilot_dep(self):
        return self._arr("orc_pil_dep", self.P * 8, np.float64, (self.P, 8))

    def main_t(self):
        n = int(self.off()[-1])
        return self._arr("orc_m_t", n, np.float32)

    def main_tri(self):
        n = int(self.off()[-1])
        return self._arr("orc_m_tri", n, np.int32)

    def main_rad(self):
        n = int(self.off()[-1])
        return self._arr("orc_m_rad", n * 3, np.float64, (n, 3))

    def main_dep(self):
        n = int(self.off()[-1])
        return self._arr("orc_m_dep", n, np.float64)

    def rotation(self):
        return self._arr("orc_rot", 9, np.float32, (3, 3))

    def probe_pos(self, p):
        out = np.zeros(3, np.float32)
        lib().orc_probe_pos(self.h, int(p), _p(out, C.c_float))
        return out

    def main_dir(self, m, i):
        out = np.zeros(3, np.float32)
        lib().orc_main_dir(self.h, int(m), int(i), _p(out, C.c_float))
        return out

    @property
    def voxel_diag(self):
        return float(lib().orc_voxel_diag(self.h))

    @property
    def depth_max(self):
        return float(lib().orc_depth_max(self.h))

    @property
    def tmin(self):
        return float(lib().orc_tmin(self.h))

    def set_atlas(self, irr=None, irr_n=None, dep=None, dep_n=None):
        def ptr(a, ct, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dt)
            self._hold = getattr(self, "_hold", []) + [a]
            return _p(a, ct)

        lib().orc_set_atlas(self.h, ptr(irr, C.c_double, np.float64), ptr(irr_n, C.c_uint8, np.uint8),
                            ptr(dep, C.c_double, np.float64), ptr(dep_n, C.c_uint8, np.uint8))
