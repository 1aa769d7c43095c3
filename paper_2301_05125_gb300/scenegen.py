"""Seeded synthetic workloads (input data only).

This module builds the triangle scenes, light schedules, moving occluders and
probe-grid descriptions that stand in for the paper's Bistro / Sponza / Buddha
scenes (not available here).  It holds none of the update's arithmetic and is
the one module that both the CUDA path's tests/bench and the CPU oracle use.

Workloads (sizes of the paper's evaluation, Sec. 5, scaled as stated):
  * ``box_room``   -- 12 axis-aligned boxes (144 triangles; box 0 is the room
                      shell [0,8]^3 facing inward), 1 point light on a circle
                      (1 revolution / 64 frames), 4x4x4 probes, 64 rays/probe
                      (min 8, max 256), FP32, hysteresis 0.97.
  * ``tunnel_city``-- 15k random boxes (log-uniform sizes) on a 400 x 400 m
                      ground + a 64-segment x 160-ring cylindrical tunnel +
                      20 moving occluder boxes (about 200k triangles), 3 moving
                      point lights + sun, 32x16x32 probes, 256 rays/probe
                      (min 8, max 1024).
  * ``scaled``     -- the same generator at about 2M triangles, 64x32x64
                      probes, 64 rays/probe (min 4, max 512).
"""
from dataclasses import dataclass, field
from typing import Callable, List, Tuple

import numpy as np

Light = Tuple[int, Tuple[float, float, float], Tuple[float, float, float]]

# unit cube corners, index bits (x, y, z)
_CORNERS = np.array([[(i >> 0) & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], np.float64)


def _cube_faces() -> np.ndarray:
    """12 triangles of the unit cube with outward normals (B-A)x(C-A)."""
    tris = []
    for axis in range(3):
        for side in (0, 1):
            corners = [i for i in range(8) if ((i >> axis) & 1) == side]
            # order the 4 corners of the face around its centre
            pts = _CORNERS[corners]
            ctr = pts.mean(axis=0)
            u, v = [a for a in range(3) if a != axis]
            ang = np.arctan2(pts[:, v] - ctr[v], pts[:, u] - ctr[u])
            ring = [corners[k] for k in np.argsort(ang)]
            for a, b, c in ((ring[0], ring[1], ring[2]), (ring[0], ring[2], ring[3])):
                n = np.cross(_CORNERS[b] - _CORNERS[a], _CORNERS[c] - _CORNERS[a])
                out = np.zeros(3)
                out[axis] = 1.0 if side == 1 else -1.0
                if np.dot(n, out) < 0:
                    b, c = c, b
                tris.append((a, b, c))
    return np.array(tris, np.int32)


_CUBE_TRIS = _cube_faces()


def boxes_mesh(lo: np.ndarray, hi: np.ndarray, inward: bool = False):
    """Vertices (8 per box) and triangles (12 per box) of axis-aligned boxes."""
    lo = np.asarray(lo, np.float64).reshape(-1, 3)
    hi = np.asarray(hi, np.float64).reshape(-1, 3)
    nb = lo.shape[0]
    verts = lo[:, None, :] + _CORNERS[None, :, :] * (hi - lo)[:, None, :]
    tris = _CUBE_TRIS[None, :, :] + 8 * np.arange(nb, dtype=np.int32)[:, None, None]
    if inward:
        tris = tris[:, :, [0, 2, 1]]
    return verts.reshape(-1, 3).astype(np.float32), tris.reshape(-1, 3).astype(np.int32)


def cylinder_mesh(x0, x1, radius, cy, cz, segments, rings, inward=True):
    """Open cylinder along x (a tunnel), segments around, rings along."""
    xs = np.linspace(x0, x1, rings + 1)
    ang = 2.0 * np.pi * np.arange(segments) / segments
    y = cy + radius * np.cos(ang)
    z = cz + radius * np.sin(ang)
    verts = np.stack([np.repeat(xs, segments), np.tile(y, rings + 1), np.tile(z, rings + 1)], axis=1)
    tris = []
    for r in range(rings):
        for s in range(segments):
            a = r * segments + s
            b = r * segments + (s + 1) % segments
            c = (r + 1) * segments + s
            d = (r + 1) * segments + (s + 1) % segments
            tris.append((a, b, d))
            tris.append((a, d, c))
    tris = np.array(tris, np.int32)
    # orient: inward normals point towards the axis
    v = verts.astype(np.float64)
    n = np.cross(v[tris[:, 1]] - v[tris[:, 0]], v[tris[:, 2]] - v[tris[:, 0]])
    ctr = v[tris].mean(axis=1)
    to_axis = np.stack([np.zeros(len(tris)), cy - ctr[:, 1], cz - ctr[:, 2]], axis=1)
    flip = (np.einsum("ij,ij->i", n, to_axis) < 0) if inward else (np.einsum("ij,ij->i", n, to_axis) > 0)
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts.astype(np.float32), tris


def grid_plane(x0, x1, z0, z1, y, nx, nz):
    """Upward-facing ground plane split into nx x nz quads."""
    xs = np.linspace(x0, x1, nx + 1)
    zs = np.linspace(z0, z1, nz + 1)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    verts = np.stack([X.ravel(), np.full(X.size, y), Z.ravel()], axis=1)
    tris = []
    for i in range(nx):
        for k in range(nz):
            a = i * (nz + 1) + k
            b = (i + 1) * (nz + 1) + k
            c = i * (nz + 1) + k + 1
            d = (i + 1) * (nz + 1) + k + 1
            tris.append((a, c, d))
            tris.append((a, d, b))
    tris = np.array(tris, np.int32)
    v = verts
    n = np.cross(v[tris[:, 1]] - v[tris[:, 0]], v[tris[:, 2]] - v[tris[:, 0]])
    flip = n[:, 1] < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts.astype(np.float32), tris


def uv_sphere(center, radius, n_seg, n_ring, inward=True):
    """Triangulated sphere (n_seg around, n_ring from pole to pole)."""
    center = np.asarray(center, np.float64)
    verts = [center + [0, 0, radius]]
    for r in range(1, n_ring):
        th = np.pi * r / n_ring
        for s in range(n_seg):
            ph = 2 * np.pi * s / n_seg
            verts.append(center + radius * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]))
    verts.append(center + [0, 0, -radius])
    verts = np.array(verts)
    tris = []
    for s in range(n_seg):
        tris.append((0, 1 + s, 1 + (s + 1) % n_seg))
    for r in range(n_ring - 2):
        for s in range(n_seg):
            a = 1 + r * n_seg + s
            b = 1 + r * n_seg + (s + 1) % n_seg
            c = 1 + (r + 1) * n_seg + s
            d = 1 + (r + 1) * n_seg + (s + 1) % n_seg
            tris.append((a, c, d))
            tris.append((a, d, b))
    last = len(verts) - 1
    base = 1 + (n_ring - 2) * n_seg
    for s in range(n_seg):
        tris.append((last, base + (s + 1) % n_seg, base + s))
    tris = np.array(tris, np.int32)
    n = np.cross(verts[tris[:, 1]] - verts[tris[:, 0]], verts[tris[:, 2]] - verts[tris[:, 0]])
    out = verts[tris].mean(axis=1) - center
    flip = (np.einsum("ij,ij->i", n, out) > 0) if inward else (np.einsum("ij,ij->i", n, out) < 0)
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts.astype(np.float32), tris


@dataclass
class Workload:
    name: str
    seed: int
    verts: np.ndarray          # (nv, 3) float32
    idx: np.ndarray            # (nt, 3) int32
    albedo: np.ndarray         # (nt, 3) float32
    volume: dict               # probe grid / budget description
    frames: int
    sky: Tuple[float, float, float]
    lights_at: Callable[[int], List[Light]]
    dyn_first: int = 0         # first moving vertex
    dyn_count: int = 0         # number of moving vertices
    dyn_at: Callable[[int], np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n_tris(self):
        return int(self.idx.shape[0])

    @property
    def n_probes(self):
        d = self.volume["dims"]
        return int(d[0] * d[1] * d[2])

    @property
    def rays_per_update(self):
        return self.n_probes * int(self.volume["rays_avg"])


def box_room(seed: int = 1) -> Workload:
    rng = np.random.default_rng(seed)
    lo = [np.zeros(3)]
    hi = [np.full(3, 8.0)]
    for _ in range(11):
        size = rng.uniform(0.5, 2.0, 3)
        size[1] = rng.uniform(0.5, 3.0)
        pos = rng.uniform(0.5, 7.5 - size)
        pos[1] = 0.0
        lo.append(pos)
        hi.append(pos + size)
    v_shell, t_shell = boxes_mesh(lo[:1], hi[:1], inward=True)
    v_box, t_box = boxes_mesh(np.array(lo[1:]), np.array(hi[1:]))
    verts = np.concatenate([v_shell, v_box])
    idx = np.concatenate([t_shell, t_box + len(v_shell)])
    box_alb = rng.uniform(0.2, 0.9, (12, 3)).astype(np.float32)
    albedo = np.repeat(box_alb, 12, axis=0)

    def lights_at(f):
        a = 2.0 * np.pi * f / 64.0
        return [(0, (4.0 + 3.0 * np.cos(a), 6.5, 4.0 + 3.0 * np.sin(a)), (40.0, 36.0, 30.0))]

    vol = dict(origin=(1.0, 1.0, 1.0), spacing=(2.0, 2.0, 2.0), dims=(4, 4, 4), irr_interior=6, depth_interior=14,
               rays_avg=64, rays_min=8, rays_max=256, hysteresis=0.97, depth_max=0.0, atlas_fp16=0, tr_theta=16)
    return Workload("box_room", seed, verts, idx, albedo, vol, 4, (0.0, 0.0, 0.0), lights_at)


def _city(seed, n_boxes, rings, dims, origin, spacing, rays_avg, rays_min, rays_max, frames, name):
    rng = np.random.default_rng(seed)
    parts_v, parts_t, parts_a = [], [], []
    nv = 0

    def add(v, t, alb):
        nonlocal nv
        parts_v.append(v)
        parts_t.append(t + nv)
        parts_a.append(np.broadcast_to(np.asarray(alb, np.float32), (len(t), 3)))
        nv += len(v)

    gv, gt = grid_plane(-200.0, 200.0, -200.0, 200.0, 0.0, 32, 32)
    add(gv, gt, (0.45, 0.43, 0.40))
    # static boxes, kept out of the tunnel corridor
    sx = np.exp(rng.uniform(np.log(1.0), np.log(12.0), n_boxes))
    sz = np.exp(rng.uniform(np.log(1.0), np.log(12.0), n_boxes))
    sy = np.exp(rng.uniform(np.log(1.0), np.log(30.0), n_boxes))
    px = rng.uniform(-200.0, 200.0 - sx)
    pz = rng.uniform(-200.0, 200.0 - sz)
    clear = ~((px < 84) & (px + sx > -84) & (pz < 9) & (pz + sz > -9))
    px, pz, sx, sy, sz = px[clear], pz[clear], sx[clear], sy[clear], sz[clear]
    lo = np.stack([px, np.zeros_like(px), pz], 1)
    hi = lo + np.stack([sx, sy, sz], 1)
    bv, bt = boxes_mesh(lo, hi)
    balb = rng.uniform(0.2, 0.9, (len(lo), 3)).astype(np.float32)
    parts_v.append(bv)
    parts_t.append(bt + nv)
    parts_a.append(np.repeat(balb, 12, axis=0))
    nv += len(bv)
    cv, ct = cylinder_mesh(-80.0, 80.0, 7.0, 3.0, 0.0, 64, rings, inward=True)
    add(cv, ct, (0.6, 0.6, 0.62))
    # 20 moving occluder boxes: gates at the two tunnel mouths and blocks near the probes
    n_occ = 20
    occ_lo = np.zeros((n_occ, 3))
    occ_size = np.zeros((n_occ, 3))
    occ_axis = np.zeros(n_occ, np.int64)
    occ_amp = np.zeros(n_occ)
    occ_period = np.zeros(n_occ)
    occ_phase = np.zeros(n_occ)
    for i in range(n_occ):
        if i < 4:
            occ_lo[i] = ((-82.0 if i % 2 == 0 else 80.0), 0.0, -8.0 + 8.0 * (i // 2))
            occ_size[i] = (2.0, 10.0, 8.0)
            occ_axis[i] = 1
            occ_amp[i] = 9.0
        else:
            occ_lo[i] = (rng.uniform(-60, 50), 0.0, rng.uniform(-60, 50))
            occ_size[i] = (rng.uniform(2, 6), rng.uniform(3, 12), rng.uniform(2, 6))
            occ_axis[i] = rng.integers(0, 3) if False else (0 if i % 2 else 2)
            occ_amp[i] = rng.uniform(4.0, 12.0)
        occ_period[i] = rng.uniform(24.0, 64.0)
        occ_phase[i] = rng.uniform(0.0, 2 * np.pi)
    ov, ot = boxes_mesh(occ_lo, occ_lo + occ_size)
    oalb = rng.uniform(0.2, 0.9, (n_occ, 3)).astype(np.float32)
    dyn_first = nv
    parts_v.append(ov)
    parts_t.append(ot + nv)
    parts_a.append(np.repeat(oalb, 12, axis=0))
    nv += len(ov)
    verts = np.concatenate(parts_v).astype(np.float32)
    idx = np.concatenate(parts_t).astype(np.int32)
    albedo = np.ascontiguousarray(np.concatenate(parts_a), np.float32)

    def dyn_at(f):
        off = np.zeros((n_occ, 3))
        s = np.sin(2 * np.pi * f / occ_period + occ_phase)
        off[np.arange(n_occ), occ_axis] = occ_amp * s
        off[:4, 1] = occ_amp[:4] * 0.5 * (1.0 + s[:4])  # gates slide up and down
        lo_f = occ_lo + off
        v, _ = boxes_mesh(lo_f, lo_f + occ_size)
        return v

    lp = rng.uniform(0, 2 * np.pi, 3)
    lr = rng.uniform(20.0, 50.0, 3)
    lh = rng.uniform(15.0, 35.0, 3)
    lc = rng.uniform(-30.0, 30.0, (3, 2))

    def lights_at(f):
        out = []
        for k in range(3):
            a = lp[k] + 2 * np.pi * f / (48.0 + 16.0 * k)
            out.append((0, (lc[k, 0] + lr[k] * np.cos(a), lh[k], lc[k, 1] + lr[k] * np.sin(a)),
                        (3000.0, 2800.0, 2500.0)))
        out.append((1, (-0.3, -1.0, -0.2), (2.0, 1.9, 1.7)))
        return out

    vol = dict(origin=origin, spacing=spacing, dims=dims, irr_interior=6, depth_interior=14, rays_avg=rays_avg,
               rays_min=rays_min, rays_max=rays_max, hysteresis=0.97, depth_max=0.0, atlas_fp16=0, tr_theta=16)
    return Workload(name, seed, verts, idx, albedo, vol, frames, (0.3, 0.4, 0.6), lights_at,
                    dyn_first=dyn_first, dyn_count=len(ov), dyn_at=dyn_at,
                    meta=dict(n_static_boxes=int(len(lo)), n_occluders=n_occ))


def tunnel_city(seed: int = 1, n_boxes: int = 15000) -> Workload:
    return _city(seed, n_boxes, 160, (32, 16, 32), (-62.0, 1.0, -62.0), (4.0, 4.0, 4.0), 256, 8, 1024, 60,
                 "tunnel_city")


def scaled(seed: int = 1, n_boxes: int = 165000) -> Workload:
    return _city(seed, n_boxes, 320, (64, 32, 64), (-126.0, 1.0, -126.0), (4.0, 4.0, 4.0), 64, 4, 512, 30,
                 "scaled")


def small_city(seed: int = 1, n_boxes: int = 600, dims=(8, 4, 8), rays_avg=48) -> Workload:
    """A reduced tunnel+city (same generator) that the oracle finishes in
    seconds while still spanning many probes, tiles and a ragged tail."""
    return _city(seed, n_boxes, 20, dims, (-30.0, 1.0, -30.0), (8.0, 8.0, 8.0), rays_avg, 8, 160, 4, "small_city")


def batched(seed: int = 1, n_volumes: int = 24, n_scenes: int = 6, tri_lo: float = 20e3, tri_hi: float = 500e3,
            dims_lo=(8, 8, 8), dims_hi=(48, 16, 48), rays_avg: int = 64, fp16: int = 1) -> List[Workload]:
    """Batched volumes: n_volumes probe volumes of uneven size (dims log-uniform
    between dims_lo and dims_hi) over n_scenes seeded city scenes whose
    triangle counts are log-uniform in [tri_lo, tri_hi]; every volume has its
    own light phase and occluder motion; FP16 atlases."""
    rng = np.random.default_rng(seed)
    tris = np.exp(rng.uniform(np.log(tri_lo), np.log(tri_hi), n_scenes))
    scenes = []
    for k in range(n_scenes):
        # fixed part: ground 2048 + tunnel 64x40x2 + occluders 240 triangles;
        # about 3% of the boxes fall in the tunnel corridor and are dropped
        n_boxes = max(100, int((tris[k] - 7408) / 12 / 0.97))
        scenes.append(_city(seed * 100 + k, n_boxes, 40, (2, 2, 2), (0.0, 1.0, 0.0), (4.0, 4.0, 4.0), 64, 8, 256, 1,
                            "scene%d" % k))
    out = []
    for i in range(n_volumes):
        base = scenes[i % n_scenes]
        dims = tuple(int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for lo, hi in zip(dims_lo, dims_hi))
        spacing = 3.0 + 2.0 * rng.random()
        origin = (-dims[0] * spacing / 2 + rng.uniform(-20, 20), 1.0, -dims[2] * spacing / 2 + rng.uniform(-20, 20))
        phase = 7 * i
        vol = dict(origin=origin, spacing=(spacing, spacing, spacing), dims=dims, irr_interior=6, depth_interior=14,
                   rays_avg=rays_avg, rays_min=8, rays_max=256, hysteresis=0.97, depth_max=0.0, atlas_fp16=fp16,
                   tr_theta=16)
        w = Workload("batched%d" % i, seed * 1000 + i, base.verts, base.idx, base.albedo, vol, 30, base.sky,
                     (lambda f, b=base, ph=phase: b.lights_at(f + ph)), dyn_first=base.dyn_first,
                     dyn_count=base.dyn_count, dyn_at=(lambda f, b=base, ph=phase: b.dyn_at(f + ph)),
                     meta=dict(scene=i % n_scenes, scene_tris=int(base.n_tris)))
        out.append(w)
    return out


def serving(seed: int = 1, n_clients: int = 64, n_scenes: int = 8, tri_lo: float = 50e3, tri_hi: float = 1e6,
            probes_lo: int = 512, probes_hi: int = 65536, rays_avg: int = 64, fp16: int = 1) -> List[Workload]:
    """Serving mix: n_clients volumes, each owned by one client, whose probe
    counts are log-uniform in [probes_lo, probes_hi] (grids 2a x a x 2a) over
    n_scenes seeded city scenes of log-uniform triangle count in [tri_lo,
    tri_hi]; every volume has its own light phase and occluder motion."""
    rng = np.random.default_rng(seed)
    tris = np.exp(rng.uniform(np.log(tri_lo), np.log(tri_hi), n_scenes))
    scenes = []
    for k in range(n_scenes):
        n_boxes = max(100, int((tris[k] - 7408) / 12 / 0.97))
        scenes.append(_city(seed * 100 + 50 + k, n_boxes, 40, (2, 2, 2), (0.0, 1.0, 0.0), (4.0, 4.0, 4.0), 64, 8,
                            256, 1, "scene%d" % k))
    out = []
    for i in range(n_clients):
        base = scenes[i % n_scenes]
        P = np.exp(rng.uniform(np.log(probes_lo), np.log(probes_hi)))
        a = max(4, int(round((P / 4.0) ** (1.0 / 3.0))))
        dims = (2 * a, a, 2 * a)
        spacing = float(np.clip(160.0 / (2 * a), 2.0, 8.0))
        origin = (-a * spacing + rng.uniform(-30, 30), 1.0, -a * spacing + rng.uniform(-30, 30))
        phase = 5 * i
        vol = dict(origin=origin, spacing=(spacing, spacing, spacing), dims=dims, irr_interior=6, depth_interior=14,
                   rays_avg=rays_avg, rays_min=8, rays_max=256, hysteresis=0.97, depth_max=0.0, atlas_fp16=fp16,
                   tr_theta=16)
        out.append(Workload("client%d" % i, seed * 1000 + i, base.verts, base.idx, base.albedo, vol, 0, base.sky,
                            (lambda f, b=base, ph=phase: b.lights_at(f + ph)), dyn_first=base.dyn_first,
                            dyn_count=base.dyn_count, dyn_at=(lambda f, b=base, ph=phase: b.dyn_at(f + ph)),
                            meta=dict(scene=i % n_scenes, scene_tris=int(base.n_tris))))
    return out


def poisson_schedule(seed: int, n_clients: int, rate_hz: float, n_requests: int):
    """Arrival times (s) and client ids of the first n_requests arrivals of
    n_clients independent Poisson processes of rate rate_hz each."""
    rng = np.random.default_rng(seed)
    per = int(np.ceil(n_requests / n_clients * 1.5)) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_hz, (n_clients, per)), axis=1)
    cid = np.repeat(np.arange(n_clients), per)
    order = np.argsort(t.ravel(), kind="stable")[:n_requests]
    return t.ravel()[order], cid[order]
