"""Oracle backend of the probe-slab split driver (paper_2301_05125_gb300.slab),
for the CPU tests: each rank is an oracle volume restricted to its probes
(orc_slab_*), and its slices travel as torch CPU tensors (gloo) or are
copied directly (one process)."""
import numpy as np
import torch

from oracle import oracle as O


class OracleSlabRank:
    HALO = ("TRV", "TRR")
    ATLAS = ("IRR", "IRR_N", "DEP", "DEP_N")

    def __init__(self, w, threads=2):
        vd = w.volume
        self.w = w
        self.ov = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], vd["irr_interior"], vd["depth_interior"],
                                 vd["rays_avg"], vd["rays_min"], vd["rays_max"], vd["hysteresis"], vd["depth_max"],
                                 vd["tr_theta"], threads=threads)
        self.ov.set_scene(w.verts, w.idx, w.albedo)

    def step(self, k, f, p0, p1):
        w = self.w
        if k == 0 and w.dyn_at is not None and w.dyn_count:
            self.ov.move_vertices(w.dyn_first, w.dyn_at(f))
        fn = (self.ov.slab_begin, self.ov.slab_weights, self.ov.slab_finish)[k]
        fn(f, w.seed, w.lights_at(f), p0, p1, w.sky)

    # slices travel as raw bytes (gloo has no unsigned 16- or 32-bit types)
    def empty(self, which, p0, p1):
        _, dt, per = self.ov._slab_elems(which)
        return torch.zeros((p1 - p0) * per * np.dtype(dt).itemsize, dtype=torch.uint8)

    def get(self, which, p0, p1):
        return torch.from_numpy(self.ov.slab_get(which, p0, p1).view(np.uint8))

    def put(self, which, p0, p1, buf):
        _, dt, _ = self.ov._slab_elems(which)
        self.ov.slab_set(which, p0, p1, np.ascontiguousarray(buf.numpy()).view(dt))


def single_run(w, frames, threads=2):
    """The unsplit oracle over the same frames: per-frame W, n, off and hits,
    then the final atlases"""
    vd = w.volume
    ov = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], vd["irr_interior"], vd["depth_interior"],
                        vd["rays_avg"], vd["rays_min"], vd["rays_max"], vd["hysteresis"], vd["depth_max"],
                        vd["tr_theta"], threads=threads)
    ov.set_scene(w.verts, w.idx, w.albedo)
    per = []
    for f in range(frames):
        if w.dyn_at is not None and w.dyn_count:
            ov.move_vertices(w.dyn_first, w.dyn_at(f))
        ov.update(f, w.seed, w.lights_at(f), w.sky)
        per.append(dict(W=ov.W(), n=ov.n(), off=ov.off(), pilot_tri=ov.pilot_tri(), pilot_t=ov.pilot_t(),
                        main_tri=ov.main_tri(), main_t=ov.main_t()))
    final = dict(irr=ov.irr(), irr_n=ov.irr_n(), dep=ov.dep(), dep_n=ov.dep_n())
    ov.close()
    return per, final


def rank_record(rank, rng):
    """what a rank holds for its probes after a frame"""
    ov = rank.ov
    p0, p1 = rng
    off = ov.off()
    r0, r1 = int(off[p0]), int(off[p1])
    return dict(W=ov.W()[p0:p1], n=ov.n(), off=off, pilot_tri=ov.pilot_tri()[p0:p1], pilot_t=ov.pilot_t()[p0:p1],
                main_tri=ov.main_tri()[r0:r1], main_t=ov.main_t()[r0:r1])
