"""Shared test helpers: building matching oracle / GPU volumes from a seeded
workload, and the comparison tolerances.

Tolerances (FP32 GPU path vs FP64 oracle):
  * integer and index outputs (allocation, heuristics, hit indices, counts,
    FP32-path luminance): bit-exact;
  * irradiance texels: |a - b| <= 1e-3 * max(|b|, 1e-3 * mean|b|);
  * depth moments:     |a - b| <= 1e-4 * max(|b|, 1e-3 * mean|b|).
"""
import numpy as np

IRR_RTOL = 1e-3
DEP_RTOL = 1e-4


def oracle_volume(O, w, **over):
    vd = dict(w.volume)
    vd.update(over)
    v = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], vd["irr_interior"], vd["depth_interior"],
                       vd["rays_avg"], vd["rays_min"], vd["rays_max"], vd["hysteresis"], vd["depth_max"],
                       vd["tr_theta"], packed=int(vd.get("atlas_fp16", 0)) == 3, sampler=int(vd.get("sampler", 0)),
                       alpha=float(vd.get("alpha", 1.0)))
    v.set_scene(w.verts, w.idx, w.albedo)
    return v


def gpu_volume(adgi, w, stream=None, **over):
    vd = dict(w.volume)
    vd.update(over)
    v = adgi.Volume(stream=stream, **vd)
    v.set_scene(w.verts, w.idx, w.albedo)
    return v


def rel_check(a, b, rtol, what="", dump=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(float(np.abs(b).mean()), 1e-30) if b.size else 1e-30
    bound = rtol * np.maximum(np.abs(b), 1e-3 * scale)
    bad = np.abs(a - b) > bound
    if bad.any():
        if dump is not None:
            dump(np.flatnonzero(bad.reshape(bad.shape[0], -1).any(axis=1)))
        i = np.flatnonzero(bad.ravel())[:5]
        raise AssertionError("%s: %d of %d outside tolerance %g; first: gpu %s oracle %s" %
                             (what, int(bad.sum()), bad.size, rtol, a.ravel()[i], b.ravel()[i]))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3 * scale))) if a.size else 0.0
