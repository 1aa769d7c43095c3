"""Shared test helpers: building matching oracle / GPU volumes from a seeded
workload, and the comparison tolerances.

Tolerances (FP32 GPU path vs FP64 oracle):
  * integer and index outputs (allocation, heuristics, hit indices, counts,
    FP32-path luminance): bit-exact;
  * irradiance texels: |a - b| <= 1e-3 * max(|b|, 1e-3 * mean|b|);
  * depth moments:     |a - b| <= 1e-4 * max(|b|, 1e-3 * mean|b|).
"""
import os
import tempfile

import numpy as np

from oracle import oracle as O

IRR_RTOL = 1e-3
DEP_RTOL = 1e-4


def diag_path(name):
    """where a test writes a diagnostic file (measured errors, failing
    rays): the folder named by ADGI_DIAG_DIR, else a temporary folder"""
    d = os.environ.get("ADGI_DIAG_DIR") or os.path.join(tempfile.gettempdir(), "adgi_diag")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, name)


def oracle_volume(O, w, **over):
    vd = dict(w.volume)
    vd.update(over)
    v = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], vd["irr_interior"], vd["depth_interior"],
                       vd["rays_avg"], vd["rays_min"], vd["rays_max"], vd["hysteresis"], vd["depth_max"],
                       vd["tr_theta"], packed=int(vd.get("atlas_fp16", 0)) == 3, sampler=int(vd.get("sampler", 0)),
                       alpha=float(vd.get("alpha", 1.0)), dyn_ratio=int(vd.get("dyn_ratio", 0)),
                       hyst_dyn=float(vd.get("hysteresis_dyn", 0.91)), blend_mode=int(vd.get("blend_mode", 0)),
                       cheb_var_floor_rel=float(vd.get("cheb_var_floor_rel", 0.0)))
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


def dir_cell(d):
    """Morton index of each direction's cell in a 16 x 16 grid over the
    octahedral square (the order of the samples inside a probe), FP32 steps"""
    d = np.asarray(d, np.float32)
    ax = np.abs(d)
    l1 = (ax[:, 0] + ax[:, 1]) + ax[:, 2]
    px, py = d[:, 0] / l1, d[:, 1] / l1
    sx = np.where(px >= 0, np.float32(1), np.float32(-1))
    sy = np.where(py >= 0, np.float32(1), np.float32(-1))
    neg = d[:, 2] < 0
    qx = (np.float32(1) - np.abs(py)) * sx
    qy = (np.float32(1) - np.abs(px)) * sy
    px, py = np.where(neg, qx, px), np.where(neg, qy, py)
    f16 = np.float32(16)
    cx = np.clip(np.floor(((px + np.float32(1)) * np.float32(0.5)) * f16), 0, 15).astype(np.int64)
    cy = np.clip(np.floor(((py + np.float32(1)) * np.float32(0.5)) * f16), 0, 15).astype(np.int64)
    for k in range(0, len(d), max(1, len(d) // 200)):  # the oracle's texel binning, 16 x 16 interior
        assert O.texel_of_dir(d[k], 16) == (cy[k] + 1) * 18 + cx[k] + 1
    m = np.zeros(len(d), np.int64)
    for b in range(4):
        m |= ((cx >> b) & 1) << (2 * b) | ((cy >> b) & 1) << (2 * b + 1)
    return m


def mh_compare(A, gv, ov, tag, check_atlas=True, rad_rtol=IRR_RTOL):
    """Metropolis volumes: chain states, samples, grouping and hits bit-exact
    against the oracle; +w radiance and atlases within tolerance."""
    gv.stats()  # raises if a device-side anomaly flag was set
    np.testing.assert_array_equal(gv.W(), ov.W(), err_msg=tag + " W")
    np.testing.assert_array_equal(gv.qv(), ov.qv(), err_msg=tag + " qv")
    B = ov.mh_samples
    g, u = gv.mh_chains()
    og, ou = ov.mh_chain_state()
    np.testing.assert_array_equal(g.view(np.uint32), og.view(np.uint32), err_msg=tag + " chain positions")
    np.testing.assert_array_equal(u.view(np.uint32), ou.view(np.uint32), err_msg=tag + " chain directions")
    probe, d = gv.mh_samples()
    np.testing.assert_array_equal(probe, ov.mh_probe(), err_msg=tag + " sample probes")
    np.testing.assert_array_equal(d.view(np.uint32), ov.mh_dir().view(np.uint32), err_msg=tag + " sample directions")
    order = np.argsort(ov.mh_probe().astype(np.int64) * 256 + dir_cell(ov.mh_dir()), kind="stable")
    np.testing.assert_array_equal(gv.mh_order(), order, err_msg=tag + " grouping")
    counts = np.bincount(ov.mh_probe(), minlength=gv.P)
    np.testing.assert_array_equal(gv.mh_off(), np.concatenate([[0], np.cumsum(counts)]), err_msg=tag + " offsets")
    hp, hn = gv.main_hit()[:B], gv.mh_hit_neg()
    np.testing.assert_array_equal(A.hit_tri(hp), ov.mh_tri()[order], err_msg=tag + " +w tri")
    np.testing.assert_array_equal(A.hit_tri(hn), ov.mh_tri_neg()[order], err_msg=tag + " -w tri")
    m = ov.mh_tri()[order] >= 0
    np.testing.assert_array_equal(A.hit_t(hp)[m], ov.mh_t()[order][m], err_msg=tag + " +w t")
    m = ov.mh_tri_neg()[order] >= 0
    np.testing.assert_array_equal(A.hit_t(hn)[m], ov.mh_t_neg()[order][m], err_msg=tag + " -w t")
    if B:
        rel_check(gv.main_rec()[:B, :3], ov.mh_rad()[order], rad_rtol, tag + " +w radiance")
    if check_atlas:
        gi = gv.irr()
        np.testing.assert_array_equal(gi[..., 3].astype(np.int64), ov.irr_n().astype(np.int64),
                                      err_msg=tag + " irr counts")
        np.testing.assert_array_equal(gv.dep_n(), ov.dep_n(), err_msg=tag + " depth counts")
        rel_check(gi[..., :3], ov.irr(), IRR_RTOL, tag + " irradiance atlas")
        rel_check(gv.dep_moments(), ov.dep(), DEP_RTOL, tag + " depth atlas")
