"""The order-of-magnitude configuration on the GPU against the FP64 oracle.

64 x 32 x 64 = 131,072 probes at 4 m over the seeded city generator scaled
to about 2M triangles (a moving tunnel gate, 3 moving point lights and the
sun), 64 rays per probe on average (min 4, which the pilots raise to 8; max
512): 8,388,608 rays per update.  Four updates run in lockstep on the GPU
(FP32 atlases, and half atlases with FP32 blending) and in the oracle, which
computes every probe, so nothing here is extrapolated:

* FP32: every integer output is bit-exact on every frame (W, n, offsets,
  q_v, q_r, triggers, every pilot and main hit index and t); ray radiance
  and the atlases stay within 1e-3 (irradiance) and 1e-4 (depth moments),
  and a 65,536-point query within 1e-3.
* Half atlases: allocation and hits stay bit-exact (the atlases feed
  neither); the atlas and query errors against the oracle are written to
  scaled_errors.json in the diagnostics folder and bounded as stated below.

The FP32 ray records are also checked on a 1 % probe sample (every 100th
probe) with their own error statistics, the sample the configuration names.
"""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S

from _helpers import DEP_RTOL, IRR_RTOL, diag_path, gpu_volume, oracle_volume, rel_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FRAMES = 4


@pytest.fixture(scope="module")
def adgi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05125_gb300 import adgi as A
    from paper_2301_05125_gb300 import build

    build.build()
    A.load()
    return A


def _err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(float(np.abs(b).mean()), 1e-30)
    r = np.abs(a - b) / np.maximum(np.abs(b), 1e-3 * scale)
    return {"max": float(r.max()), "mean": float(r.mean()), "p99": float(np.percentile(r, 99))}


def test_scaled_config_against_oracle(adgi):
    w = S.scaled(1)
    assert w.n_probes == 131072 and w.n_tris > 1_900_000
    gv = gpu_volume(adgi, w)
    gh = gpu_volume(adgi, w, atlas_fp16=1)
    ov = oracle_volume(O, w)
    sample = np.arange(0, w.n_probes, 100)  # the 1 % probe sample
    out = {"probes": w.n_probes, "triangles": int(w.n_tris), "rays_per_update": int(w.rays_per_update),
           "frames": FRAMES, "sample_probes": int(len(sample))}
    wsum = 0
    for f in range(FRAMES):
        if w.dyn_at is not None and w.dyn_count:
            dv = w.dyn_at(f)
            for v in (gv, gh, ov):
                v.move_vertices(w.dyn_first, dv)
        for v in (gv, gh, ov):
            v.update(f, w.seed, w.lights_at(f), w.sky)
        tag = "scaled frame %d" % f
        gv.stats()
        gh.stats()
        W = ov.W()
        wsum += int(W.astype(np.int64).sum())
        for g in (gv, gh):
            np.testing.assert_array_equal(g.W(), W, err_msg=tag + " W")
            np.testing.assert_array_equal(g.n(), ov.n(), err_msg=tag + " n")
            np.testing.assert_array_equal(g.off(), ov.off(), err_msg=tag + " off")
        for name in ("qv", "qr", "trv", "trr"):
            np.testing.assert_array_equal(getattr(gv, name)(), getattr(ov, name)(), err_msg=tag + " " + name)
        ph = gv.pilot_hit()
        np.testing.assert_array_equal(adgi.hit_tri(ph), ov.pilot_tri(), err_msg=tag + " pilot tri")
        m = ov.pilot_tri() >= 0
        np.testing.assert_array_equal(adgi.hit_t(ph)[m], ov.pilot_t()[m], err_msg=tag + " pilot t")
        np.testing.assert_array_equal(gv.pilot_lum(), ov.pilot_lum().astype(np.float32), err_msg=tag + " pilot lum")
        R = int(ov.off()[-1])
        mh = gv.main_hit()[:R]
        otri = ov.main_tri()
        np.testing.assert_array_equal(adgi.hit_tri(mh), otri, err_msg=tag + " main tri")
        m = otri >= 0
        np.testing.assert_array_equal(adgi.hit_t(mh)[m], ov.main_t()[m], err_msg=tag + " main t")
        np.testing.assert_array_equal(adgi.hit_tri(gh.main_hit()[:R]), otri, err_msg=tag + " main tri (half)")
        rec = gv.main_rec()[:R]
        rel_check(rec[:, :3], ov.main_rad(), IRR_RTOL, tag + " main radiance")
        rel_check(rec[:, 3], ov.main_dep(), DEP_RTOL, tag + " main depth")
        # the 1 % probe sample: its rays' radiance and depth statistics
        off = ov.off().astype(np.int64)
        rows = np.concatenate([np.arange(off[p], off[p + 1]) for p in sample])
        out["frame%d_sample_rays" % f] = int(len(rows))
        out["frame%d_sample_radiance" % f] = _err(rec[rows, :3], ov.main_rad()[rows])
        out["frame%d_sample_depth" % f] = _err(rec[rows, 3], ov.main_dep()[rows])
    assert wsum > 0  # the change measure drove a non-uniform allocation
    # FP32 atlases and queries
    oi, od = ov.irr(), ov.dep()
    gi = gv.irr()
    np.testing.assert_array_equal(gi[..., 3].astype(np.int64), ov.irr_n().astype(np.int64), err_msg="irr counts")
    np.testing.assert_array_equal(gv.dep_n(), ov.dep_n(), err_msg="depth counts")
    out["fp32_irradiance_atlas"] = _err(gi[..., :3], oi)
    out["fp32_depth_moments"] = _err(gv.dep_moments(), od)
    rel_check(gi[..., :3], oi, IRR_RTOL, "scaled irradiance atlas")
    rel_check(gv.dep_moments(), od, DEP_RTOL, "scaled depth atlas")
    rng = np.random.default_rng(31)
    lo = np.array(w.volume["origin"], np.float32)
    ext = np.array(w.volume["spacing"], np.float32) * (np.array(w.volume["dims"]) - 1)
    pos = (lo + rng.random((65536, 3)) * ext).astype(np.float32)
    nrm = rng.normal(size=(65536, 3)).astype(np.float32)
    oq = ov.query(pos, nrm)
    out["fp32_query"] = _err(gv.query(pos, nrm), oq)
    # half atlases: errors stated per atlas and per query
    hi = gh.irr()
    np.testing.assert_array_equal(hi[..., 3].astype(np.int64), ov.irr_n().astype(np.int64), err_msg="half irr counts")
    out["fp16_irradiance_atlas"] = _err(hi[..., :3], oi)
    out["fp16_depth_moments"] = _err(gh.dep_moments(), od)
    out["fp16_query"] = _err(gh.query(pos, nrm), oq)
    json.dump(out, open(diag_path("scaled_errors.json"), "w"), indent=1)
    rel_check(gv.query(pos, nrm), oq, IRR_RTOL, "scaled query")
    # half storage has 11 significant bits (2^-11 ~ 4.9e-4 relative rounding)
    assert out["fp16_irradiance_atlas"]["mean"] < 1e-3 and out["fp16_depth_moments"]["mean"] < 1e-3, out
    assert out["fp16_query"]["mean"] < 1e-3 and out["fp16_query"]["p99"] < 5e-3, out
    for v in (gv, gh, ov):
        v.close()
