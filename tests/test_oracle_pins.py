"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
test vectors, closed forms, invariants, special cases that reduce to a
textbook result, or brute force on tiny inputs.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_05125_gb300 import scenegen as S


# --------------------------------------------------------------- generators
def test_splitmix64_published_vectors():
    # SplitMix64 seeded with 0: first two outputs (Steele, Lea, Flood 2014;
    # reference outputs of Vigna's splitmix64.c).
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_pilot_dirs_one_per_octant_and_pairs_repeat():
    # Sec. 4.4: stratified random, one ray per octant; AABBCC pattern.
    for probe in range(50):
        for f in (0, 2, 7):
            for o in range(8):
                d = O.pilot_dir(3, f, probe, o)
                assert abs(float(np.linalg.norm(d.astype(np.float64))) - 1.0) < 3e-7
                sx = np.signbit(d[0]) if d[0] == 0 else d[0] < 0
                sy = np.signbit(d[1]) if d[1] == 0 else d[1] < 0
                sz = np.signbit(d[2]) if d[2] == 0 else d[2] < 0
                assert int(sx) | (int(sy) << 1) | (int(sz) << 2) == o
                np.testing.assert_array_equal(d, O.pilot_dir(3, f ^ 1, probe, o))
    assert not np.array_equal(O.pilot_dir(3, 0, 5, 1), O.pilot_dir(3, 2, 5, 1))


def test_pilot_dirs_uniform_within_octant():
    # Uniform on the octant's spherical triangle in barycentric (u1,u2,u3)
    # parametrisation before normalisation: the simplex mean is (1/3,1/3,1/3).
    vs = np.array([O.pilot_dir(11, 0, p, 0) for p in range(4000)], np.float64)
    l1 = vs / vs.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(l1.mean(axis=0), [1 / 3] * 3, atol=0.015)


def test_frame_rotation_is_a_rotation():
    zs = []
    for f in range(200):
        R = O.frame_rotation(7, f).astype(np.float64)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=2e-7)
        assert abs(np.linalg.det(R) - 1.0) < 5e-7
        zs.append(R[:, 2])
    # a uniform random rotation maps e_z to a uniform direction: mean ~ 0
    assert np.linalg.norm(np.mean(zs, axis=0)) < 0.15
    assert not np.array_equal(O.frame_rotation(7, 0), O.frame_rotation(7, 1))


def test_sf_points_closed_form():
    # Spherical Fibonacci (Keinert et al. 2015): z_i = 1-(2i+1)/m,
    # phi_i = i * pi * (3 - sqrt 5), compared with libm cos/sin.
    for m in (1, 2, 7, 64, 1016):
        pts = O.sf_points(m).astype(np.float64)
        i = np.arange(m)
        z = 1.0 - (2 * i + 1) / m
        phi = i * math.pi * (3.0 - math.sqrt(5.0))
        r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        ref = np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
        np.testing.assert_allclose(pts, ref, atol=2e-7)
        np.testing.assert_allclose(np.linalg.norm(pts, axis=1), 1.0, atol=3e-7)


# --------------------------------------------------------------- octahedral
def test_oct_round_trip_and_special_directions():
    rng = np.random.default_rng(0)
    w = rng.normal(size=(2000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    for x in w:
        np.testing.assert_allclose(O.oct_decode(O.oct_encode(x)), x, atol=1e-14)
    np.testing.assert_allclose(O.oct_encode([0, 0, 1]), [0, 0], atol=0)
    np.testing.assert_allclose(O.oct_encode([1, 0, 0]), [1, 0], atol=0)
    np.testing.assert_allclose(O.oct_encode([0, -1, 0]), [0, -1], atol=0)
    p = O.oct_encode([0, 0, -1])
    assert abs(p[0]) == 1 and abs(p[1]) == 1
    # the upper hemisphere maps inside the diamond |x|+|y| <= 1
    for x in w[:200]:
        p = O.oct_encode(x)
        assert (abs(p[0]) + abs(p[1]) <= 1 + 1e-12) == (x[2] >= 0) or abs(x[2]) < 1e-12


def test_texel_centres_bin_to_themselves():
    for n in (6, 14):
        T = n + 2
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                p = [((j - 1) + 0.5) / n * 2 - 1, ((i - 1) + 0.5) / n * 2 - 1]
                w = O.oct_decode(p)
                assert O.texel_of_dir(w.astype(np.float32), n) == i * T + j


def _fold_partner(i, j, n):
    """Interior texel whose centre is the mirror image of border texel (i,j)
    across the nearest square edge, using the octahedral map's edge identity
    (x, +-1 +- e) ~ (-x, +-1 -+ e) and (+-1 +- e, y) ~ (+-1 -+ e, -y)."""
    # padded coordinates of the centre in units of one texel, edges at 1, n+1
    cy, cx = i + 0.5, j + 0.5
    if cy < 1:
        cy, cx = 2 - cy, (n + 2) - cx
    elif cy > n + 1:
        cy, cx = 2 * (n + 1) - cy, (n + 2) - cx
    if cx < 1:
        cx, cy = 2 - cx, (n + 2) - cy
    elif cx > n + 1:
        cx, cy = 2 * (n + 1) - cx, (n + 2) - cy
    return int(math.floor(cy)), int(math.floor(cx))


def test_octahedral_edge_identity_and_border_copy():
    # the identity used by _fold_partner: the square's edges fold onto
    # themselves mirrored, and all four corners are the direction -z
    rng = np.random.default_rng(1)
    for a in rng.uniform(-1, 1, 200):
        for e in (1.0, -1.0):
            np.testing.assert_allclose(O.oct_decode([a, e]), O.oct_decode([-a, e]), atol=1e-15)
            np.testing.assert_allclose(O.oct_decode([e, a]), O.oct_decode([e, -a]), atol=1e-15)
    for cx in (-1, 1):
        for cy in (-1, 1):
            np.testing.assert_allclose(O.oct_decode([cx, cy]), [0, 0, -1], atol=1e-15)
    for n in (6, 14):
        T = n + 2
        tile = rng.normal(size=(T, T, 2))
        cnt = rng.integers(0, 255, (T, T)).astype(np.uint8)
        t2, c2 = O.border_copy(tile, cnt, n)
        np.testing.assert_array_equal(t2[1:-1, 1:-1], tile[1:-1, 1:-1])
        for i in range(T):
            for j in range(T):
                if 1 <= i <= n and 1 <= j <= n:
                    continue
                si, sj = _fold_partner(i, j, n)
                assert 1 <= si <= n and 1 <= sj <= n
                np.testing.assert_array_equal(t2[i, j], tile[si, sj])
                assert c2[i, j] == cnt[si, sj]


# --------------------------------------------------------------- intersection
def test_intersection_closed_form_and_facing():
    # triangle in z = 0 with normal +z; a ray straight down hits at t = 1
    hit, t, det = O.intersect_tri([0.25, 0.25, 1.0], [0, 0, -1], [0, 0, 0], [1, 0, 0], [0, 1, 0])
    assert hit and t == 1.0 and det > 0  # front face: det > 0
    hit, t, det = O.intersect_tri([0.25, 0.25, -2.0], [0, 0, 1], [0, 0, 0], [1, 0, 0], [0, 1, 0])
    assert hit and t == 2.0 and det < 0  # back face: det < 0
    hit, _, _ = O.intersect_tri([2.0, 2.0, 1.0], [0, 0, -1], [0, 0, 0], [1, 0, 0], [0, 1, 0])
    assert not hit


def test_intersection_against_fp64_barycentrics():
    rng = np.random.default_rng(2)
    n_mis = 0
    for _ in range(20000):
        A, B, Cv = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
        o = rng.uniform(-3, 3, 3).astype(np.float32)
        target = (rng.dirichlet([1, 1, 1]) * 1.4 - 0.2) @ np.stack([A, B, Cv]).astype(np.float64)
        d = (target - o).astype(np.float32)
        hit, t, det = O.intersect_tri(o, d, A, B, Cv)
        # FP64 reference: Moller-Trumbore style barycentrics in double
        A64, B64, C64, o64, d64 = (x.astype(np.float64) for x in (A, B, Cv, o, d))
        e1, e2 = B64 - A64, C64 - A64
        n = np.cross(e1, e2)
        denom = -np.dot(d64, n)
        if abs(denom) < 1e-12:
            continue
        s = o64 - A64
        t64 = np.dot(s, n) / denom
        u = np.dot(d64, np.cross(s, e2)) / np.dot(d64, np.cross(e2, e1)) if False else None
        # barycentrics of the line/plane point
        x = o64 + t64 * d64
        M = np.stack([e1, e2], 1)
        uv, *_ = np.linalg.lstsq(M, x - A64, rcond=None)
        b = np.array([1 - uv.sum(), uv[0], uv[1]])
        inside = b.min() >= 0
        if abs(b.min()) < 1e-5:
            continue  # on an edge: either answer is correct
        if hit != inside:
            n_mis += 1
            continue
        if hit:
            assert abs(t - t64) <= 1e-4 * max(1.0, abs(t64))
            # det sign: front face <=> geometric normal faces the ray origin
            assert (det > 0) == (np.dot(n, d64) < 0)
    assert n_mis == 0


def test_watertight_closed_mesh_never_misses():
    # rays from inside a closed box shell must hit it (no leaks on edges)
    v, t = S.boxes_mesh([[0, 0, 0]], [[8, 8, 8]], inward=True)
    rng = np.random.default_rng(3)
    O_ = np.repeat(np.array([[4.0, 4.0, 4.0]], np.float32), 20000, 0)
    # aim exactly at edges and corners of the shell
    tgt = rng.integers(0, 2, (20000, 3)).astype(np.float32) * 8.0
    k = rng.integers(0, 3, 20000)
    tgt[np.arange(20000), k] = rng.uniform(0, 8, 20000)
    D = (tgt - O_).astype(np.float32)
    tt, tri, det = O.trace_closest(v, t, O_, D, 1e-4, np.inf, use_bvh=False)
    assert (tri >= 0).all()
    assert (det > 0).all()  # the shell faces inward: all front-face hits


def _random_rays(n, lo, hi, rng):
    O_ = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    D = rng.normal(size=(n, 3)).astype(np.float32)
    return O_, D


@pytest.mark.parametrize("scene", ["room", "city"])
def test_bvh_equals_brute_force(scene):
    rng = np.random.default_rng(4)
    if scene == "room":
        w = S.box_room(1)
        O_, D = _random_rays(20000, 0.2, 7.8, rng)
    else:
        w = S.small_city(2, n_boxes=200)
        O_, D = _random_rays(3000, -30, 30, rng)
        O_[:, 1] = np.abs(O_[:, 1])
    t1, i1, d1 = O.trace_closest(w.verts, w.idx, O_, D, 1e-4, np.inf, use_bvh=False)
    t2, i2, d2 = O.trace_closest(w.verts, w.idx, O_, D, 1e-4, np.inf, use_bvh=True)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(t1, t2)
    a1 = O.trace_any(w.verts, w.idx, O_, D, 0.0, 0.7, use_bvh=False)
    a2 = O.trace_any(w.verts, w.idx, O_, D, 0.0, 0.7, use_bvh=True)
    np.testing.assert_array_equal(a1, a2)


def test_nearest_hit_ties_take_smaller_index():
    # two identical triangles: the hit must report the smaller index
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    idx = np.array([[0, 1, 2], [0, 1, 2], [0, 1, 2]], np.int32)
    O_ = np.array([[0.2, 0.2, 1.0]] * 3, np.float32)
    D = np.array([[0, 0, -1]] * 3, np.float32)
    for bvh in (False, True):
        t, tri, _ = O.trace_closest(v, idx, O_, D, 1e-4, np.inf, use_bvh=bvh)
        assert (tri == 0).all() and (t == 1.0).all()


# --------------------------------------------------------------- allocation
def _alloc_checks(W, avg, rmin, rmax):
    n, off = O.allocate(W, avg, rmin, rmax)
    P = len(W)
    m0 = max(rmin, 8)
    assert int(n.astype(np.int64).sum()) == avg * P
    assert (n >= m0).all() and (n <= rmax).all()
    np.testing.assert_array_equal(off[1:] - off[:-1], n - 8)
    assert off[0] == 0
    return n


def test_allocation_closed_forms():
    # uniform when nothing changes: E = P*(avg-m0) spread evenly, remainder to
    # the lowest indices
    n = _alloc_checks(np.zeros(5, np.uint32), 11, 8, 40)
    np.testing.assert_array_equal(n, [11, 11, 11, 11, 11])
    n = _alloc_checks(np.zeros(4, np.uint32), 9, 6, 40)  # m0 = 8, E = 4
    np.testing.assert_array_equal(n, [9, 9, 9, 9])
    n = _alloc_checks(np.zeros(3, np.uint32), 10, 8, 40)
    np.testing.assert_array_equal(n, [10, 10, 10])
    # proportional: W = (1, 3), E = 8 -> extras (2, 6)
    n = _alloc_checks(np.array([1, 3], np.uint32), 12, 8, 100)
    np.testing.assert_array_equal(n, [10, 14])
    # cap: probe 1 capped at max, the rest of the extra goes to probe 0
    n = _alloc_checks(np.array([1, 1000], np.uint32), 16, 8, 18)  # E = 16, cap 10
    np.testing.assert_array_equal(n, [14, 18])
    # only one probe changes: it takes min(cap, E), the remainder is spread
    # one by one over the others in index order
    n = _alloc_checks(np.array([0, 5, 0, 0], np.uint32), 14, 8, 20)  # E = 24, cap 12
    np.testing.assert_array_equal(n, [12, 20, 12, 12])
    # equal weights behave like the uniform case
    n = _alloc_checks(np.full(3, 7, np.uint32), 10, 8, 40)
    np.testing.assert_array_equal(n, [10, 10, 10])
    n = _alloc_checks(np.full(3, 7, np.uint32), 9, 8, 40)  # E = 3 -> one each
    np.testing.assert_array_equal(n, [9, 9, 9])
    with pytest.raises(ValueError):
        O.allocate(np.zeros(3, np.uint32), 7, 8, 40)  # avg below the pilot floor


def test_allocation_invariants_random():
    rng = np.random.default_rng(5)
    for trial in range(300):
        P = int(rng.integers(1, 300))
        rmin = int(rng.integers(4, 20))
        rmax = int(rng.integers(max(rmin, 8), 300))
        avg = int(rng.integers(max(rmin, 8), rmax + 1))
        kind = trial % 4
        if kind == 0:
            W = rng.integers(0, 1 << 24, P)
        elif kind == 1:
            W = rng.integers(0, 4, P)  # heavy ties and zeros
        elif kind == 2:
            W = np.where(rng.random(P) < 0.05, rng.integers(1, 1 << 24, P), 0)  # sparse, caps bite
        else:
            W = rng.integers(0, 2, P) * 1000
        W = W.astype(np.uint32)
        n = _alloc_checks(W, avg, rmin, rmax)
        m0 = max(rmin, 8)
        # scaling all weights by a constant does not change the allocation
        if W.max() < (1 << 20):
            n2, _ = O.allocate(W * 7, avg, rmin, rmax)
            np.testing.assert_array_equal(n, n2)
        # monotone up to the one-ray remainder
        order = np.argsort(W, kind="stable")
        Ws, ns = W[order], n[order].astype(np.int64)
        for a in range(len(Ws) - 1):
            if Ws[a + 1] > Ws[a]:
                assert ns[a + 1] >= ns[a] - 1
        # proportionality when nothing is capped
        if W.sum() > 0 and n.max() < rmax:
            E = (avg - m0) * P
            share = E * W.astype(np.float64) / W.sum()
            assert np.all(np.abs((n - m0) - share) < 2.0 + 1e-9)


def _waterfill_exact(W, E, cap):
    """The continuous water-filling of E extra rays: x_p = min(cap, lam W_p)
    with sum x = E, found by brute force over every candidate capped set of
    the probes with W_p > 0 (exact rational arithmetic).  Returns x, or None
    when every weighted probe is capped (the rest then goes to W = 0 probes)."""
    P = len(W)
    pos = [p for p in range(P) if W[p] > 0]
    found = None
    for r in range(len(pos) + 1):
        for C in itertools.combinations(pos, r):
            Er = E - cap * len(C)
            U = [p for p in pos if p not in C]
            SU = sum(int(W[p]) for p in U)
            if Er < 0 or SU == 0:
                continue
            lam = Fraction(Er, SU)
            if all(lam * int(W[p]) >= cap for p in C) and all(lam * int(W[p]) <= cap for p in U):
                x = [Fraction(cap) if p in C else lam * int(W[p]) for p in range(P)]
                assert found is None or found == x  # the water level is unique
                found = x
    return found


def test_allocation_brute_force_waterfill():
    # P <= 8: the integer allocation against the exact continuous
    # water-filling share x_p of the extra rays (the fixed budget spread in
    # proportion to W_p, capped at rays_max; Sec. 3.4 fixes the budget).  The
    # proportional passes hand out floors of the shares, and the residual
    # (fewer rays than probes after the first pass) goes one ray at a time in
    # index order, so no probe may drift by 3 or more rays from x_p; probes
    # with W = 0 take nothing while a weighted probe is below its cap.
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(3000):
        P = int(rng.integers(1, 9))
        rmax = int(rng.integers(8, 40))
        avg = int(rng.integers(8, rmax + 1))
        kind = trial % 4
        if kind == 0:
            W = rng.integers(0, 50, P)
        elif kind == 1:
            W = rng.integers(0, 3, P)
        elif kind == 2:
            W = np.where(rng.random(P) < 0.3, rng.integers(1, 1 << 24, P), 0)
        else:
            W = rng.integers(0, 1 << 32, P, dtype=np.uint64)
        W = W.astype(np.uint32)
        n = _alloc_checks(W, avg, 8, rmax)
        extra = n.astype(np.int64) - 8
        E, cap = (avg - 8) * P, rmax - 8
        x = _waterfill_exact(W, E, cap)
        if x is None:
            continue
        checked += 1
        dev = [abs(Fraction(int(extra[p])) - x[p]) for p in range(P)]
        assert max(dev) < 3, (W, avg, rmax, extra, [float(v) for v in x])
        if any(W[p] > 0 and extra[p] < cap for p in range(P)):
            assert all(extra[p] == 0 for p in range(P) if W[p] == 0), (W, extra)
    assert checked > 2000


# --------------------------------------------------------------- heuristics
def test_luts_closed_forms_and_no_boundary_ambiguity():
    s = math.sqrt(12.0)
    lv, lc = O.luts(s)
    assert lv[0] == 1019  # floor(1023 e^{-1/256})
    assert lv[256] == 137  # f_v at t = s: floor(1023 e^{-2 * 256.5/256}) = floor(137.9)
    assert (np.diff(lv.astype(int)) <= 0).all() and (np.diff(lc.astype(int)) <= 0).all()
    # every LUT value is far from an integer boundary, so any faithful exp()
    # gives the same table
    i = np.arange(4096)
    xv = 1023.0 * np.exp(-2.0 * (i + 0.5) / 256.0)
    xc = 1023.0 * np.exp(-(i + 0.5) * s / 64.0)
    for x, lut in ((xv, lv), (xc, lc)):
        frac = x - np.floor(x)
        big = x >= 1.0
        assert np.min(np.minimum(frac, 1 - frac)[big]) > 1e-9
        np.testing.assert_array_equal(np.floor(x).astype(int), lut.astype(int))


def _tiny_vol(**kw):
    args = dict(origin=(0, 0, 0), spacing=(1, 1, 1), dims=(6, 5, 7), rays_avg=16, rays_min=8, rays_max=64,
                theta=16)
    args.update(kw)
    return O.OracleVolume(**args)


def test_trigger_impulse_closed_form():
    # One probe/octant changes between the two frames of a pair: the trigger
    # jumps to the delta (Fig. TrCam(a)) and then decays linearly over theta
    # frames; the 5x5x5 x octant convolution spreads it to exactly the
    # clipped box and the octant's three edge neighbours (Sec. 4.1).
    v = _tiny_vol()
    P = v.P
    X, Y, Z = 6, 5, 7
    t = np.full((P, 8), 0.5, np.float32)  # all pilot rays hit at t = 0.5
    tri = np.zeros((P, 8), np.int32)
    lum0 = np.full((P, 8), 1.0, np.float32)
    p0 = 2 + X * (1 + Y * 3)  # (2,1,3)
    o0 = 5
    lum1 = lum0.copy()
    lum1[p0, o0] = 3.0  # q_r: 204 -> 613, delta 409
    v.change_from_pilots(0, t, tri, lum0)
    assert (v.W() == 0).all()
    v.change_from_pilots(1, t, tri, lum1)
    delta = int(np.floor(3.0 * 1023 / 5)) - int(np.floor(1.0 * 1023 / 5))
    trr = v.trr()
    assert trr[p0, o0] == delta and trr.sum() == delta and v.trv().sum() == 0
    qv = v.qv()
    W = v.W()
    theta = 16
    for p in range(P):
        ix, iy, iz = p % X, (p // X) % Y, p // (X * Y)
        inbox = abs(ix - 2) <= 2 and abs(iy - 1) <= 2 and abs(iz - 3) <= 2
        exp = 0
        for o in range(8):
            f = delta if inbox and o in (o0, o0 ^ 1, o0 ^ 2, o0 ^ 4) else 0
            exp += (1023 * int(qv[p, o]) * 2 * f) >> 20
        assert W[p] == min(exp, (1 << 24) - 1)
    # linear decay: the pair after is unchanged (lum1 on both frames)
    for k in range(1, 20):
        v.change_from_pilots(1 + k, t, tri, lum1)
        assert v.trr()[p0, o0] == (delta * (theta - k)) // theta if k < theta else v.trr()[p0, o0] == 0


def test_static_scene_allocates_uniformly():
    w = S.box_room(1)
    vd = w.volume
    v = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], rays_avg=vd["rays_avg"], rays_min=8, rays_max=256)
    v.set_scene(w.verts, w.idx, w.albedo)
    light = w.lights_at(0)
    for f in range(6):
        v.update(f, 9, light)
        assert (v.W() == 0).all() and (v.trv() == 0).all() and (v.trr() == 0).all()
        assert (v.n() == 64).all()


def test_light_toggle_pulse_then_linear_decay():
    w = S.box_room(1)
    vd = w.volume
    v = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], rays_avg=64, rays_min=8, rays_max=256, theta=8)
    v.set_scene(w.verts, w.idx, w.albedo)
    on = w.lights_at(0)
    v.update(0, 9, [])  # light off on the first frame of the pair
    v.update(1, 9, on)  # switched on: pulse of |q_r(on) - q_r(off)| = q_r(on)
    qr_on = v.qr().astype(int)
    tr1 = v.trr().astype(int)
    np.testing.assert_array_equal(tr1, qr_on)
    assert v.W().sum() > 0
    for k in range(1, 10):
        v.update(1 + k, 9, on)
        np.testing.assert_array_equal(v.trr().astype(int), (qr_on * max(0, 8 - k)) // 8)


# --------------------------------------------------------------- shading / blend
def _sky_volume(avg=16, rmin=8, rmax=64, h=0.97, dims=(3, 3, 3)):
    v = O.OracleVolume((0, 0, 0), (1, 1, 1), dims, rays_avg=avg, rays_min=rmin, rays_max=rmax, hysteresis=h)
    v.set_scene(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.float32))
    return v


def test_constant_environment_blends_to_itself():
    # Texel estimate = texel-average of g (Sec. 3.6): a constant-radiance
    # environment gives exactly that radiance in every touched texel.
    v = _sky_volume()
    c = (0.7, 1.3, 2.9)
    for f in range(5):
        v.update(f, 1, [], sky=c)
        irr, n = v.irr(), v.irr_n()
        touched = n > 0
        assert touched.any()
        c32 = np.array(c, np.float32).astype(np.float64)  # the sky radiance is an FP32 input
        np.testing.assert_allclose(irr[touched], np.broadcast_to(c32, irr[touched].shape), rtol=1e-15)
        assert (irr[~touched] == 0).all()
        dep, dn = v.dep(), v.dep_n()
        dm = v.depth_max
        np.testing.assert_allclose(dep[dn > 0][:, 0], dm, rtol=1e-15)
        np.testing.assert_allclose(dep[dn > 0][:, 1], dm * dm, rtol=1e-14)


def _touches(v, frame, seed):
    """texel sample counts per probe for this frame, recomputed from the ray
    directions the oracle reports (pilot directions and rotated SF sets)."""
    P, Ti = v.P, v.Ti
    k = np.zeros((P, Ti * Ti), np.int64)
    n = v.n()
    pd = v.pilot_dir()
    for p in range(P):
        dirs = []
        if frame % 2 == 0:
            dirs += list(pd[p])
        m = int(n[p]) - 8
        dirs += [v.main_dir(m, i) for i in range(m)]
        for d in dirs:
            k[p, O.texel_of_dir(d, v.n_irr)] += 1
    return k.reshape(P, Ti, Ti)


def test_true_moving_average_then_hysteresis():
    # Alg. MovingAvgUpdate: a true running mean while n is small, then an EMA
    # with weight 1-h.  Closed forms: mean of all samples; step response
    # c1 + (c0 - c1) * prod(1 - w_f).
    h = 0.97
    v = _sky_volume(avg=24, rmax=64, h=h)
    skies = [0.5, 2.0, 1.0, 4.0]
    S_ = np.zeros((v.P, v.Ti, v.Ti))
    K = np.zeros((v.P, v.Ti, v.Ti))
    for f, c in enumerate(skies):
        v.update(f, 5, [], sky=(c, c, c))
        k = _touches(v, f, 5)
        S_ += k * c
        K += k
    irr = v.irr()[..., 0]
    inner = (slice(None), slice(1, -1), slice(1, -1))
    sel = K[inner] > 0
    # every texel here has n small enough for the true-mean regime (n/k < 32)
    np.testing.assert_allclose(irr[inner][sel], (S_[inner] / np.maximum(K[inner], 1))[sel], rtol=1e-13)
    # saturated regime: counts at 255, sky steps from 1.0 to 3.0
    v2 = _sky_volume(avg=8, rmin=8, rmax=8, h=h)
    Pn = v2.P
    v2.set_atlas(irr=np.ones((Pn, v2.Ti, v2.Ti, 3)), irr_n=np.full((Pn, v2.Ti, v2.Ti), 255, np.uint8))
    pred = np.ones((Pn, v2.Ti, v2.Ti))
    for f in range(8):
        v2.update(f, 3, [], sky=(3.0, 3.0, 3.0))
        k = _touches(v2, f, 3)
        h32 = float(np.float32(h))  # the hysteresis is an FP32 parameter
        w = np.where(k > 0, np.maximum(1 - h32, k / (255.0 + k)), 0.0)
        pred = 3.0 + (pred - 3.0) * (1.0 - w)
    got = v2.irr()[..., 0]
    np.testing.assert_allclose(got[inner], pred[inner], rtol=1e-12)


def test_sphere_depth_moments():
    # a probe at the centre of a triangulated sphere of radius r: every depth
    # sample is the distance to a facet, between the inscribed distance and r;
    # so the mean is r to ~1e-3 and the variance ~ 0.
    r = 3.0
    sv, st = S.uv_sphere((0, 0, 0), r, 64, 32, inward=True)
    # probe 0 sits exactly at the centre; the other probes of the 2x2x2 grid
    # are off-centre and not checked
    v = O.OracleVolume((0, 0, 0), (0.25, 0.25, 0.25), (2, 2, 2), rays_avg=200, rays_min=8, rays_max=400,
                       depth_max=10.0)
    v.set_scene(sv, st, np.full((len(st), 3), 0.5, np.float32))
    for f in range(3):
        v.update(f, 2, [])
    dep, dn = v.dep()[0], v.dep_n()[0]
    m = dn > 0
    assert m.sum() > 150
    mu, mu2 = dep[m][:, 0], dep[m][:, 1]
    lo = r * math.cos(math.pi / 64) * math.cos(math.pi / 32)
    assert (mu <= r * (1 + 1e-6)).all() and (mu >= lo * (1 - 1e-6)).all()
    assert abs(mu.mean() - r) < 2e-3 * r
    # every sample of a texel lies in [lo, r], so its variance is at most
    # (r - lo)^2 / 4 ~ 1e-5 r^2: the texel variance is ~0 at 1e-4 r^2
    assert (r - lo) ** 2 / 4 < 1e-4 * r * r
    assert np.max(np.abs(mu2 - mu * mu)) < 1e-4 * r * r


def test_direct_light_closed_form_and_shadow():
    # a large floor (albedo a) under a point light of intensity I: a probe
    # ray hitting x has radiance a/pi * I * cos / d^2 (Sec. 4.1 f_r uses the
    # direct light at the hit); an occluder between removes it.
    fv, ft = S.grid_plane(-50, 50, -50, 50, 0.0, 1, 1)
    a = np.array([0.5, 0.25, 0.75], np.float32)
    v = O.OracleVolume((-1, 1, -1), (2, 2, 2), (2, 2, 2), rays_avg=8, rays_min=8, rays_max=8, depth_max=1000.0)
    v.set_scene(fv, ft, np.tile(a, (len(ft), 1)))
    L = np.array([0.3, 10.0, -0.2])
    I = 100.0
    v.update(0, 4, [(0, L, (I, I, I))], sky=(0.2, 0.2, 0.2))
    tri = v.pilot_tri()
    t = v.pilot_t()
    dirs = v.pilot_dir()
    rad = v.pilot_rad()
    lum = v.pilot_lum()
    for p in range(v.P):
        o = v.probe_pos(p).astype(np.float64)
        for k in range(8):
            d = dirs[p, k].astype(np.float64)
            tp = -o[1] / d[1] if d[1] < 0 else np.inf
            xp = o + tp * d if np.isfinite(tp) else None
            if xp is None or max(abs(xp[0]), abs(xp[2])) > 49.9:
                assert tri[p, k] < 0  # leaves above the floor or beyond its edge
                np.testing.assert_allclose(rad[p, k], np.float32(0.2))
                continue
            assert tri[p, k] >= 0
            x = o + float(t[p, k]) * d
            assert abs(x[1]) < 1e-5
            Dl = L - x
            g = Dl[1] / np.linalg.norm(Dl) ** 3
            ref = a.astype(np.float64) / math.pi * I * g
            np.testing.assert_allclose(rad[p, k], ref, rtol=2e-6)
            lref = 0.2126 * ref[0] + 0.7152 * ref[1] + 0.0722 * ref[2]
            assert abs(lum[p, k] - lref) < 1e-5 * max(1.0, lref)
    # occluder: a big horizontal quad at y = 5 facing down blocks the light
    ov, ot = S.grid_plane(-50, 50, -50, 50, 5.0, 1, 1)
    allv = np.concatenate([fv, ov])
    allt = np.concatenate([ft, ot + len(fv)])
    # fresh volume: the atlas is empty, so the multi-bounce term is 0 too
    v = O.OracleVolume((-1, 1, -1), (2, 2, 2), (2, 2, 2), rays_avg=8, rays_min=8, rays_max=8, depth_max=1000.0)
    v.set_scene(allv, allt, np.tile(a, (len(allt), 1)))
    v.update(2, 4, [(0, L, (I, I, I))], sky=(0.2, 0.2, 0.2))
    rad, tri = v.pilot_rad(), v.pilot_tri()
    floor_hits = (tri >= 0) & (tri < len(ft))
    assert floor_hits.any()
    assert (rad[floor_hits] == 0).all()


def test_backface_hits_are_black():
    v, t = S.boxes_mesh([[-5, -5, -5]], [[5, 5, 5]], inward=False)  # outward: probes see back faces
    vol = O.OracleVolume((-1, -1, -1), (2, 2, 2), (2, 2, 2), rays_avg=8, rays_min=8, rays_max=8)
    vol.set_scene(v, t, np.full((len(t), 3), 0.8, np.float32))
    vol.update(0, 1, [(0, (0, 4, 0), (50, 50, 50))], sky=(1, 1, 1))
    assert (vol.pilot_tri() >= 0).all()
    assert (vol.pilot_rad() == 0).all()


# --------------------------------------------------------------- query
def _query_volume(values, depth_mu, depth_mu2=None, cheb_var_floor_rel=0.0):
    v = O.OracleVolume((0, 0, 0), (1, 1, 1), (2, 2, 2), rays_avg=8, rays_min=8, rays_max=8,
                       cheb_var_floor_rel=cheb_var_floor_rel)
    P = 8
    irr = np.zeros((P, v.Ti, v.Ti, 3))
    dep = np.zeros((P, v.Td, v.Td, 2))
    for p in range(P):
        irr[p] = values[p]
        dep[p, ..., 0] = depth_mu[p]
        dep[p, ..., 1] = depth_mu[p] ** 2 if depth_mu2 is None else depth_mu2[p]
    v.set_atlas(irr=irr, dep=dep)
    return v


def test_query_equal_probes_and_trilinear():
    rng = np.random.default_rng(6)
    v = _query_volume([np.array([0.3, 0.6, 0.9])] * 8, [10.0] * 8)
    pts = rng.uniform(0, 1, (100, 3)).astype(np.float32)
    nrm = rng.normal(size=(100, 3)).astype(np.float32)
    np.testing.assert_allclose(v.query(pts, nrm), np.tile([0.3, 0.6, 0.9], (100, 1)), rtol=1e-14)
    # distinct constant probes, depth far away: Chebyshev weight 1 -> plain
    # trilinear interpolation (weights sum to 1)
    vals = rng.uniform(0, 5, (8, 3))
    v = _query_volume(list(vals), [10.0] * 8)
    q = v.query(pts, nrm)
    for i, x in enumerate(pts.astype(np.float64)):
        ref = np.zeros(3)
        for c in range(8):
            o = [(c >> k) & 1 for k in range(3)]
            w = np.prod([x[k] if o[k] else 1 - x[k] for k in range(3)])
            ref += w * vals[c]
        np.testing.assert_allclose(q[i], ref, rtol=1e-12)
    # a point exactly on probe 5 returns probe 5's value
    q = v.query(np.array([[1, 0, 1]], np.float32), np.array([[0, 1, 0]], np.float32))
    np.testing.assert_allclose(q[0], vals[5], rtol=1e-14)


def test_query_chebyshev_weight():
    # probe 0 sees a wall at mean depth 0.1 with zero variance: for a point at
    # distance d > mu its weight is scaled by var/(var + (d-mu)^2), the
    # one-sided Chebyshev bound of variance shadow maps, with var raised to
    # the minimum 1e-6 s^2 (s^2 = 3 here).  A volume may opt in to a further
    # floor r * mu2; at r = 1e-3 that floor (1e-5) is above 1e-6 s^2 here, so
    # the two settings must give different weights.
    rng = np.random.default_rng(7)
    vals = rng.uniform(0, 5, (8, 3))
    mu = [0.1] + [10.0] * 7
    s2 = 3.0
    x = np.array([0.5, 0.25, 0.4])
    xf = x.astype(np.float32).astype(np.float64)
    got = {}
    for rel in (0.0, 1e-3):
        v = _query_volume(list(vals), mu, cheb_var_floor_rel=rel)
        q = v.query(x[None].astype(np.float32), np.array([[0, 0, 1]], np.float32))[0]
        ref_w = []
        for c in range(8):
            o = [(c >> k) & 1 for k in range(3)]
            w = np.prod([xf[k] if o[k] else 1 - xf[k] for k in range(3)])
            if c == 0:
                d = np.linalg.norm(xf)
                var = max(rel * 0.1 ** 2, 1e-6 * s2)
                w *= var / (var + (d - 0.1) ** 2)
            ref_w.append(w)
        ref_w = np.array(ref_w)
        np.testing.assert_allclose(q, (ref_w[:, None] * vals).sum(0) / ref_w.sum(), rtol=1e-12)
        got[rel] = q
    assert np.max(np.abs(got[0.0] - got[1e-3])) > 1e-6 * np.max(np.abs(got[0.0]))
    # a positive variance above both floors is used as it is
    v = _query_volume(list(vals), mu, depth_mu2=[0.1 ** 2 + 0.02] + [100.0] * 7)
    q = v.query(x[None].astype(np.float32), np.array([[0, 0, 1]], np.float32))[0]
    ref_w = []
    for c in range(8):
        o = [(c >> k) & 1 for k in range(3)]
        w = np.prod([xf[k] if o[k] else 1 - xf[k] for k in range(3)])
        if c == 0:
            d = np.linalg.norm(xf)
            w *= 0.02 / (0.02 + (d - 0.1) ** 2)
        ref_w.append(w)
    ref_w = np.array(ref_w)
    np.testing.assert_allclose(q, (ref_w[:, None] * vals).sum(0) / ref_w.sum(), rtol=1e-10)


# --------------------------------------------------------------- packed atlases
# The paper's 32-bit atlas codec (Sec. "Probe irradiance cache", "Probe
# visibility cache", appendix "Probe compression"): u = min(ln(gamma v + 1),
# beta) / beta, rounded down to b bits, decoded by (exp(beta u) - 1) / gamma.
CODECS = ((9, 5.0, 15.0), (8, 5.0, 15.0), (13, 5.0, 15.0), (13, 8.0, 20.0))


@pytest.mark.parametrize("which", range(4))
def test_codec_closed_form_and_round_down(which):
    bits, beta, gamma = CODECS[which]
    kmax = (1 << bits) - 1
    tab = O.codec_table(which).astype(np.float64)
    k = np.arange(kmax + 1)
    # decode: the closed form at u = k / kmax (FP32 rounding of the FP64 value)
    np.testing.assert_array_equal(tab.astype(np.float32), ((np.exp(beta * k / kmax) - 1.0) / gamma).astype(np.float32))
    assert tab[0] == 0.0 and (np.diff(tab) > 0).all()
    # every code decodes and codes back to itself
    for kk in list(range(0, kmax + 1, max(1, kmax // 300))) + [kmax]:
        assert O.codec_enc(which, tab[kk]) == kk
    # rounding down: dec(enc(v)) <= v < dec(enc(v) + 1), and the closed form
    # floor(u kmax) wherever v is not within FP32 rounding of a boundary
    rng = np.random.default_rng(3 + which)
    vals = np.concatenate([rng.exponential(0.3, 400), rng.uniform(0, tab[-1] * 1.2, 200), [0.0, -1.0, 1e9]])
    for v in vals.astype(np.float32):
        q = O.codec_enc(which, float(v))
        if v <= 0:
            assert q == 0
            continue
        assert tab[q] <= v
        assert q == kmax or v < tab[q + 1]
        u = min(math.log(gamma * float(v) + 1.0), beta) / beta * kmax
        if abs(u - round(u)) > 1e-4:
            assert q == min(int(math.floor(u)), kmax)
    assert O.codec_enc(which, float("nan")) == 0


def test_moving_average_step_and_floor_codec_dynamics():
    # Alg. MovingAvgUpdate: V = v/(n+1) + n o/(n+1); the first sample is taken as is
    assert O.codec_mav(0.25, 3.0, 0) == np.float32(3.0)
    assert O.codec_mav(2.0, 4.0, 1) == np.float32(3.0)
    # a constant stream settles at the code just below it and never above;
    # a dark stream then drives the code to exactly 0 (the reason the paper
    # rounds down: round-to-nearest could stall above zero)
    tab = O.codec_table(0)
    code, n = 0, 0
    for _ in range(200):
        code = O.codec_enc(0, O.codec_mav(tab[code], 1.7, n))
        n = min(n + 1, 63)
        assert tab[code] <= np.float32(1.7)
    assert code == O.codec_enc(0, 1.7) or tab[code + 1] > np.float32(1.7) * (1 - 0.02)
    steps = 0
    while code and steps < 5000:
        code = O.codec_enc(0, O.codec_mav(tab[code], 0.0, 63))
        steps += 1
    assert code == 0 and steps < 5000


def test_packed_constant_environment():
    # a constant sky radiance c: every touched irradiance texel decodes to the
    # largest code value not above c (monotone approach from below), and the
    # miss depth to the largest code value not above depth_max / s
    v = O.OracleVolume((0, 0, 0), (1, 1, 1), (3, 3, 3), rays_avg=16, rays_min=8, rays_max=64, packed=True)
    v.set_scene(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.float32))
    c = np.array((0.7, 1.3, 2.9), np.float32)
    t9, t8 = O.codec_table(0), O.codec_table(1)
    target = [t9[O.codec_enc(0, c[0])], t9[O.codec_enc(0, c[1])], t8[O.codec_enc(1, c[2])]]
    for f in range(40):
        v.update(f, 1, [], sky=tuple(c))
    pk = v.irr_packed()
    n = pk >> 26
    touched = n > 0
    assert touched.any() and (n[touched] >= 1).all() and n.max() >= 8
    dec = v.irr()[touched]
    assert (dec <= c.astype(np.float64) + 1e-7).all()
    # the first sample codes c exactly; later steps stay within [dec(enc(c)), c]
    # up to one FP32 rounding below
    for ch, tb, which in ((0, t9, 0), (1, t9, 0), (2, t8, 1)):
        codes = (pk[touched] >> (9 * ch)) & (511 if ch < 2 else 255)
        assert (np.abs(codes.astype(int) - O.codec_enc(which, c[ch])) <= 1).all()
    dpk = v.dep_packed()
    dn = dpk >> 26
    x = np.float32(v.depth_max) / np.float32(v.cage_diag)
    km = O.codec_enc(2, x)
    assert (np.abs((dpk[dn > 0] & 8191).astype(int) - km) <= 1).all()
    v.close()


# --------------------------------------------------------------- Metropolis sampler
# Eq. DDGIBays with the static guide h = exp(min(alpha g / f_s, 1)) f_s, chains
# of Alg. MarkovChainMT stepped by Alg. MetropolisStep.
def test_mh_tables():
    from statistics import NormalDist

    nd = NormalDist()
    q = np.array([O.mh_normal_quantile(i) for i in range(4096)], np.float64)
    ref = np.array([nd.inv_cdf((i + 0.5) / 4096) for i in range(4096)])
    np.testing.assert_allclose(q, ref, rtol=2e-7, atol=2e-7)
    np.testing.assert_array_equal(q[:2048], -q[::-1][:2048])  # symmetric
    e = np.array([O.mh_exp(k) for k in range(1024)], np.float32)
    np.testing.assert_array_equal(e, np.exp(np.arange(1024) / 1023.0).astype(np.float32))


def _mh_room(alpha, **kw):
    w = S.box_room(1)
    vd = dict(w.volume)
    v = O.OracleVolume(vd["origin"], vd["spacing"], vd["dims"], rays_avg=24, rays_min=8, rays_max=64,
                       sampler=1, alpha=alpha, **kw)
    v.set_scene(w.verts, w.idx, w.albedo)
    return v, w


def test_mh_guide_special_cases():
    v, w = _mh_room(0.0)
    for f in range(2):
        v.update(f, w.seed, w.lights_at(f), w.sky)
    qv = v.qv()
    dims = np.array(w.volume["dims"])
    rng = np.random.default_rng(5)
    seen_zero = seen_pos = 0
    for _ in range(300):
        g = (rng.random(3) * (dims - 1)).astype(np.float32)
        u = (rng.random(2) * 2 - 1).astype(np.float32)
        p = np.clip(np.floor(g + np.float32(0.5)).astype(int), 0, dims - 1)
        pi = int(p[0] + dims[0] * (p[1] + dims[1] * p[2]))
        # direction octant from the octahedral coordinates: sign of x, y, and
        # z < 0 outside the central diamond
        o = int(u[0] < 0) | (int(u[1] < 0) << 1) | (int(abs(u[0]) + abs(u[1]) > 1) << 2)
        fs = np.float32(1023 * int(qv[pi, o])) * np.float32(1.0 / 1046529.0)
        h0 = v.mh_guide(1, g, u)
        assert h0 == fs  # alpha = 0: exp(0) = 1, h = f_s
        seen_zero += fs == 0
        seen_pos += fs > 0
    assert seen_pos > 0
    # where nothing is hit (open sky) f_v, hence f_s and h, vanish
    sky = O.OracleVolume((0, 0, 0), (1, 1, 1), (3, 3, 3), rays_avg=16, rays_min=8, rays_max=64, sampler=1, alpha=1.0)
    sky.set_scene(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.float32))
    sky.update(0, 1, [], (0.5, 0.5, 0.5))
    sky.update(1, 1, [], (0.5, 0.5, 0.5))
    assert (sky.qv() == 0).all()
    assert sky.mh_guide(1, np.float32([1, 1, 1]), np.float32([0.2, -0.3])) == 0.0
    # a huge confidence saturates the cache term at e where the texel is lit
    v2, _ = _mh_room(1e9)
    for f in range(2):
        v2.update(f, w.seed, w.lights_at(f), w.sky)
    e = np.float32(math.e)
    hits = 0
    for _ in range(300):
        g = (rng.random(3) * (dims - 1)).astype(np.float32)
        u = (rng.random(2) * 2 - 1).astype(np.float32)
        h0, h1 = v.mh_guide(1, g, u), v2.mh_guide(1, g, u)
        if h0 > 0 and h1 > h0:
            assert h1 == np.float32(np.float32(O.mh_exp(1023)) * np.float32(h0))
            hits += 1
    assert hits > 20


def test_mh_budget_grouping_and_determinism():
    a, w = _mh_room(0.5)
    b, _ = _mh_room(0.5)
    for f in range(3):
        a.update(f, w.seed, w.lights_at(f), w.sky)
        b.update(f, w.seed, w.lights_at(f), w.sky)
        assert a.mh_samples == (24 - 8) * a.P
        pa, da = a.mh_probe(), a.mh_dir()
        np.testing.assert_array_equal(pa, b.mh_probe())
        np.testing.assert_array_equal(da, b.mh_dir())
        assert pa.min() >= 0 and pa.max() < a.P
        np.testing.assert_allclose(np.linalg.norm(da.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert a.mh_chains == -(-a.mh_samples // 5)


def test_mh_samples_follow_the_guide():
    # Stationarity of Alg. MarkovChainMT / MetropolisStep: on a fixed,
    # piecewise-constant guide h(probe cell, octant) the samples are
    # distributed in proportion to h times the cell volume (boundary probe
    # cells are half as wide per axis; octants have equal area in octahedral
    # coordinates), and cells with h = 0 get no samples once the chains sit
    # where h > 0 (the initial states are uniform).
    dims = np.array([3, 3, 3])
    P = 27
    rng = np.random.default_rng(2)
    tab = (rng.random((P, 8)) ** 2).astype(np.float32)
    tab[rng.random((P, 8)) < 0.3] = 0.0
    counts = O.mh_run_table(dims, tab, 200, 400, 10)
    i = np.arange(P)
    vol = np.ones(P)
    for ax in (i % 3, (i // 3) % 3, i // 9):
        vol *= np.where((ax == 0) | (ax == 2), 0.5, 1.0)
    target = tab.astype(np.float64) * vol[:, None]
    target /= target.sum()
    emp = counts / counts.sum()
    assert counts[tab == 0].sum() == 0
    tv = 0.5 * np.abs(emp - target).sum()
    assert tv < 0.05, tv  # measured 0.026 at 390k samples (0.012 at 1.95M)


def test_mh_visibility_ray_is_opposite():
    # a probe at the centre of a triangulated sphere: the -w ray of every
    # sample of that probe hits the sphere at distance r (chord bound), and
    # the +w ray hits it too
    r = 3.0
    sv, st = S.uv_sphere((0, 0, 0), r, 64, 32, inward=True)
    v = O.OracleVolume((0, 0, 0), (0.25, 0.25, 0.25), (2, 2, 2), rays_avg=64, rays_min=8, rays_max=128,
                       depth_max=10.0, sampler=1, alpha=0.0)
    v.set_scene(sv, st, np.full((len(st), 3), 0.5, np.float32))
    for f in range(3):
        v.update(f, 2, [])
    p = v.mh_probe()
    m = p == 0
    assert m.sum() > 10
    dep = v.mh_dep()[m]
    lo = r * math.cos(math.pi / 64) * math.cos(math.pi / 32)
    assert (dep <= r * (1 + 1e-6)).all() and (dep >= lo * (1 - 1e-6)).all()
    assert (v.mh_tri()[m] >= 0).all() and (v.mh_tri_neg()[m] >= 0).all()


# --------------------------------------------------------------- dynamic chains (virtual proxies)
def test_dyn_texel_centre_table():
    # every interior irradiance texel appears in exactly one octant list; its
    # FP32 centre direction is unit length, lies in that octant and bins back
    # to the texel (so a dynamic ray updates exactly the texel it was aimed at)
    for n in (1, 2, 6, 7):
        v = O.OracleVolume((0, 0, 0), (1, 1, 1), (3, 3, 3), n_irr=n, rays_avg=16, rays_min=8, rays_max=64,
                           sampler=1, dyn_ratio=4)
        tabs = v.dyn_texels()
        seen = np.concatenate([t for t, _ in tabs])
        T = n + 2
        interior = sorted((i + 1) * T + (j + 1) for i in range(n) for j in range(n))
        assert sorted(seen.tolist()) == interior
        for o, (ts, ds) in enumerate(tabs):
            for t, d in zip(ts, ds):
                assert abs(float(np.linalg.norm(d.astype(np.float64))) - 1.0) < 1e-6
                assert ((d[0] < 0) | ((d[1] < 0) << 1) | ((d[2] < 0) << 2)) == o
                assert O.texel_of_dir(d, n) == t
                np.testing.assert_array_equal(d, O.texel_centre_dir(t % T - 1, t // T - 1, n))


def test_dyn_budget_split():
    # adaptive samples B = (avg - 8) P split r:1: the static chains draw
    # floor(B r / (r + 1)) samples, the dynamic rays get twice the rest (a
    # static sample traces two rays), with ceil(C_s / r) dynamic chains
    for r, avg, dims in ((4, 64, (4, 4, 4)), (1, 16, (3, 5, 2)), (3, 8, (2, 2, 2)), (7, 40, (9, 5, 7))):
        v = O.OracleVolume((0, 0, 0), (1, 1, 1), dims, rays_avg=avg, rays_min=8, rays_max=256, sampler=1, dyn_ratio=r)
        P = int(np.prod(dims))
        B = (avg - 8) * P
        Bs = B * r // (r + 1)
        Cs = (Bs + 4) // 5
        s = v.dyn_sizes()
        assert v.mh_samples == Bs and v.mh_chains == Cs
        assert s["budget"] == 2 * (B - Bs)
        assert s["chains"] == (Cs + r - 1) // r and s["samples"] == 5 * s["chains"]
        assert s["proxies"] == int(np.prod([(d + 2) // 3 for d in dims]))
    with pytest.raises(ValueError):  # the dynamic chains belong to the Metropolis mode
        O.OracleVolume((0, 0, 0), (1, 1, 1), (3, 3, 3), rays_avg=16, sampler=0, dyn_ratio=4)


def _proxy_probes(q, dims):
    Dp = [(d + 2) // 3 for d in dims]
    qx, qy, qz = q % Dp[0], (q // Dp[0]) % Dp[1], q // (Dp[0] * Dp[1])
    return [x + dims[0] * (y + dims[1] * z) for z in range(3 * qz, min(3 * qz + 3, dims[2]))
            for y in range(3 * qy, min(3 * qy + 3, dims[1])) for x in range(3 * qx, min(3 * qx + 3, dims[0]))]


def _dyn_room(hyst=0.97, hyst_dyn=0.91, dims=(4, 4, 4), r=4, frames=6):
    w = S.box_room(1)
    vd = w.volume
    spacing = tuple(7.0 / (d - 1) for d in dims)
    v = O.OracleVolume((0.5, 0.5, 0.5), spacing, dims, rays_avg=48, rays_min=8, rays_max=128, hysteresis=hyst,
                       theta=8, sampler=1, alpha=1.0, dyn_ratio=r, hyst_dyn=hyst_dyn)
    v.set_scene(w.verts, w.idx, w.albedo)
    on = w.lights_at(0)
    for f in range(frames):  # the light is off on the second frame of every pair: a change in each pair
        v.update(f, 9, on if f % 2 == 0 else [])
    return w, v, dims


def test_dyn_marks_proxy_max_and_rays():
    w, v, dims = _dyn_room()
    qd = v.qd().astype(np.int64)
    assert qd.sum() > 0  # the toggling light gives the scene a dynamic component
    proxy, d, cell = v.dyn_samples()
    octant = (d[:, 0] < 0) | ((d[:, 1] < 0) << 1) | ((d[:, 2] < 0) << 2)
    # the coarsened target: max of q_d over the proxy's (clipped) 3x3x3 probes
    target = np.array([qd[_proxy_probes(q, dims), o].max() for q, o in zip(proxy, octant)])
    np.testing.assert_array_equal(cell, np.where(target > 0, proxy * 8 + octant, -1))
    # marks: each positive cell once, in the order of its first sample
    pos = np.flatnonzero(cell >= 0)
    _, first = np.unique(cell[pos], return_index=True)
    marks, traced = v.dyn_marks()
    np.testing.assert_array_equal(marks, cell[pos][np.sort(first)])
    ntex = [len(t) for t, _ in v.dyn_texels()]
    per_mark = np.array([len(_proxy_probes(c // 8, dims)) * ntex[c % 8] for c in marks], np.int64)
    s = v.dyn_sizes()
    csum = np.cumsum(per_mark)
    assert traced == int((csum <= s["budget"]).sum()) and s["rays"] == (int(csum[traced - 1]) if traced else 0)
    assert 0 < traced < len(marks)  # the budget cap binds in this case
    # the rays, grouped by probe: from every probe of a traced cell, one ray
    # per texel of the octant, through the texel centre
    R = v.dyn_rays()
    tabs = v.dyn_texels()
    nn = 36
    expect = []
    X, Y = dims[0], dims[1]
    inc = set(marks[:traced].tolist())
    for p in range(int(np.prod(dims))):
        q = (p % X) // 3 + ((dims[0] + 2) // 3) * (((p // X) % Y) // 3 + ((dims[1] + 2) // 3) * ((p // (X * Y)) // 3))
        for o in range(8):
            if q * 8 + o in inc:
                expect += [(p, o * nn + j) for j in range(ntex[o])]
    assert [(int(a), int(b)) for a, b in zip(R["probe"], R["key"])] == expect
    np.testing.assert_array_equal(R["off"], np.searchsorted(R["probe"], np.arange(len(R["off"])), side="left"))
    # hits against the brute-force trace
    o_ = np.stack([v.probe_pos(int(p)) for p in R["probe"]]).astype(np.float32)
    dirs = np.stack([tabs[k // nn][1][k % nn] for k in R["key"]]).astype(np.float32)
    t, tri, _ = O.trace_closest(w.verts, w.idx, o_, dirs, v.tmin, np.inf, use_bvh=False)
    np.testing.assert_array_equal(tri, R["tri"])
    hit = tri >= 0
    np.testing.assert_array_equal(t[hit], R["t"][hit])


def test_dyn_blend_step_closed_form():
    # hyst_dyn = 0: the dynamic batch weight is max(1, k/(n+k)) = 1, so after
    # the update a texel reached by k dynamic rays holds their mean radiance
    # (and their mean depth moments) whatever the static samples did before
    w, v, dims = _dyn_room(hyst_dyn=0.0)
    R = v.dyn_rays()
    assert len(R["probe"]) > 0
    tabs = v.dyn_texels()
    nn = 36
    irr, dep = v.irr(), v.dep()
    sums, cnt = {}, {}
    dsum, dcnt = {}, {}
    for p, k, rad, dp in zip(R["probe"], R["key"], R["rad"], R["dep"]):
        t = int(tabs[k // nn][0][k % nn])
        sums[(p, t)] = sums.get((p, t), 0) + rad
        cnt[(p, t)] = cnt.get((p, t), 0) + 1
        td = O.texel_of_dir(tabs[k // nn][1][k % nn], 14)
        dsum[(p, td)] = dsum.get((p, td), 0) + np.array([dp, dp * dp])
        dcnt[(p, td)] = dcnt.get((p, td), 0) + 1
    for (p, t), s_ in sums.items():
        np.testing.assert_allclose(irr[p].reshape(-1, 3)[t], s_ / cnt[(p, t)], rtol=1e-12, atol=1e-15)
    for (p, t), s_ in dsum.items():
        np.testing.assert_allclose(dep[p].reshape(-1, 2)[t], s_ / dcnt[(p, t)], rtol=1e-12, atol=1e-15)


def test_dyn_static_samples_snap_to_texel_centres():
    # static samples whose probe and octant carry q_d > 0 trace through texel
    # centres: +w through the centre of its irradiance texel, -w through the
    # centre of the visibility texel of -w
    w, v, dims = _dyn_room(frames=6)
    qd = v.qd()
    p, d = v.mh_probe(), v.mh_dir()
    octant = (d[:, 0] < 0) | ((d[:, 1] < 0) << 1) | ((d[:, 2] < 0) << 2)
    snap = qd[p, octant] > 0
    assert snap.sum() > 0
    idx = np.flatnonzero(snap)[:300]
    o_ = np.stack([v.probe_pos(int(q)) for q in p[idx]]).astype(np.float32)
    dp, dn = [], []
    for k in idx:
        t = O.texel_of_dir(d[k], 6)
        dp.append(O.texel_centre_dir(t % 8 - 1, t // 8 - 1, 6))
        tn = O.texel_of_dir(-d[k], 14)
        dn.append(O.texel_centre_dir(tn % 16 - 1, tn // 16 - 1, 14))
    _, trp, _ = O.trace_closest(w.verts, w.idx, o_, np.array(dp), v.tmin, np.inf, use_bvh=False)
    _, trn, _ = O.trace_closest(w.verts, w.idx, o_, np.array(dn), v.tmin, np.inf, use_bvh=False)
    np.testing.assert_array_equal(trp, v.mh_tri()[idx])
    np.testing.assert_array_equal(trn, v.mh_tri_neg()[idx])
    # the first frame has no pair yet (q_d = 0): samples trace their own directions
    w, v, dims = _dyn_room(frames=1)
    assert v.qd().sum() == 0
    p, d = v.mh_probe()[:300], v.mh_dir()[:300]
    o_ = np.stack([v.probe_pos(int(q)) for q in p]).astype(np.float32)
    _, trp, _ = O.trace_closest(w.verts, w.idx, o_, d, v.tmin, np.inf, use_bvh=False)
    _, trn, _ = O.trace_closest(w.verts, w.idx, o_, -d, v.tmin, np.inf, use_bvh=False)
    np.testing.assert_array_equal(trp, v.mh_tri()[:300])
    np.testing.assert_array_equal(trn, v.mh_tri_neg()[:300])


# --------------------------------------------------------------- camera clip volumes
def _clip_room(sampler=0, avg=32, dims=(5, 5, 5)):
    w = S.box_room(2)
    v = O.OracleVolume((-2.0, -2.0, -2.0), (1.0, 1.0, 1.0), dims, rays_avg=avg, rays_min=8, rays_max=128, theta=8,
                       sampler=sampler, alpha=0.0)
    # the room spans [0, 8]; probes at -2..2 sit partly outside: fine for classification
    v.set_scene(w.verts, w.idx, w.albedo)
    return w, v


def test_clip_volume_classification_closed_form():
    # M = identity: clip = (x, y, z, 1), so the extended frusta are the slabs
    # |x|, |y| <= 1.2 (V_in) and <= 1.4 (V_out); a camera at the origin with a
    # large k keeps f_c = 1 (probe grid at integer coordinates -2..2)
    w, v = _clip_room()
    M = np.eye(4, dtype=np.float32)
    v.update(0, 1, [], camera=((0.0, 0.0, 0.0), 100.0, M))
    cls = v.cls().reshape(5, 5, 5)  # [z][y][x]
    xs = np.arange(-2, 3)
    inner = (np.abs(xs)[None, :] <= 1) & (np.abs(xs)[:, None] <= 1)  # [y][x]
    expect = np.where(inner, 2, 0)[None, :, :].repeat(5, axis=0)
    np.testing.assert_array_equal(cls, expect)
    # a camera whose distance heuristic falls off: f_c >= 0.75 needs q_c >= 768
    v2 = _clip_room()[1]
    v2.update(0, 1, [], camera=((0.0, 0.0, 0.0), 0.0, M))
    lut_c = O.luts(v2.voxel_diag)[1]
    scale = np.float32(64.0 / v2.voxel_diag)
    qc = []
    for p in range(125):
        x = np.asarray(v2.probe_pos(p), np.float32)  # the camera at the origin: FP32 distance, then the LUT bin
        dist = np.sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2], dtype=np.float32)
        qc.append(int(lut_c[min(int(np.floor(np.float32(dist * scale))), 4095)]))
    qc = np.array(qc)
    c2 = v2.cls()
    assert ((c2 == 2) == ((qc >= 768) & (expect.reshape(-1) == 2))).all()
    # no matrix: every probe in V_in
    v3 = _clip_room()[1]
    v3.update(0, 1, [], camera=((0.0, 0.0, 0.0), 100.0))
    assert (v3.cls() == 2).all()


def test_clip_allocation_masked_invariants():
    rng = np.random.default_rng(5)
    for _ in range(200):
        P = int(rng.integers(1, 60))
        rmin = int(rng.integers(0, 20))
        m0 = max(rmin, 8)
        rmax = int(rng.integers(m0, 80))
        avg = int(rng.integers(m0, rmax + 1))
        W = (rng.integers(0, 4, P) * rng.integers(0, 1000, P)).astype(np.uint32)
        cls = rng.integers(0, 3, P).astype(np.uint8)
        n, off = O.allocate_masked(W, cls, avg, rmin, rmax)
        assert (n[cls == 0] == 0).all() and (n[cls == 1] == 8).all()
        vin = cls == 2
        assert (n[vin] >= m0).all() and (n[vin] <= rmax).all()
        # the adaptive budget (avg - 8) P, beyond the V_in floors, as far as the caps allow
        spend = min((avg - 8) * P - (m0 - 8) * int(vin.sum()), int(vin.sum()) * (rmax - m0))
        assert int(n[vin].sum()) - int(vin.sum()) * m0 == spend
        a = np.where(n > 8, n - 8, 0).astype(np.int64)
        np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(a)]))
        # every probe in V_in: the plain rule
        n2, off2 = O.allocate_masked(W, np.full(P, 2, np.uint8), avg, rmin, rmax)
        n3, off3 = O.allocate(W, avg, rmin, rmax)
        np.testing.assert_array_equal(n2, n3)
        np.testing.assert_array_equal(off2, off3)


def test_clip_outside_probes_frozen_and_static_scene_stays_quiet():
    # a static scene while the camera (hence the clip volumes) moves: probes
    # outside V_out trace nothing and keep their atlases; gradients need both
    # frames of a pair inside V_out, so W stays 0 (no spurious triggers)
    w, v = _clip_room(avg=32)
    light = [(0, (4.0, 6.0, 4.0), (30.0, 30.0, 30.0))]
    M = np.eye(4, dtype=np.float32)
    for f in range(12):
        Mf = M.copy()
        Mf[0, 3] = [0.0, 1.0, -1.0, 0.5][f % 4]  # slide the slab in x every frame
        before_irr, before_n = v.irr().copy(), v.irr_n().copy()
        v.update(f, 3, light, camera=((0.0, 0.0, 0.0), 100.0, Mf))
        cls = v.cls()
        out = cls == 0
        assert (v.pilot_tri()[out] == -1).all()
        np.testing.assert_array_equal(v.irr()[out], before_irr[out])
        np.testing.assert_array_equal(v.irr_n()[out], before_n[out])
        assert (v.n()[out] == 0).all() and (v.n()[cls == 1] == 8).all()
        assert v.W().sum() == 0, f


def test_clip_catch_up_counts_and_vin_keeps_counting():
    # V_out - V_in probes have every texel count set down to 16 (Sec.
    # "Adaptive sampling - static", last paragraph); V_in probes keep counting
    w, v = _clip_room(avg=64)
    light = [(0, (4.0, 6.0, 4.0), (30.0, 30.0, 30.0))]
    M = np.eye(4, dtype=np.float32)
    M[0, 0] = M[1, 1] = 0.65  # V_in: |x|, |y| <= 1.2 / 0.65 = 1.85; V_out: <= 1.4 / 0.65 = 2.15
    for f in range(16):
        v.update(f, 3, light)  # everything in V_in: counts grow past 16
    assert v.irr_n().max() > 16
    v.update(16, 3, light, camera=((0.0, 0.0, 0.0), 100.0, M))
    cls = v.cls()
    assert (cls == 1).any() and (cls == 2).any()
    assert (v.irr_n()[cls == 1] <= 16).all() and (v.dep_n()[cls == 1] <= 16).all()
    assert v.irr_n()[cls == 2].max() > 16


def test_clip_metropolis_samples_only_inside_vin():
    w, v = _clip_room(sampler=1, avg=32)
    M = np.eye(4, dtype=np.float32)
    light = [(0, (4.0, 6.0, 4.0), (30.0, 30.0, 30.0))]
    for f in range(4):
        v.update(f, 3, light, camera=((0.0, 0.0, 0.0), 100.0, M))
    cls = v.cls()
    p = v.mh_probe()
    outside = cls[p] != 2
    assert outside.any() and (~outside).any()
    assert (v.mh_tri()[outside] == -1).all() and (v.mh_tri_neg()[outside] == -1).all()


# --------------------------------------------------------------- DDGI cosine-gather blend
def test_cosine_gather_constant_environment():
    # sky only (radiance c everywhere, every ray a miss): the c-weighted mean
    # of a constant is that constant, and the depth moments are those of
    # depth_max, at every texel after the first frame
    v = O.OracleVolume((0, 0, 0), (1, 1, 1), (2, 2, 2), rays_avg=64, rays_min=8, rays_max=64, blend_mode=1)
    v.set_scene(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.float32))
    sky = (0.3, 1.2, 2.5)
    v.update(0, 1, [], sky)
    irr, dep = v.irr(), v.dep()
    np.testing.assert_allclose(irr, np.broadcast_to(np.float32(sky).astype(np.float64), irr.shape), rtol=1e-12)
    dm = v.depth_max
    np.testing.assert_allclose(dep[..., 0], dm, rtol=1e-12)
    np.testing.assert_allclose(dep[..., 1], dm * dm, rtol=1e-12)
    assert (v.irr_n() > 16).all()  # about half of the 64 rays face each texel


def test_cosine_gather_half_space_closed_form():
    # a probe high above an infinite black floor under a sky of radiance c:
    # the cosine-weighted share of the hemisphere around n that sees the sky
    # is (1 + n_z)/2, so the irradiance texel at n holds c (1 + n_z)/2; a
    # downward depth texel (the sharp c^50 lobe) holds about h / |n_z|
    h = 3.0
    big = 1e4
    verts = np.array([[-big, -big, 0], [big, -big, 0], [big, big, 0], [-big, big, 0]], np.float32)
    idx = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    v = O.OracleVolume((0, 0, h), (0.5, 0.5, 0.5), (2, 2, 2), rays_avg=1024, rays_min=1024, rays_max=1024,
                       depth_max=100.0, blend_mode=1, hysteresis=0.0)
    v.set_scene(verts, idx, np.zeros((2, 3), np.float32))
    c = 2.0
    v.update(1, 5, [], (c, c, c))  # an odd frame: no pilots, the 1016 spherical-Fibonacci rays alone
    irr = v.irr()[0]  # probe 0 at (0, 0, 3)
    dep = v.dep()[0]
    n = 6
    for cy in range(n):
        for cx in range(n):
            nt = O.oct_decode([((cx + 0.5) / n) * 2 - 1, ((cy + 0.5) / n) * 2 - 1])
            np.testing.assert_allclose(irr[cy + 1, cx + 1], c * (1 + nt[2]) / 2, atol=0.02 * c)
    nd = 14
    for cy in range(nd):
        for cx in range(nd):
            nt = O.oct_decode([((cx + 0.5) / nd) * 2 - 1, ((cy + 0.5) / nd) * 2 - 1])
            if nt[2] < -0.9:  # the lobe's spread (~1/sqrt(50) rad) biases h / |n_z| upward by ~1-2 %
                assert abs(dep[cy + 1, cx + 1, 0] / (h / -nt[2]) - 1) < 0.03
            elif nt[2] > 0.6:  # sky: misses at depth_max (floor rays are >= 37 deg off the lobe: weight < 2e-5)
                assert abs(dep[cy + 1, cx + 1, 0] / v.depth_max - 1) < 1e-3
