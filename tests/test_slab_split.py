"""Probe-slab split of one volume's update (paper_2301_05125_gb300.slab) on
CPU ranks with the oracle as each rank's engine.

The split must reproduce the unsplit update exactly: every integer output
(W, n, offsets, pilot and adaptive hit indices and t) and the FP64 atlases
are compared for equality, on the ragged small city (9 x 5 x 7 probes, a
z-extent that does not divide evenly) over four frames, so the change
measure has fired and the allocation is not uniform.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2301_05125_gb300 import scenegen as S
from paper_2301_05125_gb300.slab import LocalExchange, SlabPart, halo_ranges, slab_ranges, slab_update

FRAMES = 4


def _world():
    return S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)


def test_slab_ranges_and_halos():
    # 7 planes of 45 probes over 3 ranks: 3 + 2 + 2 (the first Z mod n ranks
    # take one plane more)
    assert slab_ranges((9, 5, 7), 3) == [(0, 135), (135, 225), (225, 315)]


def test_slab_ranges_split_planes_evenly():
    dims = (9, 5, 7)
    plane = 45
    for n in range(1, 8):
        r = slab_ranges(dims, n)
        assert r[0][0] == 0 and r[-1][1] == 315
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [(hi - lo) // plane for lo, hi in r]
        assert all(lo % plane == 0 for lo, _ in r) and max(sizes) - min(sizes) <= 1 and sum(sizes) == 7
    with pytest.raises(ValueError):
        slab_ranges(dims, 8)
    # halos: two planes on each side, clipped to the grid
    assert halo_ranges(dims, (0, 135)) == [(135, 225)]
    assert halo_ranges(dims, (135, 225)) == [(45, 135), (225, 315)]
    assert halo_ranges(dims, (270, 315)) == [(180, 270)]


def _compare(ranks_out, single, what):
    per, final = single
    for f in range(FRAMES):
        ref = per[f]
        for rng, rec in ranks_out[f]:
            p0, p1 = rng
            off = ref["off"]
            r0, r1 = int(off[p0]), int(off[p1])
            tag = "%s frame %d probes %d-%d" % (what, f, p0, p1)
            np.testing.assert_array_equal(rec["W"], ref["W"][p0:p1], err_msg=tag + " W")
            np.testing.assert_array_equal(rec["n"], ref["n"], err_msg=tag + " n")
            np.testing.assert_array_equal(rec["off"], ref["off"], err_msg=tag + " off")
            np.testing.assert_array_equal(rec["pilot_tri"], ref["pilot_tri"][p0:p1], err_msg=tag + " pilot tri")
            np.testing.assert_array_equal(rec["pilot_t"], ref["pilot_t"][p0:p1], err_msg=tag + " pilot t")
            np.testing.assert_array_equal(rec["main_tri"], ref["main_tri"][r0:r1], err_msg=tag + " main tri")
            np.testing.assert_array_equal(rec["main_t"], ref["main_t"][r0:r1], err_msg=tag + " main t")
    assert sum(int(x["W"].astype(np.int64).sum()) for x in per) > 0  # the allocation was not uniform


@pytest.mark.parametrize("n_ranks", [2, 3])
def test_split_in_one_process_equals_unsplit_oracle(n_ranks):
    pytest.importorskip("torch")
    from _slab_oracle import OracleSlabRank, rank_record, single_run

    w = _world()
    single = single_run(w, FRAMES)
    ranges = slab_ranges(w.volume["dims"], n_ranks)
    parts = [SlabPart(OracleSlabRank(w), r, ranges[r]) for r in range(n_ranks)]
    ex = LocalExchange(w.volume["dims"], ranges)
    out = []
    for f in range(FRAMES):
        slab_update(parts, ex, f)
        out.append([(p.rng, rank_record(p.backend, p.rng)) for p in parts])
    _compare(out, single, "%d ranks" % n_ranks)
    # after the tile gather every rank holds the whole atlas of the unsplit run
    _, final = single
    for p in parts:
        ov = p.backend.ov
        np.testing.assert_array_equal(ov.irr(), final["irr"])
        np.testing.assert_array_equal(ov.irr_n(), final["irr_n"])
        np.testing.assert_array_equal(ov.dep(), final["dep"])
        np.testing.assert_array_equal(ov.dep_n(), final["dep_n"])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_on_two_gloo_ranks_equals_unsplit_oracle(tmp_path):
    pytest.importorskip("torch")
    from _mp_workers import slab_worker
    from _slab_oracle import single_run

    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=slab_worker, args=(r, 2, port, str(tmp_path), FRAMES)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    w = _world()
    single = single_run(w, FRAMES)
    ranges = slab_ranges(w.volume["dims"], 2)
    out = [[] for _ in range(FRAMES)]
    for r in range(2):
        d = np.load(os.path.join(str(tmp_path), "slab_rank%d.npz" % r))
        for f in range(FRAMES):
            rec = {k: d["f%d_%s" % (f, k)] for k in ("W", "n", "off", "pilot_tri", "pilot_t", "main_tri", "main_t")}
            out[f].append((ranges[r], rec))
        _, final = single
        for k in ("irr", "irr_n", "dep", "dep_n"):
            np.testing.assert_array_equal(d["final_" + k], final[k], err_msg="rank %d %s" % (r, k))
    _compare(out, single, "gloo ranks")
