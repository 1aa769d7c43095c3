"""Probe-slab split of one volume's update on the GPU (adgi_update_slab,
adgi_slab_copy and the driver in paper_2301_05125_gb300.slab).

This pool gives one GPU to a run, so the ranks are emulated: each rank is a
volume of its own on the same device and stream, and LocalExchange moves the
slices between them (the multi-process path, DistExchange over NCCL, differs
only in how the bytes travel; its logic runs with gloo ranks in
tests/test_slab_split.py).  The split must equal one unsplit volume's update
bit for bit: W, n, offsets, every hit, and the raw atlas bytes.
"""
import numpy as np
import pytest

from paper_2301_05125_gb300 import scenegen as S

from _helpers import gpu_volume

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


@pytest.mark.parametrize("n_ranks,over", [(2, {}), (3, {}), (2, {"atlas_fp16": 1}), (3, {"blend_mode": 1})])
def test_split_equals_unsplit_update(adgi, n_ranks, over):
    from paper_2301_05125_gb300.slab import CudaSlabRank, LocalExchange, SlabPart, slab_ranges, slab_update

    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    full = gpu_volume(adgi, w, stream=stream, **over)
    ranges = slab_ranges(w.volume["dims"], n_ranks)
    vols = [gpu_volume(adgi, w, stream=stream, **over) for _ in range(n_ranks)]
    parts = [SlabPart(CudaSlabRank(v, dev), r, ranges[r]) for r, v in enumerate(vols)]
    ex = LocalExchange(w.volume["dims"], ranges)
    wsum = 0
    for f in range(5):
        fr = adgi.make_frame(f, w.seed, w.lights_at(f), w.sky)
        if w.dyn_at is not None and w.dyn_count:
            dv = np.ascontiguousarray(w.dyn_at(f), np.float32)
            for v in [full] + vols:
                v.move_vertices(w.dyn_first, dv)
        adgi.adgi_update(full.h, fr)
        slab_update(parts, ex, fr)
        torch.cuda.synchronize()
        full.stats()
        W, n, off = full.W(), full.n(), full.off()
        wsum += int(W.astype(np.int64).sum())
        ph, mh = full.pilot_hit(), full.main_hit()
        for (p0, p1), v in zip(ranges, vols):
            tag = "frame %d probes %d-%d" % (f, p0, p1)
            v.stats()
            np.testing.assert_array_equal(v.W()[p0:p1], W[p0:p1], err_msg=tag + " W")
            np.testing.assert_array_equal(v.n(), n, err_msg=tag + " n")
            np.testing.assert_array_equal(v.off(), off, err_msg=tag + " off")
            np.testing.assert_array_equal(v.pilot_hit()[p0:p1], ph[p0:p1], err_msg=tag + " pilot hits")
            r0, r1 = int(off[p0]), int(off[p1])
            np.testing.assert_array_equal(v.main_hit()[r0:r1], mh[r0:r1], err_msg=tag + " main hits")
            for which in ("IRR", "DEP", "DEP_N"):  # every rank holds the whole atlas after the gather
                np.testing.assert_array_equal(v.state(which, np.uint8), full.state(which, np.uint8),
                                              err_msg=tag + " " + which)
    assert wsum > 0  # the change measure fired: the allocation was not uniform
    for v in [full] + vols:
        v.close()


def test_slab_steps_are_checked(adgi):
    w = S.box_room(1)
    v = gpu_volume(adgi, w)
    fr = adgi.make_frame(0, w.seed, w.lights_at(0), w.sky)
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_update_slab(v.h, fr, 1, 0, 16)  # step 1 before step 0
    adgi.adgi_update_slab(v.h, fr, 0, 0, 16)
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_update_slab(v.h, fr, 1, 0, 32)  # another probe range
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_update_slab(v.h, fr, 0, 0, 65)  # beyond the grid
    v.close()
