"""Failure paths, with the failures made on the host.

A device allocation is made to fail the way cudaMalloc fails on a full
device (adgi_inject_alloc_failure: the call reports the error without
allocating), at the first, a middle and a late allocation of a volume.  The
call must return OOM, release everything it had allocated, and leave the
library able to build and update the next volume.  Nothing here faults,
traps or stalls a GPU.
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


def test_allocation_failure_returns_oom_and_releases_memory(adgi):
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    ref = gpu_volume(adgi, w)  # the same frames on an undisturbed volume
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for n in (1, 9, 20):
            adgi.adgi_inject_alloc_failure(n)
            with pytest.raises(adgi.AdgiError) as e:
                adgi.Volume(**w.volume)
            assert e.value.code == -2, "allocation %d" % n
    finally:
        adgi.adgi_inject_alloc_failure(0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (16 << 20), "device memory not released: %d bytes" % (free0 - free1)
    v = gpu_volume(adgi, w)
    for f in range(2):
        for x in (ref, v):
            if w.dyn_at is not None and w.dyn_count:
                x.move_vertices(w.dyn_first, w.dyn_at(f))
            x.update(f, w.seed, w.lights_at(f), w.sky)
    np.testing.assert_array_equal(v.n(), ref.n())
    np.testing.assert_array_equal(v.main_hit(), ref.main_hit())
    np.testing.assert_array_equal(v.irr(), ref.irr())
    v.close()
    ref.close()


def test_injection_rejects_negative_counts(adgi):
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_inject_alloc_failure(-1)
