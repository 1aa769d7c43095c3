"""The allocation-free BVH build (adgi_build_bvh_noalloc).

It exists for callers that may not allocate device memory while they run
(a frame loop that must not stall on cudaMalloc/cudaFree, or a plugin whose
host application's allocator owns the device memory).  It must produce
exactly what the allocating adgi_build_bvh produces -- the BVH is integer and
bit-copy work, so the comparison is bit-exact -- on consecutive calls that
reuse the same fixed scratch array.

This file is collected last so that a failure here leaves every other test
already run; it builds and loads the library itself, so it also runs alone.
"""
import numpy as np
import pytest

from paper_2301_05125_gb300 import scenegen as S

torch = pytest.importorskip("torch")


def _lib():
    from paper_2301_05125_gb300 import adgi as A
    from paper_2301_05125_gb300 import build

    build.build()
    A.load()
    return A


def _bufs(nt, dev):
    nodes = torch.full((max(nt - 1, 1) * 16,), -7, dtype=torch.int32, device=dev)
    tris = torch.full((nt * 12,), -7.0, dtype=torch.float32, device=dev)
    return nodes, tris


@pytest.mark.gpu
def test_noalloc_build_matches_allocating_build_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A = _lib()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    scenes = [S.small_city(7, n_boxes=2000), S.box_room(1), S.small_city(8, n_boxes=1800)]
    for w in scenes:
        assert w.n_tris <= A.BVH_NOALLOC_MAX_TRIS
        V = torch.from_numpy(w.verts).to(dev)
        I = torch.from_numpy(w.idx).to(dev)
        eps = A.scene_eps(w.verts)
        ref_nodes, ref_tris = _bufs(w.n_tris, dev)
        A.adgi_build_bvh(V, I, eps, ref_nodes, ref_tris, stream)
        ref_n, ref_t = ref_nodes.cpu().numpy(), ref_tris.cpu().numpy().view(np.int32)
        for call in range(2):  # two calls in a row on the shared scratch
            nodes, tris = _bufs(w.n_tris, dev)
            A.adgi_build_bvh_noalloc(V, I, eps, nodes, tris, stream)
            np.testing.assert_array_equal(nodes.cpu().numpy(), ref_n, err_msg="%s call %d nodes" % (w.name, call))
            np.testing.assert_array_equal(tris.cpu().numpy().view(np.int32), ref_t,
                                          err_msg="%s call %d triangles" % (w.name, call))


@pytest.mark.gpu
def test_noalloc_build_at_its_maximum_size():
    """A build of exactly BVH_NOALLOC_MAX_TRIS triangles fills the fixed
    scratch to its limit and still equals the allocating build."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A = _lib()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    w = S.small_city(9, n_boxes=3000)
    n = A.BVH_NOALLOC_MAX_TRIS
    assert w.n_tris >= n
    idx = np.ascontiguousarray(w.idx.reshape(-1, 3)[:n])
    V = torch.from_numpy(w.verts).to(dev)
    I = torch.from_numpy(idx).to(dev)
    eps = A.scene_eps(w.verts)
    ref_nodes, ref_tris = _bufs(n, dev)
    A.adgi_build_bvh(V, I, eps, ref_nodes, ref_tris, stream)
    for call in range(2):
        nodes, tris = _bufs(n, dev)
        A.adgi_build_bvh_noalloc(V, I, eps, nodes, tris, stream)
        np.testing.assert_array_equal(nodes.cpu().numpy(), ref_nodes.cpu().numpy(), err_msg="call %d nodes" % call)
        np.testing.assert_array_equal(tris.cpu().numpy().view(np.int32), ref_tris.cpu().numpy().view(np.int32),
                                      err_msg="call %d triangles" % call)


def test_noalloc_build_rejects_sizes_beyond_its_scratch():
    """Host-side check, before any device work: too many triangles is an
    INVALID_ARG with a message that names the limit."""
    A = _lib()
    n = A.BVH_NOALLOC_MAX_TRIS + 1
    verts = np.zeros((3, 3), np.float32)
    idx = np.zeros((1, 3), np.int32)
    with pytest.raises(A.AdgiError) as e:
        A.adgi_build_bvh_noalloc(verts, idx, 1e-4, verts, verts, None, n_tris=n)
    assert e.value.code == -1
    assert str(A.BVH_NOALLOC_MAX_TRIS) in str(e.value)
