// noalloc.cu -- adgi_build_bvh_noalloc: the BVH build of adgi_build_bvh with
// its scratch in a fixed, file-scope device array instead of memory allocated
// per call.
//
// Some callers may not allocate device memory while they run: a renderer's
// frame loop that must never stall on an allocation (cudaMalloc and cudaFree
// can synchronise the whole device), or a plugin living inside a host
// application whose own allocator has already reserved the device memory it is
// allowed to use.  This entry point serves them: the caller passes the inputs
// and the outputs, and the scratch (sort keys and values, parent links, flags,
// histograms) lives in g_bvh_scratch below.
//
// Costs and rules:
//   * every GPU that loads this library holds the array (kNoallocScratchBytes,
//     about 2.6 MiB) until the process exits;
//   * host code cannot use the array's name as a device address (on the host
//     it is only a stand-in symbol), so each call looks the address up with
//     cudaGetSymbolAddress in the context current on the calling thread and
//     checks the result.  The lookup allocates nothing once the library's
//     device code is loaded in that context (the first call in a context may
//     load it), and it is right in any context, primary or not, and after a
//     cudaDeviceReset;
//   * all calls share the one array and it keeps the last call's contents;
//     each call re-initialises what must start at zero (flags, bounds, error
//     word) on its own stream;
//   * two calls whose work overlaps on the GPU (different streams, or host
//     threads racing) corrupt each other's scratch: order them on one stream
//     or serialise them;
//   * a call reads the build's error word back and synchronises its stream,
//     so it must not be called while that stream is being captured.
#include <string>

#include "adgi_internal.cuh"
#include "bvh.cuh"

namespace adgi {
const char* noalloc_fail(const std::string& msg);
}

using namespace adgi;

namespace {

constexpr int kMaxTris = ADGI_BVH_NOALLOC_MAX_TRIS;
// the layout carve_bvh_scratch() cuts for kMaxTris triangles
constexpr size_t kNoallocScratchBytes = bvh_scratch_layout_bytes(kMaxTris);
static_assert(kNoallocScratchBytes < (3u << 20), "the fixed scratch stays a modest static array");

static __device__ __align__(256) unsigned char g_bvh_scratch[kNoallocScratchBytes];

}  // namespace

extern "C" int adgi_build_bvh_noalloc(const float* verts, int32_t nv, const int32_t* idx, int32_t nt, float eps,
                                      void* nodes_out, void* tris_out, void* cuda_stream)
{
    if (nt > kMaxTris) {
        noalloc_fail("adgi_build_bvh_noalloc: " + std::to_string(nt) + " triangles exceed the fixed scratch for " +
                     std::to_string(kMaxTris) + "; use adgi_build_bvh");
        return ADGI_ERR_INVALID_ARG;
    }
    if (nv < 0 || nt < 0 || (nt > 0 && (nv <= 0 || !verts || !idx || !nodes_out || !tris_out)) || !(eps >= 0.0f)) {
        noalloc_fail("adgi_build_bvh_noalloc: bad arguments");
        return ADGI_ERR_INVALID_ARG;
    }
    if (nt == 0) return ADGI_OK;
    // the array's device address in the calling thread's current context
    void* base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, g_bvh_scratch);
    if (e != cudaSuccess || !base) {
        noalloc_fail(std::string("adgi_build_bvh_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return ADGI_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BvhBufs B;
    const size_t need = carve_bvh_scratch(nullptr, nt, B);
    if (need != bvh_scratch_layout_bytes((size_t)nt) || need > kNoallocScratchBytes) {
        noalloc_fail("adgi_build_bvh_noalloc: scratch layout does not fit the fixed array");
        return ADGI_ERR_INVALID_ARG;
    }
    carve_bvh_scratch(base, nt, B);
    B.tri_v = (float4*)tris_out;
    B.nodes = (BNode*)nodes_out;
    int root = -1;
    e = cudaMemsetAsync(B.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = build_lbvh(B, verts, idx, nv, nt, eps, B.err, s, &root);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        noalloc_fail(std::string("adgi_build_bvh_noalloc: ") + cudaGetErrorString(e));
        return ADGI_ERR_CUDA;
    }
    if (herr & kErrIndex) {
        noalloc_fail("adgi_build_bvh_noalloc: triangle index outside [0, n_verts)");
        return ADGI_ERR_INVALID_ARG;
    }
    if (herr) {
        noalloc_fail("adgi_build_bvh_noalloc: device anomaly flags set: " + std::to_string(herr));
        return ADGI_ERR_CUDA;
    }
    return ADGI_OK;
}
