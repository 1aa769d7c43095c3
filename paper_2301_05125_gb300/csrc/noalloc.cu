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
//     it is only a stand-in symbol), so the first call on each device looks the
//     address up with cudaGetSymbolAddress while that device is current and
//     keeps it; make that first call before any stream capture begins;
//   * all calls share the one array and it keeps the last call's contents;
//     each call re-initialises what must start at zero (flags, bounds, error
//     word) on its own stream;
//   * two calls whose work overlaps on the GPU (different streams, or host
//     threads racing) corrupt each other's scratch: order them on one stream
//     or serialise them.
#include <mutex>
#include <string>

#include "adgi_internal.cuh"
#include "bvh.cuh"

namespace adgi {
const char* noalloc_fail(const std::string& msg);
}

using namespace adgi;

namespace {

// Scratch layout of carve_bvh_scratch() for kMaxTris triangles: each piece is
// rounded up to 256 bytes.
constexpr size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t scratch_bytes_for(size_t n)
{
    return r256(48 * n) + 3 * r256(4 * n) + 2 * r256(8 * n) + 2 * r256(4 * n) + r256(1024 * ((n + 4095) / 4096)) +
           r256(32) + r256(8);
}
constexpr int kMaxTris = ADGI_BVH_NOALLOC_MAX_TRIS;
constexpr size_t kNoallocScratchBytes = scratch_bytes_for(kMaxTris);

static __device__ __align__(256) unsigned char g_bvh_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        noalloc_fail(std::string("adgi_build_bvh_noalloc: no usable current device: ") + cudaGetErrorString(e));
        return ADGI_ERR_CUDA;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            // set-up, once per device, with that device current
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_bvh_scratch);
            if (e != cudaSuccess || !p) {
                noalloc_fail(std::string("adgi_build_bvh_noalloc: cudaGetSymbolAddress failed: ") +
                             cudaGetErrorString(e));
                return ADGI_ERR_CUDA;
            }
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BvhBufs B;
    if (carve_bvh_scratch(nullptr, nt, B) > kNoallocScratchBytes) {
        noalloc_fail("adgi_build_bvh_noalloc: scratch layout exceeds the fixed array");
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
