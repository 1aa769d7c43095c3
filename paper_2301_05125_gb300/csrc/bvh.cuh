// bvh.cuh -- device LBVH owned by a volume (see bvh.cu).
#pragma once
#include <cuda_runtime.h>

#include "adgi_internal.cuh"

namespace adgi {

// Device buffers of one build: the outputs (tri_v, nodes) and the scratch.
struct BvhBufs {
    float4* tri_v = nullptr;     // [3*n] output: BVH order, v0.w = original index
    BNode* nodes = nullptr;      // [n-1] output
    float4* tri_orig = nullptr;  // [3*n] scratch (kept by volumes for shading normals)
    int* par_int = nullptr;
    int* par_leaf = nullptr;
    int* flags = nullptr;
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    uint32_t* bounds = nullptr;
    int* err = nullptr;
};

size_t bvh_scratch_bytes(int nt);
size_t carve_bvh_scratch(void* base, int nt, BvhBufs& B);
cudaError_t build_lbvh(const BvhBufs& B, const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err,
                       cudaStream_t s, int* root_leaf);

struct Bvh {
    int n_tris = 0;
    int root_leaf = -1;
    float4* tri_orig = nullptr;  // [3*n] original order (inside scratch)
    float4* tri_v = nullptr;     // [3*n] BVH order, v0.w = original index
    BNode* nodes = nullptr;      // [n-1]
    void* scratch = nullptr;
    BvhBufs bufs;
    int cap_ = 0;
    size_t bytes_ = 0;

    cudaError_t reserve(int nt);
    cudaError_t build(const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err, cudaStream_t s);
    void release();
    size_t bytes() const;
    SceneDev view(const float* albedo, int nv, int* err) const;
};

}  // namespace adgi
