// bvh.cuh -- device LBVH owned by a volume (see bvh.cu).
#pragma once
#include <cuda_runtime.h>

#include "adgi_internal.cuh"

namespace adgi {

struct Bvh {
    int n_tris = 0;
    int root_leaf = -1;
    float4* tri_orig = nullptr;  // [3*n] original order
    float4* tri_v = nullptr;     // [3*n] BVH order, v0.w = original index
    BNode* nodes = nullptr;      // [n-1]
    int* par_int = nullptr;
    int* par_leaf = nullptr;
    int* flags = nullptr;
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    uint32_t* bounds = nullptr;
    int cap_ = 0;
    size_t bytes_ = 0;

    cudaError_t reserve(int nt);
    cudaError_t build(const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err, cudaStream_t s);
    void release();
    size_t bytes() const;
    SceneDev view(const float* albedo, int nv, int* err) const;
};

}  // namespace adgi
