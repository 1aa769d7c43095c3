// bvh.cuh -- device LBVH owned by a volume (see bvh.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "adgi_internal.cuh"

namespace adgi {

// Device buffers of one build: the outputs (tri_v, nodes) and the scratch.
struct BvhBufs {
    float4* tri_v = nullptr;     // [3*n] output: BVH order, v0.w = original index
    BNode* nodes = nullptr;      // [n-1] output
    float4* tri_in = nullptr;    // [3*n] scratch: the listed triangles, v0.w = original index
    int* par_int = nullptr;
    int* par_leaf = nullptr;
    int* flags = nullptr;
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    uint32_t* bounds = nullptr;
    int* err = nullptr;
};

// extra scratch of the PLOC build
struct PlocBufs {
    int* cid[2] = {nullptr, nullptr};
    float4* blo[2] = {nullptr, nullptr};
    float4* bhi[2] = {nullptr, nullptr};
    int* nn = nullptr;
    uint64_t* flags = nullptr;
    uint64_t* pre = nullptr;
    uint64_t* sums = nullptr;
    uint64_t* total = nullptr;
};

// Bytes of the scratch block carve_bvh_scratch() cuts for a linear build of
// nt triangles: the listed triangles (48 B each), parent links and flags
// (3 x 4 B), sort keys (2 x 8 B) and values (2 x 4 B), one 256-bin histogram
// per radix tile of kBvhSortTile keys, the centroid bounds and the error
// word, every piece rounded up to 256 bytes.
constexpr int kBvhSortTile = 4096;
constexpr size_t bvh_r256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t bvh_scratch_layout_bytes(size_t nt)
{
    const size_t n = nt > 0 ? nt : 1;
    return bvh_r256(48 * n) + 3 * bvh_r256(4 * n) + 2 * bvh_r256(8 * n) + 2 * bvh_r256(4 * n) +
           bvh_r256(4 * 256 * ((n + kBvhSortTile - 1) / kBvhSortTile)) + bvh_r256(4 * 8) + bvh_r256(4 * 2);
}

// The 4-wide tree of the static part (wide.cu): collapse the binary tree of
// n_bnodes internal nodes (root 0) into out (7 float4 a node: the four
// children's boxes as lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, then int32 refs:
// >= 0 a wide node, < 0 ~(triangle slot), kWideEmpty none); *depth receives
// the tree depth.  Returns the number of wide nodes, or -1 on a malformed tree.
int collapse_wide4(const BNode* bn, int n_bnodes, std::vector<float4>& out, int* depth);

size_t bvh_scratch_bytes(int nt);
size_t radix_hist_entries(int n);
cudaError_t scan_exclusive_u32(uint32_t* a, int n, uint32_t* part, cudaStream_t s);
cudaError_t radix_sort_pairs(uint64_t* const keys[2], uint32_t* const vals[2], uint32_t* hist, int n, int bits,
                             cudaStream_t s, int* cur_out, uint32_t* part = nullptr);
size_t carve_bvh_scratch(void* base, int nt, BvhBufs& B);
size_t ploc_scratch_bytes(int nt);
size_t carve_ploc_scratch(void* base, int nt, PlocBufs& Q);
cudaError_t build_lbvh(const BvhBufs& B, const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err,
                       cudaStream_t s, int* root_leaf, const int* list = nullptr);
cudaError_t build_ploc(const BvhBufs& B, const PlocBufs& Q, const float* d_verts, const int* d_idx, int nv, int nt,
                       float eps, int* err, cudaStream_t s, int* root_leaf, const int* list = nullptr);
cudaError_t split_static_moving(const int* d_idx, const uint8_t* vmoved, int nt, int nv, const PlocBufs& Q,
                                int* slist, int* dlist, int* ns, int* nd, cudaStream_t s);
cudaError_t fill_tri_orig(const float* d_verts, const int* d_idx, const int* list, int nv, int nt, float4* tri_orig,
                          cudaStream_t s);
// add node_off to the internal-node references and tri_off to the triangle
// slots of n_nodes nodes (a tree built on its own, placed after another)
cudaError_t relocate_nodes(BNode* nodes, int n_nodes, int node_off, int tri_off, cudaStream_t s);

// A BVH owned by a volume (static part: PLOC; moving part: linear BVH).
struct Bvh {
    int n_tris = 0;
    int root_leaf = -1;
    float4* tri_v = nullptr;  // [3*n] BVH order, v0.w = original index
    BNode* nodes = nullptr;   // [n-1]
    void* scratch = nullptr;
    void* pscratch = nullptr;
    BvhBufs bufs;
    PlocBufs pbufs;
    int cap_ = 0;
    size_t bytes_ = 0;

    cudaError_t reserve(int nt, bool ploc);
    // build into the own tri_v / nodes, or into tri_out / nodes_out when given
    cudaError_t build(const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err, cudaStream_t s,
                      const int* list, bool ploc, float4* tri_out = nullptr, BNode* nodes_out = nullptr);
    void release();
    size_t bytes() const;
};

}  // namespace adgi
