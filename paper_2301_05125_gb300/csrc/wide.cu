// wide.cu -- 4-wide BVH of the static part of the scene, collapsed on the
// host from the binary PLOC tree (sm_103a library, host code).
//
// Each wide node holds up to four children taken from the binary tree: the
// two children of a binary node, then, while fewer than four and an internal
// one is left, the internal child with the largest surface area is replaced by
// its two children.  The child boxes are the binary tree's own boxes (already
// enlarged by the builder), so every triangle stays inside every box on its
// path and a traversal finds exactly the hits the binary tree finds.
//
// Node layout (7 x 16 bytes, children in slots 0..3):
//   [0] lo.x of the four children   [1] hi.x
//   [2] lo.y                        [3] hi.y
//   [4] lo.z                        [5] hi.z
//   [6] int32 refs: >= 0 a wide node, < 0 ~(triangle slot), kWideEmpty none
// An empty slot has the box [+inf, -inf]: whatever the ray direction, its
// entry distance is +inf, so it never reports a hit.  A traversal reads the
// near and far plane arrays of each axis by the sign of the ray direction
// (lo is near for a positive direction), so it needs no per-child min / max.
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "bvh.cuh"

namespace adgi {

namespace {

struct Cand {
    int ref;
    float lo[3], hi[3];
};

inline float area(const Cand& c)
{
    const float dx = c.hi[0] - c.lo[0], dy = c.hi[1] - c.lo[1], dz = c.hi[2] - c.lo[2];
    return dx * dy + dy * dz + dz * dx;
}

inline void children_of(const BNode& n, Cand out[2])
{
    out[0].ref = n.d.x;
    out[0].lo[0] = n.a.x, out[0].lo[1] = n.a.y, out[0].lo[2] = n.a.z;
    out[0].hi[0] = n.a.w, out[0].hi[1] = n.b.x, out[0].hi[2] = n.b.y;
    out[1].ref = n.d.y;
    out[1].lo[0] = n.b.z, out[1].lo[1] = n.b.w, out[1].lo[2] = n.c.x;
    out[1].hi[0] = n.c.y, out[1].hi[1] = n.c.z, out[1].hi[2] = n.c.w;
}

}  // namespace

int collapse_wide4(const BNode* bn, int n_bnodes, std::vector<float4>& out, int* depth_out)
{
    out.clear();
    *depth_out = 0;
    if (n_bnodes < 1) return 0;
    struct Item {
        int bnode, depth;
    };
    std::vector<Item> queue;
    queue.push_back({0, 1});
    size_t head = 0;
    const float inf = std::numeric_limits<float>::infinity();
    while (head < queue.size()) {
        const Item it = queue[head];
        const int w = (int)head++;
        if (it.bnode < 0 || it.bnode >= n_bnodes) return -1;
        Cand c[4];
        children_of(bn[it.bnode], c);
        int n = 2;
        while (n < 4) {
            int best = -1;
            float ba = -1.0f;
            for (int k = 0; k < n; ++k)
                if (c[k].ref >= 0 && area(c[k]) > ba) {
                    ba = area(c[k]);
                    best = k;
                }
            if (best < 0) break;
            if (c[best].ref >= n_bnodes) return -1;
            Cand two[2];
            children_of(bn[c[best].ref], two);
            c[best] = two[0];
            c[n++] = two[1];
        }
        float4 box[6];
        int4 ref;
        int* r = &ref.x;
        for (int k = 0; k < 4; ++k) {
            float* lx = &box[0].x + k;
            float* hx = &box[1].x + k;
            float* ly = &box[2].x + k;
            float* hy = &box[3].x + k;
            float* lz = &box[4].x + k;
            float* hz = &box[5].x + k;
            if (k < n) {
                *lx = c[k].lo[0], *hx = c[k].hi[0], *ly = c[k].lo[1], *hy = c[k].hi[1], *lz = c[k].lo[2],
                *hz = c[k].hi[2];
                if (c[k].ref >= 0) {  // an internal child becomes the next wide node in breadth-first order
                    r[k] = (int)queue.size();
                    queue.push_back({c[k].ref, it.depth + 1});
                } else {
                    r[k] = c[k].ref;
                }
            } else {
                *lx = *ly = *lz = inf;
                *hx = *hy = *hz = -inf;
                r[k] = kWideEmpty;
            }
        }
        if (it.depth > *depth_out) *depth_out = it.depth;
        (void)w;
        for (int j = 0; j < 6; ++j) out.push_back(box[j]);
        float4 rf;
        std::memcpy(&rf, &ref, sizeof(rf));
        out.push_back(rf);
    }
    return (int)queue.size();
}

}  // namespace adgi
