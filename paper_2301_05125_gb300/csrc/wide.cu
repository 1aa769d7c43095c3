// wide.cu -- 4-wide BVH of the static part of the scene, collapsed on the
// host from the binary PLOC tree (sm_103a library, host code).
//
// Each wide node holds up to four children: a cut of its binary subtree into
// at most four nodes.  The cuts minimise the surface-area cost of the whole
// wide tree (below), found bottom up by dynamic programming over the binary
// tree.  The child boxes are the binary tree's own boxes (already enlarged by
// the builder), so every triangle stays inside every box on its path and a
// traversal finds exactly the hits the binary tree finds.
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
    int ref;  // >= 0 a binary node, < 0 ~(triangle slot)
    float lo[3], hi[3];
};

inline double area(const Cand& c)
{
    const double dx = (double)c.hi[0] - c.lo[0], dy = (double)c.hi[1] - c.lo[1], dz = (double)c.hi[2] - c.lo[2];
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

// Surface-area cost of a wide tree: a ray enters a box with a chance in
// proportion to its surface area, a visit of a wide node costs kCostNode and
// a triangle test kCostTri.  A wide node made at binary node u costs
// kCostNode A(u) plus the cost of its children; a triangle child costs
// kCostTri times its own box's area.  The weights are lane operations of the
// traversal: a visit tests four boxes (13 each) and spends about 20 more on
// ordering the hits and on the stack; a watertight triangle test takes 55.
constexpr double kCostNode = 72.0, kCostTri = 55.0;

// The dynamic programme.  For binary node v and a budget of k slots (1..4):
//   F(v, k) = least cost of covering v's subtree with at most k children of
//             the wide node above it;
//   F(v, 1) = cost of v as one child (a wide node of its own made at v);
//   F(v, k) = min(F(v, 1), min over a of F(l, a) + F(r, k - a)), k >= 2,
// where l, r are v's binary children (a triangle costs the same in any
// budget).  The wide node made at v takes the best cut of v into four:
//   S(v) = min over a in 1..3 of F(l, a) + F(r, 4 - a).
struct CutPlan {
    std::vector<double> F;         // [4 n]: F(v, k) at 4 v + k - 1 (k = 4 unused)
    std::vector<signed char> cut;  // [4 n]: a of the best split at budget k; 0: keep v whole
};

inline double cost_of(const CutPlan& P, const Cand& c, int k)
{
    return c.ref < 0 ? kCostTri * area(c) : P.F[4 * (size_t)c.ref + (k - 1)];
}

// best split of binary node v (children c) into budget k >= 2
inline double best_split(const CutPlan& P, const Cand c[2], int k, int* a_out)
{
    double best = std::numeric_limits<double>::infinity();
    int arg = 1;
    for (int a = 1; a < k; ++a) {
        const double x = cost_of(P, c[0], a) + cost_of(P, c[1], k - a);
        if (x < best) {
            best = x;
            arg = a;
        }
    }
    *a_out = arg;
    return best;
}

// Returns false on a malformed tree (a child index out of range or a node
// reached twice).
bool plan_cuts(const BNode* bn, int n, CutPlan& P)
{
    P.F.assign(4 * (size_t)n, 0.0);
    P.cut.assign(4 * (size_t)n, 0);
    // a pre-order list; walked backwards it visits children before parents
    std::vector<int> order;
    std::vector<char> seen((size_t)n, 0);
    order.reserve(n);
    std::vector<int> st{0};
    while (!st.empty()) {
        const int v = st.back();
        st.pop_back();
        if (v >= n || seen[v]) return false;
        seen[v] = 1;
        order.push_back(v);
        if (bn[v].d.x >= 0) st.push_back(bn[v].d.x);
        if (bn[v].d.y >= 0) st.push_back(bn[v].d.y);
    }
    for (size_t i = order.size(); i-- > 0;) {
        const int v = order[i];
        Cand c[2];
        children_of(bn[v], c);
        Cand u;
        for (int j = 0; j < 3; ++j) {
            u.lo[j] = std::min(c[0].lo[j], c[1].lo[j]);
            u.hi[j] = std::max(c[0].hi[j], c[1].hi[j]);
        }
        int a4 = 1;
        const double whole = kCostNode * area(u) + best_split(P, c, 4, &a4);
        double* F = &P.F[4 * (size_t)v];
        signed char* cut = &P.cut[4 * (size_t)v];
        F[0] = whole;
        cut[0] = 0;
        for (int k = 2; k <= 3; ++k) {
            int a = 1;
            const double s = best_split(P, c, k, &a);
            F[k - 1] = s < whole ? s : whole;
            cut[k - 1] = s < whole ? (signed char)a : 0;
        }
        F[3] = F[2];  // no child of a wide node gets four slots
        cut[3] = (signed char)a4;  // the split of v's own wide node
    }
    return true;
}

// the slots of budget k that cover c (c an internal node cut at budget k,
// or kept whole)
void emit_cut(const BNode* bn, const CutPlan& P, const Cand& c, int k, Cand* out, int& n_out)
{
    const int a = c.ref < 0 ? 0 : P.cut[4 * (size_t)c.ref + (k - 1)];
    if (a == 0) {
        out[n_out++] = c;
        return;
    }
    Cand two[2];
    children_of(bn[c.ref], two);
    emit_cut(bn, P, two[0], a, out, n_out);
    emit_cut(bn, P, two[1], k - a, out, n_out);
}

}  // namespace

int collapse_wide4(const BNode* bn, int n_bnodes, std::vector<float4>& out, int* depth_out)
{
    out.clear();
    *depth_out = 0;
    if (n_bnodes < 1) return 0;
    CutPlan P;
    if (!plan_cuts(bn, n_bnodes, P)) return -1;
    struct Item {
        int bnode, depth;
    };
    std::vector<Item> queue;
    queue.push_back({0, 1});
    size_t head = 0;
    const float inf = std::numeric_limits<float>::infinity();
    while (head < queue.size()) {
        const Item it = queue[head++];
        Cand two[2], c[4];
        children_of(bn[it.bnode], two);
        const int a = P.cut[4 * (size_t)it.bnode + 3];
        int n = 0;
        emit_cut(bn, P, two[0], a, c, n);
        emit_cut(bn, P, two[1], 4 - a, c, n);
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
        for (int j = 0; j < 6; ++j) out.push_back(box[j]);
        float4 rf;
        std::memcpy(&rf, &ref, sizeof(rf));
        out.push_back(rf);
    }
    return (int)queue.size();
}

}  // namespace adgi
