// bvh.cu -- software BVH for the probe rays (the paper traces with DXR on RT
// cores, Sec. 5; here a linear BVH is built on the device every time the
// geometry moves).
//
// Build: centroid bounds -> 63-bit Morton codes -> stable LSD radix sort
// (8 passes of 8 bits, own kernels) -> Karras (HPG 2012) radix-tree hierarchy
// -> bottom-up child boxes, each leaf box enlarged by eps so that box tests
// stay conservative for the watertight triangle test.
#include <algorithm>
#include <cstdio>

#include "adgi_internal.cuh"
#include "bvh.cuh"
#include "kernels.cuh"
#include "bvhbody.cuh"

namespace adgi {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
static_assert(kSortTile == kBvhSortTile, "the scratch layout in bvh.cuh counts histograms per radix tile");



__global__ void k_init_bounds(uint32_t* __restrict__ bounds)
{
    if (threadIdx.x < 3) bounds[threadIdx.x] = 0xFFFFFFFFu;
    else if (threadIdx.x < 6) bounds[threadIdx.x] = 0u;
}


__global__ void k_tri_prep(const float* __restrict__ verts, const int* __restrict__ idx, const int* __restrict__ list,
                           int nt, int nv, float4* __restrict__ tri_in, uint32_t* __restrict__ bounds,
                           int* __restrict__ err)
{
    __shared__ uint32_t s_lo[3], s_hi[3];
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = 0xFFFFFFFFu;
        s_hi[threadIdx.x] = 0u;
    }
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) tri_fetch(verts, idx, list, nv, i, tri_in, s_lo, s_hi, err);
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&bounds[threadIdx.x], s_lo[threadIdx.x]);
        atomicMax(&bounds[3 + threadIdx.x], s_hi[threadIdx.x]);
    }
}




// vertices of the listed triangles into an original-order array (shading)
__global__ void k_fill_orig(const float* __restrict__ verts, const int* __restrict__ idx, const int* __restrict__ list,
                            int nt, int nv, float4* __restrict__ tri_orig)
{
    fill_orig_body(verts, idx, list, nt, nv, tri_orig, blockIdx.x * blockDim.x + threadIdx.x);
}

constexpr int kSmallThreads = 1024;

__global__ void __launch_bounds__(kSmallThreads) k_morton_small(const float* __restrict__ verts,
                                                                const int* __restrict__ idx,
                                                                const int* __restrict__ list, int nt, int nv,
                                                                float4* __restrict__ tri_in, uint64_t* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                float4* __restrict__ tri_v, int* __restrict__ err)
{
    __shared__ uint64_t sk[kSmallBuild];
    __shared__ uint32_t sv[kSmallBuild];
    morton_small_body(verts, idx, list, nt, nv, tri_in, keys, vals, tri_v, err, sk, sv);
}

__global__ void k_hierarchy(const uint64_t* __restrict__ keys, int n, BNode* __restrict__ nodes,
                            int* __restrict__ par_int, int* __restrict__ par_leaf)
{
    hierarchy_body(keys, n, nodes, par_int, par_leaf, blockIdx.x * blockDim.x + threadIdx.x, 0, 0);
}

__global__ void k_bounds(const float4* __restrict__ tri_v, int n, BNode* nodes, const int* __restrict__ par_int,
                         const int* __restrict__ par_leaf, int* flags, float eps, int* err)
{
    bounds_body(tri_v, n, nodes, par_int, par_leaf, flags, eps, err, blockIdx.x * blockDim.x + threadIdx.x, 0, 0);
}

__global__ void k_morton(const float4* __restrict__ tri_in, int nt, const uint32_t* __restrict__ bounds,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    keys[t] = morton_key(tri_in[3 * (size_t)t], tri_in[3 * (size_t)t + 1], tri_in[3 * (size_t)t + 2], bounds);
    vals[t] = (uint32_t)t;
}

__global__ void k_hist(const uint64_t* __restrict__ keys, int n, int shift, uint32_t* __restrict__ hist, int nblocks)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        int i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of a small array in one block of 1024 threads
__global__ void k_scan_small(uint32_t* __restrict__ a, int n)
{
    __shared__ uint32_t part[1024];
    int tid = threadIdx.x;
    int per = (n + 1023) / 1024;
    int s0 = tid * per, s1 = min(n, s0 + per);
    uint32_t sum = 0;
    for (int i = s0; i < s1; ++i) sum += a[i];
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = tid >= off ? part[tid - off] : 0u;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint32_t run = part[tid] - sum;
    for (int i = s0; i < s1; ++i) {
        uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Exclusive scan of a large array in three launches: per-chunk sums, a scan
// of the (at most 1024) sums, and a scan of each chunk from its carry.
constexpr int kScanChunks = 1024;

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* __restrict__ a, int n, int per,
                                                     uint32_t* __restrict__ part)
{
    __shared__ uint32_t red[8];
    const int b0 = blockIdx.x * per, b1 = min(n, b0 + per);
    uint32_t s = 0;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += a[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_scan_apply(uint32_t* __restrict__ a, int n, int per,
                                                    const uint32_t* __restrict__ part)
{
    __shared__ uint32_t wsum[8];
    const int b0 = blockIdx.x * per, b1 = min(n, b0 + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t carry = part[blockIdx.x];
    for (int t0 = b0; t0 < b1; t0 += 4 * (int)blockDim.x) {  // tiles of 4 items per thread
        const int i0 = t0 + 4 * (int)threadIdx.x;
        uint32_t v[4], tot = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = i0 + k < b1 ? a[i0 + k] : 0u;
            tot += v[k];
        }
        uint32_t x = tot;  // inclusive scan of the thread totals in the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t before = carry, all = 0;
        for (int w = 0; w < nw; ++w) {
            const uint32_t ws = wsum[w];
            if (w < warp) before += ws;
            all += ws;
        }
        before += x - tot;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < b1) a[i0 + k] = before;
            before += v[k];
        }
        carry += all;
        __syncthreads();
    }
}

__global__ void k_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int n, int shift,
                          const uint32_t* __restrict__ hist, int nblocks)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = hist[(size_t)tid * nblocks + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        for (int i = tid; i < (kSortThreads / 32) * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0u;
        __syncthreads();
        int idx = blockIdx.x * kSortTile + r * kSortThreads + tid;
        bool valid = idx < n;
        uint64_t k = valid ? kin[idx] : 0ull;
        uint32_t v = valid ? vin[idx] : 0u;
        uint32_t dig = valid ? ((uint32_t)(k >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) {
            uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = base[dig] + wcnt[warp][dig] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        base[tid] += run;
        __syncthreads();
    }
}

__global__ void k_tri_order(const float4* __restrict__ tri_in, const uint32_t* __restrict__ order, int nt,
                            float4* __restrict__ tri_v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    uint32_t t = order[i];
    tri_v[3 * (size_t)i] = tri_in[3 * (size_t)t];
    tri_v[3 * (size_t)i + 1] = tri_in[3 * (size_t)t + 1];
    tri_v[3 * (size_t)i + 2] = tri_in[3 * (size_t)t + 2];
}






// ---------------------------------------------------------------- PLOC
// Parallel locally-ordered clustering (Meister & Bittner, TVCG 2018): clusters
// in Morton order; each finds its nearest neighbour by the surface area of the
// merged box within +-kPlocR positions; mutual nearest neighbours merge into a
// new node; the cluster array is compacted; repeat until one cluster is left.
// A wide window finds better partners: on a 198k-triangle city, radius 256
// against 16 cut the traversals' box tests by a fifth (update 7.18 -> 6.25 ms)
// for a static build of 7 instead of 4 ms.  With the 4-wide traversal, the
// updates of the 2M- and 198k-triangle scenes took 18.56 / 5.12 ms at radius
// 256, 18.24 / 4.94 at 512, 17.19 / 4.92 at 1024, 17.16 / 4.71 at 1536 and
// 16.90 / 4.97 at 2048 (the static build of the 2M triangles: ~0.1 s).
constexpr int kPlocR = 1536;
constexpr int kRotPasses = 8;  // rotation passes after the clustering
constexpr int kPlocT = 256;

__device__ __forceinline__ float box_area(float4 lo, float4 hi)
{
    float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return 2.0f * (dx * dy + dy * dz + dz * dx);
}

__global__ void k_ploc_init(const float4* __restrict__ tri_v, int n, float eps, int* __restrict__ cid,
                            float4* __restrict__ blo, float4* __restrict__ bhi)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 A = tri_v[3 * (size_t)i], B = tri_v[3 * (size_t)i + 1], C = tri_v[3 * (size_t)i + 2];
    eps = tri_eps(eps, A, B, C);
    blo[i] = make_float4(fminf(fminf(A.x, B.x), C.x) - eps, fminf(fminf(A.y, B.y), C.y) - eps,
                         fminf(fminf(A.z, B.z), C.z) - eps, 0.f);
    bhi[i] = make_float4(fmaxf(fmaxf(A.x, B.x), C.x) + eps, fmaxf(fmaxf(A.y, B.y), C.y) + eps,
                         fmaxf(fmaxf(A.z, B.z), C.z) + eps, 0.f);
    cid[i] = ~i;
}

constexpr int kPlocWin = kPlocT + 2 * kPlocR;  // boxes of a block's window
constexpr size_t kPlocSmem = 2 * sizeof(float4) * kPlocWin;

__global__ void __launch_bounds__(kPlocT) k_ploc_nn(int count, const float4* __restrict__ blo,
                                                    const float4* __restrict__ bhi, int* __restrict__ nn)
{
    extern __shared__ float4 ploc_smem[];
    float4* slo = ploc_smem;
    float4* shi = ploc_smem + kPlocWin;
    const int base = blockIdx.x * kPlocT - kPlocR;
    for (int k = threadIdx.x; k < kPlocT + 2 * kPlocR; k += kPlocT) {
        int j = base + k;
        if (j >= 0 && j < count) {
            slo[k] = blo[j];
            shi[k] = bhi[j];
        }
    }
    __syncthreads();
    const int i = blockIdx.x * kPlocT + threadIdx.x;
    if (i >= count) return;
    const int me = threadIdx.x + kPlocR;
    float4 lo = slo[me], hi = shi[me];
    float best = __int_as_float(0x7F800000);
    int bj = i;
    for (int k = -kPlocR; k <= kPlocR; ++k) {
        int j = i + k;
        if (k == 0 || j < 0 || j >= count) continue;
        float4 l2 = slo[me + k], h2 = shi[me + k];
        float a = box_area(make_float4(fminf(lo.x, l2.x), fminf(lo.y, l2.y), fminf(lo.z, l2.z), 0.f),
                           make_float4(fmaxf(hi.x, h2.x), fmaxf(hi.y, h2.y), fmaxf(hi.z, h2.z), 0.f));
        if (a < best) {  // scanning j upwards: ties keep the smaller index
            best = a;
            bj = j;
        }
    }
    nn[i] = bj;
}

// flags of cluster i packed for one scan: keep (high word), creates a node (low word)
__global__ void k_ploc_flags(int count, const int* __restrict__ nn, uint64_t* __restrict__ fl)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int j = nn[i];
    bool mutual = j != i && nn[j] == i;
    uint64_t keep = !(mutual && j < i);
    uint64_t mrg = mutual && i < j;
    fl[i] = (keep << 32) | mrg;
}

__global__ void k_ploc_merge(int count, const int* __restrict__ nn, const uint64_t* __restrict__ pre,
                             const int* __restrict__ cid, const float4* __restrict__ blo,
                             const float4* __restrict__ bhi, int node_top, int* __restrict__ cid2,
                             float4* __restrict__ blo2, float4* __restrict__ bhi2, BNode* __restrict__ nodes,
                             int* __restrict__ par_int, int* __restrict__ par_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int j = nn[i];
    bool mutual = j != i && nn[j] == i;
    if (mutual && j < i) return;  // merged into cluster j
    uint64_t p = pre[i];
    int pos = (int)(p >> 32);
    if (mutual) {
        int node = node_top - 1 - (int)(p & 0xFFFFFFFFu);
        float4 la = blo[i], ha = bhi[i], lb = blo[j], hb = bhi[j];
        BNode b;
        b.a = make_float4(la.x, la.y, la.z, ha.x);
        b.b = make_float4(ha.y, ha.z, lb.x, lb.y);
        b.c = make_float4(lb.z, hb.x, hb.y, hb.z);
        b.d = make_int4(cid[i], cid[j], 0, 0);
        nodes[node] = b;
        for (int c2 : {cid[i], cid[j]}) {
            if (c2 < 0)
                par_leaf[~c2] = node;
            else
                par_int[c2] = node;
        }
        cid2[pos] = node;
        blo2[pos] = make_float4(fminf(la.x, lb.x), fminf(la.y, lb.y), fminf(la.z, lb.z), 0.f);
        bhi2[pos] = make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y), fmaxf(ha.z, hb.z), 0.f);
    } else {
        cid2[pos] = cid[i];
        blo2[pos] = blo[i];
        bhi2[pos] = bhi[i];
    }
}

// ---------------------------------------------------------------- rotations
// Local tree rotations (Kensler, "Tree Rotations for Improving Bounding
// Volume Hierarchies", 2008) after the PLOC build: node N may swap one child
// with a grandchild under its other child C when that shrinks C's box, or a
// grandchild under one child with one under the other when that shrinks the
// two children's boxes together (every other box keeps its leaf set).  A
// pass treats the internal nodes of one depth parity: a rotation writes only
// N and its children, so no two rotations of a pass touch the same node.
// Hits do not depend on the tree's shape.

// depth of internal node i below the root (node 0), bounded walk
__global__ void k_node_depth(int n_int, const int* __restrict__ par_int, int* __restrict__ depth)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int d = 0, x = i;
    while (x != 0 && d < 4096) {
        x = par_int[x];
        ++d;
    }
    depth[i] = d;
}

__device__ __forceinline__ void child_box(const BNode& n, int k, float4& lo, float4& hi)
{
    if (k == 0) {
        lo = make_float4(n.a.x, n.a.y, n.a.z, 0.f);
        hi = make_float4(n.a.w, n.b.x, n.b.y, 0.f);
    } else {
        lo = make_float4(n.b.z, n.b.w, n.c.x, 0.f);
        hi = make_float4(n.c.y, n.c.z, n.c.w, 0.f);
    }
}

__device__ __forceinline__ BNode make_node(float4 lo0, float4 hi0, float4 lo1, float4 hi1, int c0, int c1)
{
    BNode b;
    b.a = make_float4(lo0.x, lo0.y, lo0.z, hi0.x);
    b.b = make_float4(hi0.y, hi0.z, lo1.x, lo1.y);
    b.c = make_float4(lo1.z, hi1.x, hi1.y, hi1.z);
    b.d = make_int4(c0, c1, 0, 0);
    return b;
}

__device__ __forceinline__ float4 fmin4(float4 a, float4 b)
{
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.f);
}
__device__ __forceinline__ float4 fmax4(float4 a, float4 b)
{
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), 0.f);
}

__device__ __forceinline__ void set_parent(int ref, int parent, int* par_int, int* par_leaf)
{
    if (ref >= 0)
        par_int[ref] = parent;
    else
        par_leaf[~ref] = parent;
}

__global__ void k_rotate(int n_int, BNode* __restrict__ nodes, const int* __restrict__ depth, int parity,
                         int* __restrict__ par_int, int* __restrict__ par_leaf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || (depth[i] & 1) != parity) return;
    const BNode N = nodes[i];
    const int ch[2] = {N.d.x, N.d.y};
    float4 lo[2], hi[2], glo[2][2], ghi[2][2];
    child_box(N, 0, lo[0], hi[0]);
    child_box(N, 1, lo[1], hi[1]);
    BNode C[2];
    float cur[2];
    for (int k = 0; k < 2; ++k) {
        cur[k] = box_area(lo[k], hi[k]);
        if (ch[k] < 0) continue;
        C[k] = nodes[ch[k]];
        child_box(C[k], 0, glo[k][0], ghi[k][0]);
        child_box(C[k], 1, glo[k][1], ghi[k][1]);
    }
    // (a) child s swaps with grandchild g under the other child o: o's box
    //     becomes child s + grandchild 1-g;
    // (b) grandchild a under child 0 swaps with grandchild b under child 1:
    //     both children's boxes change
    float best = 0.0f;
    int kind = -1, bs = 0, bg = 0;
    for (int s = 0; s < 2; ++s) {
        const int o = 1 - s;
        if (ch[o] < 0) continue;
        for (int g = 0; g < 2; ++g) {
            const float gain = cur[o] - box_area(fmin4(lo[s], glo[o][1 - g]), fmax4(hi[s], ghi[o][1 - g]));
            if (gain > best && gain > 1e-6f * cur[o]) best = gain, kind = 0, bs = s, bg = g;
        }
    }
    if (ch[0] >= 0 && ch[1] >= 0)
        for (int ga = 0; ga < 2; ++ga)
            for (int gb = 0; gb < 2; ++gb) {
                const float a0 = box_area(fmin4(glo[0][1 - ga], glo[1][gb]), fmax4(ghi[0][1 - ga], ghi[1][gb]));
                const float a1 = box_area(fmin4(glo[1][1 - gb], glo[0][ga]), fmax4(ghi[1][1 - gb], ghi[0][ga]));
                const float gain = (cur[0] + cur[1]) - (a0 + a1);
                if (gain > best && gain > 1e-6f * (cur[0] + cur[1])) best = gain, kind = 1, bs = ga, bg = gb;
            }
    if (kind == 0) {
        const int s = bs, o = 1 - s, g = bg;
        // C keeps child 1-g and takes N's child s; N takes grandchild g in place of child s
        const int cref = ch[o], gref = g ? C[o].d.y : C[o].d.x, kref = g ? C[o].d.x : C[o].d.y;
        const float4 clo = fmin4(lo[s], glo[o][1 - g]), chi = fmax4(hi[s], ghi[o][1 - g]);
        nodes[cref] = make_node(lo[s], hi[s], glo[o][1 - g], ghi[o][1 - g], ch[s], kref);
        nodes[i] = s == 0 ? make_node(glo[o][g], ghi[o][g], clo, chi, gref, cref)
                          : make_node(clo, chi, glo[o][g], ghi[o][g], cref, gref);
        set_parent(ch[s], cref, par_int, par_leaf);
        set_parent(gref, i, par_int, par_leaf);
    } else if (kind == 1) {
        const int ga = bs, gb = bg;
        const int r0 = ga ? C[0].d.y : C[0].d.x, k0 = ga ? C[0].d.x : C[0].d.y;  // moves / stays under child 0
        const int r1 = gb ? C[1].d.y : C[1].d.x, k1 = gb ? C[1].d.x : C[1].d.y;  // moves / stays under child 1
        nodes[ch[0]] = make_node(glo[0][1 - ga], ghi[0][1 - ga], glo[1][gb], ghi[1][gb], k0, r1);
        nodes[ch[1]] = make_node(glo[1][1 - gb], ghi[1][1 - gb], glo[0][ga], ghi[0][ga], k1, r0);
        nodes[i] = make_node(fmin4(glo[0][1 - ga], glo[1][gb]), fmax4(ghi[0][1 - ga], ghi[1][gb]),
                             fmin4(glo[1][1 - gb], glo[0][ga]), fmax4(ghi[1][1 - gb], ghi[0][ga]), ch[0], ch[1]);
        set_parent(r1, ch[0], par_int, par_leaf);
        set_parent(r0, ch[1], par_int, par_leaf);
    }
}

// depth of every leaf below the root (node 0), bounded walk; max into *depth
__global__ void k_leaf_depth(int n, const int* __restrict__ par_int, const int* __restrict__ par_leaf,
                             int* __restrict__ depth)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = 1, x = par_leaf[i];
    while (x != 0 && d < 4096) {
        x = par_int[x];
        ++d;
    }
    atomicMax(depth, d);
}

// ---------------------------------------------------------------- 64-bit scan
// exclusive scan in three phases: per-block scans of 1024 values, a scan of
// the block totals (one block), and the add-back.
constexpr int kScanT = 256, kScanItems = 4, kScanBlock = kScanT * kScanItems;

__global__ void __launch_bounds__(kScanT) k_scan64_block(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                         uint64_t* __restrict__ sums, int n)
{
    __shared__ uint64_t wsum[kScanT / 32];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    uint64_t v[kScanItems], run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0ull;
        run += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint64_t wbase = 0;
    for (int k = 0; k < w; ++k) wbase += wsum[k];
    uint64_t pre = wbase + x - run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == kScanT - 1) sums[blockIdx.x] = wbase + x;
}

__global__ void k_scan64_small(uint64_t* __restrict__ a, int n, uint64_t* __restrict__ total)
{
    __shared__ uint64_t part[1024];
    int tid = threadIdx.x;
    int per = (n + 1023) / 1024;
    int s0 = tid * per, s1 = min(n, s0 + per);
    uint64_t sum = 0;
    for (int i = s0; i < s1; ++i) sum += a[i];
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint64_t v = tid >= off ? part[tid - off] : 0ull;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint64_t run = part[tid] - sum;
    for (int i = s0; i < s1; ++i) {
        uint64_t v = a[i];
        a[i] = run;
        run += v;
    }
    if (tid == 1023) *total = part[1023];
}

__global__ void k_scan64_add(uint64_t* __restrict__ out, const uint64_t* __restrict__ sums, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanBlock];
}

}  // namespace

size_t Bvh::bytes() const { return bytes_; }

size_t bvh_scratch_bytes(int nt)
{
    BvhBufs B;
    return carve_bvh_scratch(nullptr, nt, B);
}

// Carve the scratch buffers of a linear build for nt triangles out of one
// block (base may be null to only compute the size); every piece 256-byte
// aligned.
size_t carve_bvh_scratch(void* base, int nt, BvhBufs& B)
{
    const size_t n = (size_t)(nt > 0 ? nt : 1);
    const size_t nb = (n + kSortTile - 1) / kSortTile;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* p = base ? (void*)((char*)base + off) : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    B.tri_in = (float4*)take(sizeof(float4) * 3 * n);
    B.par_int = (int*)take(sizeof(int) * n);
    B.par_leaf = (int*)take(sizeof(int) * n);
    B.flags = (int*)take(sizeof(int) * n);
    B.keys[0] = (uint64_t*)take(sizeof(uint64_t) * n);
    B.keys[1] = (uint64_t*)take(sizeof(uint64_t) * n);
    B.vals[0] = (uint32_t*)take(sizeof(uint32_t) * n);
    B.vals[1] = (uint32_t*)take(sizeof(uint32_t) * n);
    B.hist = (uint32_t*)take(sizeof(uint32_t) * 256 * nb);
    B.bounds = (uint32_t*)take(sizeof(uint32_t) * 8);
    B.err = (int*)take(sizeof(int) * 2);
    return off;  // == bvh_scratch_layout_bytes(nt), the same pieces in the same order
}

size_t radix_hist_entries(int n) { return 256 * (size_t)((std::max(n, 1) + kSortTile - 1) / kSortTile); }

// Stable LSD radix sort of n (key, value) pairs on key bits [0, bits), eight
// bits per pass (hist -> scan -> scatter); the result is in keys[*cur],
// vals[*cur].  hist holds radix_hist_entries(n) counters; part (optional,
// 1024 entries) lets large histograms use the three-launch scan.
cudaError_t radix_sort_pairs(uint64_t* const keys[2], uint32_t* const vals[2], uint32_t* hist, int n, int bits,
                             cudaStream_t s, int* cur_out, uint32_t* part)
{
    int cur = 0;
    if (n > 0) {
        const int nb = (n + kSortTile - 1) / kSortTile;
        const int nh = 256 * nb;
        // large histograms (and a partial-sum buffer): the three-launch scan
        const int G = std::min(kScanChunks, (nh + 1023) / 1024), per = (nh + G - 1) / G;
        const bool big = part != nullptr && nh > 65536;
        for (int shift = 0; shift < bits; shift += 8) {
            k_hist<<<nb, kSortThreads, 0, s>>>(keys[cur], n, shift, hist, nb);
            count_launches(1);
            if (big) {
                k_scan_reduce<<<G, 256, 0, s>>>(hist, nh, per, part);
                k_scan_small<<<1, 1024, 0, s>>>(part, G);
                k_scan_apply<<<G, 256, 0, s>>>(hist, nh, per, part);
                count_launches(3);
            } else {
                k_scan_small<<<1, 1024, 0, s>>>(hist, nh);
                count_launches(1);
            }
            k_scatter<<<nb, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, shift, hist,
                                                   nb);
            count_launches(1);
            cur ^= 1;
        }
    }
    *cur_out = cur;
    return cudaGetLastError();
}

// Exclusive scan of a[0..n) in place: one block for small arrays, the
// three-launch scan (part: 1024 partial sums) for large ones.
cudaError_t scan_exclusive_u32(uint32_t* a, int n, uint32_t* part, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (part != nullptr && n > 65536) {
        const int G = std::min(kScanChunks, (n + 1023) / 1024), per = (n + G - 1) / G;
        k_scan_reduce<<<G, 256, 0, s>>>(a, n, per, part);
        k_scan_small<<<1, 1024, 0, s>>>(part, G);
        k_scan_apply<<<G, 256, 0, s>>>(a, n, per, part);
        count_launches(3);
    } else {
        k_scan_small<<<1, 1024, 0, s>>>(a, n);
        count_launches(1);
    }
    return cudaGetLastError();
}

// Morton order of the listed triangles into B.tri_v (all builds start here)
static cudaError_t morton_order(const BvhBufs& B, const float* d_verts, const int* d_idx, const int* list, int nv,
                                int nt, int* err, cudaStream_t s, int* cur_out)
{
    const int T = 256;
    if (nt <= kSmallBuild) {
        k_morton_small<<<1, kSmallThreads, 0, s>>>(d_verts, d_idx, list, nt, nv, B.tri_in, B.keys[0], B.vals[0],
                                                    B.tri_v, err);
        count_launches(1);
        *cur_out = 0;
        return cudaGetLastError();
    }
    k_init_bounds<<<1, 32, 0, s>>>(B.bounds);
    count_launches(1);
    k_tri_prep<<<(nt + T - 1) / T, T, 0, s>>>(d_verts, d_idx, list, nt, nv, B.tri_in, B.bounds, err);
    count_launches(1);
    k_morton<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_in, nt, B.bounds, B.keys[0], B.vals[0]);
    count_launches(1);
    int cur = 0;
    cudaError_t e = radix_sort_pairs(B.keys, B.vals, B.hist, nt, 64, s, &cur);
    if (e != cudaSuccess) return e;
    k_tri_order<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_in, B.vals[cur], nt, B.tri_v);
    count_launches(1);
    *cur_out = cur;
    return cudaGetLastError();
}

// Linear BVH (Karras 2012) of the listed triangles (list = null: all).  Every
// buffer comes from B (scratch) or the outputs B.tri_v / B.nodes; all work is
// ordered on stream s; nothing is allocated.
cudaError_t build_lbvh(const BvhBufs& B, const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err,
                       cudaStream_t s, int* root_leaf, const int* list)
{
    if (nt <= 0) {
        *root_leaf = -1;
        return cudaSuccess;
    }
    const int T = 256;
    int cur = 0;
    cudaError_t e = morton_order(B, d_verts, d_idx, list, nv, nt, err, s, &cur);
    if (e != cudaSuccess) return e;
    if (nt == 1) {
        *root_leaf = 0;
        return cudaGetLastError();
    }
    *root_leaf = -1;
    e = cudaMemsetAsync(B.flags, 0, sizeof(int) * (size_t)nt, s);
    if (e != cudaSuccess) return e;
    k_hierarchy<<<(nt - 1 + T - 1) / T, T, 0, s>>>(B.keys[cur], nt, B.nodes, B.par_int, B.par_leaf);
    count_launches(1);
    k_bounds<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_v, nt, B.nodes, B.par_int, B.par_leaf, B.flags, eps, err);
    count_launches(1);
    return cudaGetLastError();
}

// PLOC build of the listed triangles: Morton order as for the linear BVH,
// then agglomerative clustering.  The host reads the cluster count after each
// round (one synchronisation per round); meant for geometry that changes
// rarely.  Nodes are numbered from the top so that the final merge is node 0.
cudaError_t build_ploc(const BvhBufs& B, const PlocBufs& Q, const float* d_verts, const int* d_idx, int nv, int nt,
                       float eps, int* err, cudaStream_t s, int* root_leaf, const int* list)
{
    if (nt <= 0) {
        *root_leaf = -1;
        return cudaSuccess;
    }
    int cur = 0;
    cudaError_t e = morton_order(B, d_verts, d_idx, list, nv, nt, err, s, &cur);
    if (e != cudaSuccess) return e;
    if (nt == 1) {
        *root_leaf = 0;
        return cudaGetLastError();
    }
    *root_leaf = -1;
    const int T = 256;
    k_ploc_init<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_v, nt, eps, Q.cid[0], Q.blo[0], Q.bhi[0]);
    count_launches(1);
    int count = nt, node_top = nt - 1, c = 0;
    for (int round = 0; count > 1; ++round) {
        if (round > 4 * 64 + nt) return cudaErrorUnknown;  // no progress: cannot happen with strict ties
        const int nb = (count + kPlocT - 1) / kPlocT;
        if (round == 0 && kPlocSmem > 48 * 1024) {  // one constant size: set, never lowered
            cudaError_t e = cudaFuncSetAttribute(k_ploc_nn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlocSmem);
            if (e != cudaSuccess) return e;
        }
        k_ploc_nn<<<nb, kPlocT, kPlocSmem, s>>>(count, Q.blo[c], Q.bhi[c], Q.nn);
        count_launches(1);
        k_ploc_flags<<<nb, kPlocT, 0, s>>>(count, Q.nn, Q.flags);
        count_launches(1);
        const int sb = (count + kScanBlock - 1) / kScanBlock;
        k_scan64_block<<<sb, kScanT, 0, s>>>(Q.flags, Q.pre, Q.sums, count);
        count_launches(1);
        k_scan64_small<<<1, 1024, 0, s>>>(Q.sums, sb, Q.total);
        count_launches(1);
        k_scan64_add<<<(count + T - 1) / T, T, 0, s>>>(Q.pre, Q.sums, count);
        count_launches(1);
        k_ploc_merge<<<nb, kPlocT, 0, s>>>(count, Q.nn, Q.pre, Q.cid[c], Q.blo[c], Q.bhi[c], node_top, Q.cid[c ^ 1],
                                           Q.blo[c ^ 1], Q.bhi[c ^ 1], B.nodes, B.par_int, B.par_leaf);
        count_launches(1);
        uint64_t tot = 0;
        e = cudaMemcpyAsync(&tot, Q.total, sizeof(tot), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        int keeps = (int)(tot >> 32), merges = (int)(tot & 0xFFFFFFFFu);
        if (merges <= 0 || keeps != count - merges) return cudaErrorUnknown;
        count = keeps;
        node_top -= merges;
        c ^= 1;
    }
    if (node_top != 0) return cudaErrorUnknown;
    // rotations: passes over the two depth parities, depths refreshed between
    // passes (a rotation moves subtrees one level up or down)
    for (int pass = 0; pass < kRotPasses; ++pass)
        for (int parity = 0; parity < 2; ++parity) {
            k_node_depth<<<(nt - 1 + T - 1) / T, T, 0, s>>>(nt - 1, B.par_int, Q.nn);
            k_rotate<<<(nt - 1 + T - 1) / T, T, 0, s>>>(nt - 1, B.nodes, Q.nn, parity, B.par_int, B.par_leaf);
            count_launches(2);
        }
    // the traversal stack holds at most depth-1 entries: a deeper tree is
    // replaced by the linear BVH (depth <= 95 by construction)
    e = cudaMemsetAsync(Q.total, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_leaf_depth<<<(nt + T - 1) / T, T, 0, s>>>(nt, B.par_int, B.par_leaf, (int*)Q.total);
    count_launches(1);
    int depth = 0;
    e = cudaMemcpyAsync(&depth, Q.total, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (depth >= kMaxDepth) return build_lbvh(B, d_verts, d_idx, nv, nt, eps, err, s, root_leaf, list);
    return cudaGetLastError();
}

size_t ploc_scratch_bytes(int nt)
{
    PlocBufs Q;
    return carve_ploc_scratch(nullptr, nt, Q);
}

size_t carve_ploc_scratch(void* base, int nt, PlocBufs& Q)
{
    const size_t n = (size_t)(nt > 0 ? nt : 1);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* p = base ? (void*)((char*)base + off) : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    for (int k = 0; k < 2; ++k) {
        Q.cid[k] = (int*)take(sizeof(int) * n);
        Q.blo[k] = (float4*)take(sizeof(float4) * n);
        Q.bhi[k] = (float4*)take(sizeof(float4) * n);
    }
    Q.nn = (int*)take(sizeof(int) * n);
    Q.flags = (uint64_t*)take(sizeof(uint64_t) * n);
    Q.pre = (uint64_t*)take(sizeof(uint64_t) * n);
    Q.sums = (uint64_t*)take(sizeof(uint64_t) * ((n + kScanBlock - 1) / kScanBlock + 1));
    Q.total = (uint64_t*)take(sizeof(uint64_t));
    return off;
}

__global__ void k_classify(const int* __restrict__ idx, const uint8_t* __restrict__ vmoved, int nt, int nv,
                           uint64_t* __restrict__ fl)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    bool mv = false;
    for (int v = 0; v < 3; ++v) {
        int vi = idx[3 * (size_t)t + v];
        if (vi >= 0 && vi < nv && vmoved[vi]) mv = true;
    }
    fl[t] = mv ? 1ull : (1ull << 32);  // static count high, moving count low
}

__global__ void k_split(const uint64_t* __restrict__ fl, const uint64_t* __restrict__ pre, int nt,
                        int* __restrict__ slist, int* __restrict__ dlist)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    uint64_t p = pre[t];
    if (fl[t] >> 32)
        slist[p >> 32] = t;
    else
        dlist[p & 0xFFFFFFFFu] = t;
}

// Split the triangles into static (no moved vertex) and moving ones, keeping
// index order in both lists; returns the counts (synchronises the stream).
cudaError_t split_static_moving(const int* d_idx, const uint8_t* vmoved, int nt, int nv, const PlocBufs& Q,
                                int* slist, int* dlist, int* ns, int* nd, cudaStream_t s)
{
    *ns = 0;
    *nd = 0;
    if (nt <= 0) return cudaSuccess;
    const int T = 256;
    k_classify<<<(nt + T - 1) / T, T, 0, s>>>(d_idx, vmoved, nt, nv, Q.flags);
    count_launches(1);
    const int sb = (nt + kScanBlock - 1) / kScanBlock;
    k_scan64_block<<<sb, kScanT, 0, s>>>(Q.flags, Q.pre, Q.sums, nt);
    count_launches(1);
    k_scan64_small<<<1, 1024, 0, s>>>(Q.sums, sb, Q.total);
    count_launches(1);
    k_scan64_add<<<(nt + T - 1) / T, T, 0, s>>>(Q.pre, Q.sums, nt);
    count_launches(1);
    k_split<<<(nt + T - 1) / T, T, 0, s>>>(Q.flags, Q.pre, nt, slist, dlist);
    count_launches(1);
    uint64_t tot = 0;
    cudaError_t e = cudaMemcpyAsync(&tot, Q.total, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *ns = (int)(tot >> 32);
    *nd = (int)(tot & 0xFFFFFFFFu);
    return cudaSuccess;
}

cudaError_t fill_tri_orig(const float* d_verts, const int* d_idx, const int* list, int nv, int nt, float4* tri_orig,
                          cudaStream_t s)
{
    if (nt <= 0) return cudaSuccess;
    k_fill_orig<<<(nt + 255) / 256, 256, 0, s>>>(d_verts, d_idx, list, nt, nv, tri_orig);
    count_launches(1);
    return cudaGetLastError();
}

void Bvh::release()
{
    cudaFree(scratch);
    cudaFree(pscratch);
    cudaFree(tri_v);
    cudaFree(nodes);
    *this = Bvh();
}

cudaError_t Bvh::reserve(int nt, bool ploc)
{
    if (nt <= cap_ && (!ploc || pscratch)) return cudaSuccess;
    int n = nt > cap_ ? nt : cap_;
    release();
    n = n > 0 ? n : 1;
    size_t sb = bvh_scratch_bytes(n);
    cudaError_t e = cudaMalloc(&scratch, sb);
    if (e != cudaSuccess) return e;
    e = cudaMalloc((void**)&tri_v, sizeof(float4) * 3 * (size_t)n);
    if (e != cudaSuccess) return e;
    e = cudaMalloc((void**)&nodes, sizeof(BNode) * (size_t)n);
    if (e != cudaSuccess) return e;
    size_t pb = 0;
    if (ploc) {
        pb = ploc_scratch_bytes(n);
        e = cudaMalloc(&pscratch, pb);
        if (e != cudaSuccess) return e;
        carve_ploc_scratch(pscratch, n, pbufs);
    }
    carve_bvh_scratch(scratch, n, bufs);
    bufs.tri_v = tri_v;
    bufs.nodes = nodes;
    cap_ = n;
    bytes_ = sb + pb + sizeof(float4) * 3 * (size_t)n + sizeof(BNode) * (size_t)n;
    return cudaSuccess;
}

cudaError_t Bvh::build(const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err, cudaStream_t s,
                       const int* list, bool ploc, float4* tri_out, BNode* nodes_out)
{
    n_tris = 0;
    if (nt == 0) return cudaSuccess;
    cudaError_t e = reserve(nt, ploc);  // may reset every member
    if (e != cudaSuccess) return e;
    n_tris = nt;
    BvhBufs B = bufs;
    if (tri_out) B.tri_v = tri_out;
    if (nodes_out) B.nodes = nodes_out;
    return ploc ? build_ploc(B, pbufs, d_verts, d_idx, nv, nt, eps, err, s, &root_leaf, list)
                : build_lbvh(B, d_verts, d_idx, nv, nt, eps, err, s, &root_leaf, list);
}

namespace {
__global__ void k_relocate(BNode* __restrict__ nodes, int n, int node_off, int tri_off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 d = nodes[i].d;
    d.x = d.x >= 0 ? d.x + node_off : ~(~d.x + tri_off);
    d.y = d.y >= 0 ? d.y + node_off : ~(~d.y + tri_off);
    nodes[i].d = d;
}
}  // namespace

cudaError_t relocate_nodes(BNode* nodes, int n_nodes, int node_off, int tri_off, cudaStream_t s)
{
    if (n_nodes <= 0 || (node_off == 0 && tri_off == 0)) return cudaSuccess;
    k_relocate<<<(n_nodes + 255) / 256, 256, 0, s>>>(nodes, n_nodes, node_off, tri_off);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adgi
