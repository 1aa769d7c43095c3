// bvhbody.cuh -- device bodies of the linear BVH build of a small part
// (sm_103a): triangle fetch and centroid bounds, Morton keys, the one-block
// sort, the Karras hierarchy and the bottom-up boxes.  The build kernels
// (bvh.cu) and the persistent batched tick (tick.cu, which rebuilds a
// volume's moving part inside the launch) run the same bodies.
#pragma once
#include "adgi_internal.cuh"

namespace adgi {

namespace {

__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float ord2f(uint32_t u) { return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u); }

// box enlargement of one triangle: the scene's eps, or 1e-5 of the triangle's
// largest |coordinate| if that is larger (geometry moved far from where eps
// was measured); keeps box tests conservative for the watertight test
__device__ __forceinline__ float tri_eps(float eps, float4 A, float4 B, float4 C)
{
    float m = fmaxf(fmaxf(fmaxf(fabsf(A.x), fabsf(A.y)), fmaxf(fabsf(A.z), fabsf(B.x))),
                    fmaxf(fmaxf(fabsf(B.y), fabsf(B.z)), fmaxf(fmaxf(fabsf(C.x), fabsf(C.y)), fabsf(C.z))));
    return fmaxf(eps, 1e-5f * m);
}

// listed triangle i: its vertices into tri_in[3i..3i+2] (v0.w = its index),
// its centroid into the ordered-integer bounds s_lo / s_hi
__device__ __forceinline__ void tri_fetch(const float* __restrict__ verts, const int* __restrict__ idx,
                                          const int* __restrict__ list, int nv, int i, float4* __restrict__ tri_in,
                                          uint32_t* s_lo, uint32_t* s_hi, int* __restrict__ err)
{
    const int t = list ? list[i] : i;
    float c[3] = {0.f, 0.f, 0.f};
    for (int v = 0; v < 3; ++v) {
        int vi = idx[3 * (size_t)t + v];
        if (vi < 0 || vi >= nv) {  // guarded: an out-of-range index reads vertex 0
            atomicOr(err, kErrIndex);
            vi = 0;
        }
        float x = verts[3 * (size_t)vi], y = verts[3 * (size_t)vi + 1], z = verts[3 * (size_t)vi + 2];
        tri_in[3 * (size_t)i + v] = make_float4(x, y, z, v == 0 ? __int_as_float(t) : 0.f);
        c[0] += x;
        c[1] += y;
        c[2] += z;
    }
    for (int k = 0; k < 3; ++k) {
        uint32_t o = f2ord(c[k] * (1.0f / 3.0f));
        atomicMin(&s_lo[k], o);
        atomicMax(&s_hi[k], o);
    }
}

// vertices of the listed triangles into an original-order array (shading)
__device__ __forceinline__ void fill_orig_body(const float* __restrict__ verts, const int* __restrict__ idx,
                                               const int* __restrict__ list, int nt, int nv, float4* tri_orig, int i)
{
    if (i >= nt) return;
    const int t = list ? list[i] : i;
    for (int v = 0; v < 3; ++v) {
        int vi = idx[3 * (size_t)t + v];
        vi = (vi < 0 || vi >= nv) ? 0 : vi;
        tri_orig[3 * (size_t)t + v] =
            make_float4(verts[3 * (size_t)vi], verts[3 * (size_t)vi + 1], verts[3 * (size_t)vi + 2], 0.f);
    }
}

__device__ __forceinline__ uint64_t spread21(uint32_t v)
{
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// 63-bit Morton code of a triangle's centroid in the centroid bounds
// (ordered-integer lo / hi)
__device__ __forceinline__ uint64_t morton_key(float4 A, float4 B, float4 C, const uint32_t* bounds)
{
    float lo[3], ext[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = ord2f(bounds[k]);
        float hi = ord2f(bounds[3 + k]);
        ext[k] = fmaxf(hi - lo[k], 1e-30f);
    }
    float c[3] = {(A.x + B.x + C.x) * (1.0f / 3.0f), (A.y + B.y + C.y) * (1.0f / 3.0f),
                  (A.z + B.z + C.z) * (1.0f / 3.0f)};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        float u = (c[k] - lo[k]) / ext[k] * 2097152.0f;
        u = fminf(fmaxf(u, 0.0f), 2097151.0f);
        q[k] = (uint32_t)u;
    }
    return (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
}

// The Morton order of a small build (nt <= kSmallBuild) in one block: the
// triangles and their centroid bounds, the keys, a bitonic sort of (key,
// index) pairs in shared memory -- the order of the stable radix sort, since
// equal keys keep index order -- and the triangles gathered into that order.
// One launch instead of the 8 radix passes and their scans.
constexpr int kSmallBuild = 2048;

// (sk, sv: kSmallBuild keys and values of shared memory; any block size)
__device__ __forceinline__ void morton_small_body(const float* __restrict__ verts, const int* __restrict__ idx,
                                                  const int* __restrict__ list, int nt, int nv, float4* tri_in,
                                                  uint64_t* keys, uint32_t* vals, float4* tri_v, int* err,
                                                  uint64_t* sk, uint32_t* sv)
{
    __shared__ uint32_t s_b[6];
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid < 3) s_b[tid] = 0xFFFFFFFFu;
    else if (tid < 6) s_b[tid] = 0u;
    __syncthreads();
    for (int i = tid; i < nt; i += nthr) tri_fetch(verts, idx, list, nv, i, tri_in, s_b, s_b + 3, err);
    __syncthreads();  // also orders this block's tri_in writes before the reads below
    int n2 = 2;
    while (n2 < nt) n2 <<= 1;
    for (int i = tid; i < n2; i += nthr) {
        if (i < nt) {
            sk[i] = morton_key(tri_in[3 * (size_t)i], tri_in[3 * (size_t)i + 1], tri_in[3 * (size_t)i + 2], s_b);
            sv[i] = (uint32_t)i;
        } else {  // padding: after every real pair
            sk[i] = ~0ull;
            sv[i] = 0xFFFFFFFFu;
        }
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n2; i += nthr) {
                const int l = i ^ j;
                if (l <= i) continue;
                const uint64_t ka = sk[i], kb = sk[l];
                const uint32_t va = sv[i], vb = sv[l];
                const bool gt = ka > kb || (ka == kb && va > vb);
                if (gt == ((i & k) == 0)) {  // ascending where bit k of i is clear
                    sk[i] = kb, sk[l] = ka;
                    sv[i] = vb, sv[l] = va;
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < nt; i += nthr) {
        const uint32_t t = sv[i];
        keys[i] = sk[i];
        vals[i] = t;
        tri_v[3 * (size_t)i] = tri_in[3 * (size_t)t];
        tri_v[3 * (size_t)i + 1] = tri_in[3 * (size_t)t + 1];
        tri_v[3 * (size_t)i + 2] = tri_in[3 * (size_t)t + 2];
    }
}

__device__ __forceinline__ int delta(const uint64_t* keys, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    uint64_t a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clzll((long long)(a ^ b));
}

// Karras 2012: internal node i covers a key range; its split is the first
// position where the highest differing bit changes.
// node i of the radix tree; the child references are written relocated by
// node_off / tri_off (the part's place in the scene's arrays), the parent
// links stay local
__device__ __forceinline__ void hierarchy_body(const uint64_t* keys, int n, BNode* nodes, int* par_int, int* par_leaf,
                                               int i, int node_off, int tri_off)
{
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    nodes[i].d = make_int4(left < 0 ? ~(gamma + tri_off) : left + node_off,
                           right < 0 ? ~(gamma + 1 + tri_off) : right + node_off, 0, 0);
    if (left < 0)
        par_leaf[gamma] = i;
    else
        par_int[gamma] = i;
    if (right < 0)
        par_leaf[gamma + 1] = i;
    else
        par_int[gamma + 1] = i;
    if (i == 0) par_int[0] = -1;
}

// leaf i's box up the tree (the child references relocated as by hierarchy_body)
__device__ __forceinline__ void bounds_body(const float4* tri_v, int n, BNode* nodes, const int* par_int,
                                            const int* par_leaf, int* flags, float eps, int* err, int i, int node_off,
                                            int tri_off)
{
    if (i >= n) return;
    float4 A = tri_v[3 * (size_t)i], B = tri_v[3 * (size_t)i + 1], C = tri_v[3 * (size_t)i + 2];
    eps = tri_eps(eps, A, B, C);
    float lo[3] = {fminf(fminf(A.x, B.x), C.x) - eps, fminf(fminf(A.y, B.y), C.y) - eps,
                   fminf(fminf(A.z, B.z), C.z) - eps};
    float hi[3] = {fmaxf(fmaxf(A.x, B.x), C.x) + eps, fmaxf(fmaxf(A.y, B.y), C.y) + eps,
                   fmaxf(fmaxf(A.z, B.z), C.z) + eps};
    int child = ~(i + tri_off);
    int par = par_leaf[i];
    for (int depth = 0; par >= 0; ++depth) {
        if (depth > 128) {  // a radix tree over 95-bit keys is at most 95 deep
            atomicOr(err, kErrBvh);
            return;
        }
        BNode* pn = nodes + par;
        int4 ch = pn->d;
        float* f = reinterpret_cast<float*>(pn);
        int slot = (ch.x == child) ? 0 : 6;
        for (int k = 0; k < 3; ++k) {
            __stcg(f + slot + k, lo[k]);
            __stcg(f + slot + 3 + k, hi[k]);
        }
        __threadfence();
        int old = atomicAdd(&flags[par], 1);
        if (old == 0) return;
        __threadfence();
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(__ldcg(f + k), __ldcg(f + 6 + k));
            hi[k] = fmaxf(__ldcg(f + 3 + k), __ldcg(f + 9 + k));
        }
        child = par + node_off;
        par = par_int[par];
    }
}

}  // namespace

}  // namespace adgi
