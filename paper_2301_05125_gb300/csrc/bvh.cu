// bvh.cu -- software BVH for the probe rays (the paper traces with DXR on RT
// cores, Sec. 5; here a linear BVH is built on the device every time the
// geometry moves).
//
// Build: centroid bounds -> 63-bit Morton codes -> stable LSD radix sort
// (8 passes of 8 bits, own kernels) -> Karras (HPG 2012) radix-tree hierarchy
// -> bottom-up child boxes, each leaf box enlarged by eps so that box tests
// stay conservative for the watertight triangle test.
#include <cstdio>

#include "adgi_internal.cuh"
#include "bvh.cuh"
#include "kernels.cuh"

namespace adgi {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) { return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u); }

__global__ void k_init_bounds(uint32_t* __restrict__ bounds)
{
    if (threadIdx.x < 3) bounds[threadIdx.x] = 0xFFFFFFFFu;
    else if (threadIdx.x < 6) bounds[threadIdx.x] = 0u;
}

__global__ void k_tri_prep(const float* __restrict__ verts, const int* __restrict__ idx, int nt, int nv,
                           float4* __restrict__ tri_orig, uint32_t* __restrict__ bounds, int* __restrict__ err)
{
    __shared__ uint32_t s_lo[3], s_hi[3];
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = 0xFFFFFFFFu;
        s_hi[threadIdx.x] = 0u;
    }
    __syncthreads();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) {
        float c[3] = {0.f, 0.f, 0.f};
        for (int v = 0; v < 3; ++v) {
            int vi = idx[3 * (size_t)t + v];
            if (vi < 0 || vi >= nv) {  // guarded: an out-of-range index reads vertex 0
                atomicOr(err, kErrIndex);
                vi = 0;
            }
            float x = verts[3 * (size_t)vi], y = verts[3 * (size_t)vi + 1], z = verts[3 * (size_t)vi + 2];
            tri_orig[3 * (size_t)t + v] = make_float4(x, y, z, 0.f);
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
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&bounds[threadIdx.x], s_lo[threadIdx.x]);
        atomicMax(&bounds[3 + threadIdx.x], s_hi[threadIdx.x]);
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

__global__ void k_morton(const float4* __restrict__ tri_orig, int nt, const uint32_t* __restrict__ bounds,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float lo[3], ext[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = ord2f(bounds[k]);
        float hi = ord2f(bounds[3 + k]);
        ext[k] = fmaxf(hi - lo[k], 1e-30f);
    }
    float4 A = tri_orig[3 * (size_t)t], B = tri_orig[3 * (size_t)t + 1], C = tri_orig[3 * (size_t)t + 2];
    float c[3] = {(A.x + B.x + C.x) * (1.0f / 3.0f), (A.y + B.y + C.y) * (1.0f / 3.0f),
                  (A.z + B.z + C.z) * (1.0f / 3.0f)};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        float u = (c[k] - lo[k]) / ext[k] * 2097152.0f;
        u = fminf(fmaxf(u, 0.0f), 2097151.0f);
        q[k] = (uint32_t)u;
    }
    keys[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
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

__global__ void k_tri_order(const float4* __restrict__ tri_orig, const uint32_t* __restrict__ order, int nt,
                            float4* __restrict__ tri_v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    uint32_t t = order[i];
    float4 A = tri_orig[3 * (size_t)t], B = tri_orig[3 * (size_t)t + 1], C = tri_orig[3 * (size_t)t + 2];
    A.w = __int_as_float((int)t);
    tri_v[3 * (size_t)i] = A;
    tri_v[3 * (size_t)i + 1] = B;
    tri_v[3 * (size_t)i + 2] = C;
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
__global__ void k_hierarchy(const uint64_t* __restrict__ keys, int n, BNode* __restrict__ nodes,
                            int* __restrict__ par_int, int* __restrict__ par_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
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
    nodes[i].d = make_int4(left, right, 0, 0);
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

__global__ void k_bounds(const float4* __restrict__ tri_v, int n, BNode* nodes, const int* __restrict__ par_int,
                         const int* __restrict__ par_leaf, int* flags, float eps, int* err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 A = tri_v[3 * (size_t)i], B = tri_v[3 * (size_t)i + 1], C = tri_v[3 * (size_t)i + 2];
    float lo[3] = {fminf(fminf(A.x, B.x), C.x) - eps, fminf(fminf(A.y, B.y), C.y) - eps,
                   fminf(fminf(A.z, B.z), C.z) - eps};
    float hi[3] = {fmaxf(fmaxf(A.x, B.x), C.x) + eps, fmaxf(fmaxf(A.y, B.y), C.y) + eps,
                   fmaxf(fmaxf(A.z, B.z), C.z) + eps};
    int child = ~i;
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
        child = par;
        par = par_int[par];
    }
}

}  // namespace

size_t Bvh::bytes() const { return bytes_; }

size_t bvh_scratch_bytes(int nt)
{
    BvhBufs B;
    return carve_bvh_scratch(nullptr, nt, B);
}

// Carve the scratch buffers of a build for nt triangles out of one block
// (base may be null to only compute the size); every piece 256-byte aligned.
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
    B.tri_orig = (float4*)take(sizeof(float4) * 3 * n);
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
    return off;
}

// The build itself: every buffer comes from B (scratch) or the outputs
// B.tri_v / B.nodes.  All work is ordered on stream s; nothing is allocated.
cudaError_t build_lbvh(const BvhBufs& B, const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err,
                       cudaStream_t s, int* root_leaf)
{
    if (nt <= 0) {
        *root_leaf = -1;
        return cudaSuccess;
    }
    const int T = 256;
    k_init_bounds<<<1, 32, 0, s>>>(B.bounds);
    count_launches(1);
    k_tri_prep<<<(nt + T - 1) / T, T, 0, s>>>(d_verts, d_idx, nt, nv, B.tri_orig, B.bounds, err);
    count_launches(1);
    k_morton<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_orig, nt, B.bounds, B.keys[0], B.vals[0]);
    count_launches(1);
    int nb = (nt + kSortTile - 1) / kSortTile;
    int cur = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        k_hist<<<nb, kSortThreads, 0, s>>>(B.keys[cur], nt, shift, B.hist, nb);
        count_launches(1);
        k_scan_small<<<1, 1024, 0, s>>>(B.hist, 256 * nb);
        count_launches(1);
        k_scatter<<<nb, kSortThreads, 0, s>>>(B.keys[cur], B.vals[cur], B.keys[cur ^ 1], B.vals[cur ^ 1], nt, shift,
                                               B.hist, nb);
        count_launches(1);
        cur ^= 1;
    }
    k_tri_order<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_orig, B.vals[cur], nt, B.tri_v);
    count_launches(1);
    if (nt == 1) {
        *root_leaf = 0;
        return cudaGetLastError();
    }
    *root_leaf = -1;
    cudaError_t e = cudaMemsetAsync(B.flags, 0, sizeof(int) * (size_t)nt, s);
    if (e != cudaSuccess) return e;
    k_hierarchy<<<(nt - 1 + T - 1) / T, T, 0, s>>>(B.keys[cur], nt, B.nodes, B.par_int, B.par_leaf);
    count_launches(1);
    k_bounds<<<(nt + T - 1) / T, T, 0, s>>>(B.tri_v, nt, B.nodes, B.par_int, B.par_leaf, B.flags, eps, err);
    count_launches(1);
    return cudaGetLastError();
}

void Bvh::release()
{
    cudaFree(scratch);
    cudaFree(tri_v);
    cudaFree(nodes);
    *this = Bvh();
}

cudaError_t Bvh::reserve(int nt)
{
    if (nt <= cap_) return cudaSuccess;
    release();
    int n = nt > 0 ? nt : 1;
    size_t sb = bvh_scratch_bytes(n);
    cudaError_t e = cudaMalloc(&scratch, sb);
    if (e != cudaSuccess) return e;
    e = cudaMalloc((void**)&tri_v, sizeof(float4) * 3 * (size_t)n);
    if (e != cudaSuccess) return e;
    e = cudaMalloc((void**)&nodes, sizeof(BNode) * (size_t)n);
    if (e != cudaSuccess) return e;
    carve_bvh_scratch(scratch, n, bufs);
    bufs.tri_v = tri_v;
    bufs.nodes = nodes;
    tri_orig = bufs.tri_orig;
    cap_ = n;
    bytes_ = sb + sizeof(float4) * 3 * (size_t)n + sizeof(BNode) * (size_t)n;
    return cudaSuccess;
}

// Host-side: scene extent -> enlargement eps (1e-5 of the larger of the extent
// and the largest coordinate magnitude).
cudaError_t Bvh::build(const float* d_verts, const int* d_idx, int nv, int nt, float eps, int* err, cudaStream_t s)
{
    n_tris = 0;
    if (nt == 0) return cudaSuccess;
    cudaError_t e = reserve(nt);  // may reset every member
    if (e != cudaSuccess) return e;
    n_tris = nt;
    return build_lbvh(bufs, d_verts, d_idx, nv, nt, eps, err, s, &root_leaf);
}

SceneDev Bvh::view(const float* albedo, int nv, int* err) const
{
    SceneDev S;
    S.max_iter = 2 * n_tris + 16;
    S.err = err;
    S.n_tris = n_tris;
    S.n_verts = nv;
    S.tri_v = tri_v;
    S.tri_orig = tri_orig;
    S.albedo = albedo;
    S.nodes = nodes;
    S.root_leaf = root_leaf;
    return S;
}

}  // namespace adgi
