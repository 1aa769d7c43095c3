// wave.cuh -- device bodies of the ray wavefront (sm_103a): the pilot and
// adaptive nearest-hit traces and the three shading steps (prep, shadow
// rays, finish).  The ordinary kernels (trace.cu, shade.cu) and the
// persistent batched tick (tick.cu) run the same bodies.
#pragma once
#include "adgi_internal.cuh"
#include "kernels.cuh"

namespace adgi {

namespace {
// probe owning main ray r: the last p with off[p] <= r, searched in [lo, hi]
template <bool kLive = false>
__device__ __forceinline__ int probe_of_ray(const uint32_t* off, uint32_t r, int lo, int hi)
{
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ldl<kLive>(off + mid) <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// per block: bounds of the probe range of this block's rays, in shared memory
template <bool kLive = false>
__device__ __forceinline__ void block_probe_range(const uint32_t* off, int P, uint32_t r0, uint32_t r1, int* s_lo,
                                                  int* s_hi)
{
    if (threadIdx.x == 0) *s_lo = probe_of_ray<kLive>(off, r0, 0, P - 1);
    if (threadIdx.x == 32 % blockDim.x) *s_hi = probe_of_ray<kLive>(off, r1, 0, P - 1);
    __syncthreads();
}

// direction at position k of the SF row of m points, and its SF index *i
__device__ __forceinline__ float3 main_dir(const FrameConst& F, const float4* __restrict__ sf, uint32_t m, uint32_t k,
                                           uint32_t* i)
{
    float4 s = __ldg(sf + (size_t)m * (m - 1) / 2 + k);
    *i = (uint32_t)__float_as_int(s.w);
    return rotate(F.R, s);
}

// j: the thread's index in the pilot-ray launch (one warp: 32 consecutive j)
template <bool kLive = false>
__device__ __forceinline__ void pilot_trace_body(const VolConst& V, const FrameDev* FD, const SceneDev& S, int2* hit,
                                                 int j)
{
    const FrameConst& F = FD->F;
    // A warp traces one octant of 32 consecutive probes (the stratified
    // directions of one octant, from neighbouring origins), not 8 octants of
    // 4 probes.  Thread j of the launch: group g = j / 256 of 32 probes,
    // octant (j / 32) % 8, probe 32 g + j % 32; results stay at 8 p + o.
    const int p = V.p_lo + ((j >> 8) << 5) + (j & 31), o = (j >> 5) & 7;
    if (p >= V.p_hi) return;
    const int i = p * kPilots + o;
    if (V.cls[p] == 0) {  // outside V_out: no pilot rays
        hit[i] = make_int2((int)kMiss, 0x7F800000);
        return;
    }
    float3 org = probe_pos(V, p);
    float3 d = pilot_dir(F.pilot_key, (uint32_t)p, o);
    float t;
    uint32_t h;
    trace_closest<kLive>(S, org, d, V.tmin, __int_as_float(0x7F800000), t, h);
    hit[i] = make_int2((int)h, __float_as_int(t));
}

// Adaptive ray r (its probe searched in [lo, hi]): row position r - off[p]
// of probe p, whose SF index i names the slot off[p] + i of the result.
template <bool kLive>
__device__ __forceinline__ void main_trace_ray(const VolConst& V, const FrameConst& F, const SceneDev& S,
                                               const uint32_t* off, const float4* __restrict__ sf, int2* hit,
                                               uint32_t r, int lo, int hi)
{
    int p = probe_of_ray<kLive>(off, r, lo, hi);
    uint32_t base = ldl<kLive>(off + p);
    uint32_t m = ldl<kLive>(off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || r - base >= m) {
        atomicOr(V.err, kErrRayRange);
        return;
    }
    float3 org = probe_pos(V, p);
    uint32_t i;
    float3 d = main_dir(F, sf, m, r - base, &i);
    if (i >= m) {
        atomicOr(V.err, kErrRayRange);
        return;
    }
    float t;
    uint32_t h;
    trace_closest<kLive>(S, org, d, V.tmin, __int_as_float(0x7F800000), t, h);
    hit[base + i] = make_int2((int)h, __float_as_int(t));
}

// Thread r takes row position r - off[p] of probe p, whose SF index i names
// the slot off[p] + i of the result: the threads of a warp trace nearby
// directions (the rows are in a spatial order).
template <bool kLive>
__device__ __forceinline__ void main_trace_body(const VolConst& V, const FrameDev* FD, const SceneDev& S,
                                                const uint32_t* off, const float4* __restrict__ sf, uint32_t R,
                                                int2* hit, unsigned bx)
{
    const FrameConst& F = FD->F;
    __shared__ int s_lo, s_hi;
    // the rays of probes [p_lo, p_hi): [off[p_lo], off[p_hi]) (all probes:
    // [0, off[P]); with clip volumes part of the budget may stay unspent)
    const uint32_t rb = ldl<kLive>(off + V.p_lo), re = min(ldl<kLive>(off + V.p_hi), R);
    uint32_t r0 = rb + bx * blockDim.x;
    if (r0 >= re) return;  // the whole block
    uint32_t r1 = min(re - 1, r0 + blockDim.x - 1);
    block_probe_range<kLive>(off, V.P, r0, r1, &s_lo, &s_hi);
    uint32_t r = r0 + threadIdx.x;
    if (r >= re) return;
    main_trace_ray<kLive>(V, F, S, off, sf, hit, r, s_lo, s_hi);
}

// The same for one warp: rays [rb + 32 w, rb + 32 w + 32), the probe range
// found by two lanes and passed round the warp (no block barrier)
// chunk_p (optional, all probes only): the probe of ray 32 c for every
// chunk c below off[P], written by the allocation, which bounds the search.
template <bool kLive>
__device__ __forceinline__ void main_trace_warp_body(const VolConst& V, const FrameDev* FD, const SceneDev& S,
                                                     const uint32_t* off, const float4* __restrict__ sf, uint32_t R,
                                                     int2* hit, unsigned w, const uint32_t* chunk_p = nullptr)
{
    const FrameConst& F = FD->F;
    const int lane = threadIdx.x & 31;
    const uint32_t rb = ldl<kLive>(off + V.p_lo), re = min(ldl<kLive>(off + V.p_hi), R);
    const uint32_t r0 = rb + 32u * w;
    if (r0 >= re) return;  // the whole warp
    const uint32_t r1 = min(re - 1, r0 + 31u);
    int lo = 0, hi = 0;
    if (chunk_p && V.p_lo == 0) {
        lo = (int)ldl<kLive>(chunk_p + w);
        hi = r0 + 32u < re ? (int)ldl<kLive>(chunk_p + w + 1) : V.P - 1;
    } else {
        if (lane == 0) lo = probe_of_ray<kLive>(off, r0, 0, V.P - 1);
        if (lane == 1) hi = probe_of_ray<kLive>(off, r1, 0, V.P - 1);
        lo = __shfl_sync(0xFFFFFFFFu, lo, 0);
        hi = __shfl_sync(0xFFFFFFFFu, hi, 1);
    }
    const uint32_t r = r0 + lane;
    if (r >= re) return;
    main_trace_ray<kLive>(V, F, S, off, sf, hit, r, lo, hi);
}

constexpr float kInvPi = 0.31830987f;
constexpr float kLumR = 0.2126f, kLumG = 0.7152f, kLumB = 0.0722f;


// The rays of a block: pilot rays (ray r = probe r/8, octant r%8), adaptive
// rays (ray r of the prefix offsets off[]; the block's probe range is found
// once by two threads) or Metropolis samples (ray r = sample sf[r] of the
// grouped order).
struct RaySet {
    int mode;                 // 0 pilot, 1 adaptive, 2 Metropolis samples in grouped order, 3 dynamic rays
    uint32_t n;               // rays in the set (dynamic rays: the budget)
    const uint32_t* off;      // adaptive: prefix offsets
    const float4* sf;         // adaptive: spherical Fibonacci sets; samples: {w.xyz, probe bits}
    DynRays dyn;              // dynamic rays
};

// The first ray of the set for probes [p_lo, p_hi): pilot rays 8 p_lo,
// adaptive rays off[p_lo]; thread idx of the launch takes ray base + idx.
template <bool kLive>
__device__ __forceinline__ uint32_t ray_base(const VolConst& V, const RaySet& Rs)
{
    return Rs.mode == 0 ? (uint32_t)V.p_lo * kPilots : Rs.mode == 1 ? ldl<kLive>(Rs.off + V.p_lo) : 0u;
}

template <bool kLive>
__device__ __forceinline__ void block_range(const VolConst& V, const RaySet& Rs, unsigned bx, int* s_lo, int* s_hi)
{
    if (Rs.mode == 1) {
        const uint32_t b = ray_base<kLive>(V, Rs);
        uint32_t r0 = b + bx * blockDim.x;
        uint32_t r1 = b + min(Rs.n - 1, bx * blockDim.x + blockDim.x - 1);
        if (threadIdx.x == 0) *s_lo = probe_of_ray<kLive>(Rs.off, r0, 0, V.P - 1);
        if (threadIdx.x == 32 % blockDim.x) *s_hi = probe_of_ray<kLive>(Rs.off, r1, 0, V.P - 1);
    }
    __syncthreads();
}

// The ray a thread handles: thread r takes position r of the set; a pilot ray
// is stored at slot r, an adaptive ray at base + (SF index of row position
// r - base), so that a warp works on nearby directions.  Gives the slot,
// origin and direction; false if the ray range is inconsistent.
template <bool kLive>
__device__ __forceinline__ bool ray_of(const VolConst& V, const FrameConst& F, const RaySet& Rs, uint32_t r, int lo,
                                       int hi, uint32_t& slot, float3& o, float3& d)
{
    if (Rs.mode == 0) {
        int p = (int)(r >> 3);
        if (V.cls[p] == 0) return false;  // outside V_out: no pilot ray
        slot = r;
        o = probe_pos(V, p);
        d = pilot_dir(F.pilot_key, (uint32_t)p, (int)(r & 7));
        return true;
    }
    if (Rs.mode == 3) {
        int p, t;
        if (!dyn_ray_of(V, Rs.dyn, r, p, t, d)) return false;
        slot = r;
        o = probe_pos(V, p);
        return true;
    }
    if (Rs.mode == 2) {
        const float4 a = __ldg(Rs.sf + r);
        const int p = __float_as_int(a.w);
        if (p < 0 || p >= V.P || V.cls[p] != 2) return false;  // samples outside V_in are dropped
        slot = r;
        o = probe_pos(V, p);
        d = make_float3(a.x, a.y, a.z);
        return true;
    }
    if (r >= ldl<kLive>(Rs.off + V.p_hi)) return false;  // beyond the adaptive rays of the probes (unspent budget)
    int p = probe_of_ray<kLive>(Rs.off, r, lo, hi);
    uint32_t base = ldl<kLive>(Rs.off + p), m = ldl<kLive>(Rs.off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || r - base >= m) return false;
    o = probe_pos(V, p);
    float4 s = __ldg(Rs.sf + (size_t)m * (m - 1) / 2 + (r - base));
    const uint32_t i = (uint32_t)__float_as_int(s.w);
    if (i >= m) return false;
    slot = base + i;
    d = rotate(F.R, s);
    return true;
}

// exact FP32 geometric normal of triangle tri (original order; kLive: a
// moving triangle's row may have been written earlier in the same launch)
template <bool kLive = false>
__device__ __forceinline__ float3 tri_normal(const SceneDev& S, int tri)
{
    float4 A = ldl<kLive>(S.tri_orig + 3 * (size_t)tri), B = ldl<kLive>(S.tri_orig + 3 * (size_t)tri + 1),
           C = ldl<kLive>(S.tri_orig + 3 * (size_t)tri + 2);
    float e1x = fs(B.x, A.x), e1y = fs(B.y, A.y), e1z = fs(B.z, A.z);
    float e2x = fs(C.x, A.x), e2y = fs(C.y, A.y), e2z = fs(C.z, A.z);
    float cx = fs(fm(e1y, e2z), fm(e1z, e2y));
    float cy = fs(fm(e1z, e2x), fm(e1x, e2z));
    float cz = fs(fm(e1x, e2y), fm(e1y, e2x));
    float cl = fsq(dot3x(cx, cy, cz, cx, cy, cz));
    return cl > 0.0f ? make_float3(fd(cx, cl), fd(cy, cl), fd(cz, cl)) : make_float3(0.f, 0.f, 1.f);
}

__device__ __forceinline__ float3 shadow_dir(const Light& Li, float3 xs)
{
    return Li.kind == 0 ? make_float3(fs(Li.v[0], xs.x), fs(Li.v[1], xs.y), fs(Li.v[2], xs.z))
                        : make_float3(-Li.v[0], -Li.v[1], -Li.v[2]);
}

template <bool kLive>
__device__ __forceinline__ void shade_prep_body(const VolConst& V, const FrameDev* FD, const SceneDev& S,
                                                const RaySet& Rs, const int2* hit, unsigned long long* vis,
                                                uint4* jobs, uint8_t* job_light, unsigned* job_count, unsigned job_cap,
                                                unsigned bx)
{
    const FrameConst& F = FD->F;
    const LightSet& L = FD->L;
    __shared__ int s_lo, s_hi;
    block_range<kLive>(V, Rs, bx, &s_lo, &s_hi);
    const uint32_t idx = bx * blockDim.x + threadIdx.x;
    const uint32_t r = ray_base<kLive>(V, Rs) + idx;
    bool front = false;
    float3 xs = make_float3(0.f, 0.f, 0.f), n = make_float3(0.f, 0.f, 1.f);
    uint32_t slot = r;
    float3 o, d;
    if (idx < Rs.n && ray_of<kLive>(V, F, Rs, r, s_lo, s_hi, slot, o, d)) {
        vis[slot] = 0ull;
        int2 hv = hit[slot];
        uint32_t h = (uint32_t)hv.x;
        if (h != kMiss && !(h & kBackBit)) {
            float t = __int_as_float(hv.y);
            n = tri_normal<kLive>(S, (int)h);
            float3 x = make_float3(fa(o.x, fm(t, d.x)), fa(o.y, fm(t, d.y)), fa(o.z, fm(t, d.z)));
            xs = make_float3(fa(x.x, fm(V.tmin, n.x)), fa(x.y, fm(V.tmin, n.y)), fa(x.z, fm(V.tmin, n.z)));
            front = true;
        }
    }
    // The block's jobs take one range of the job list: one atomic per block
    // on the shared counter (one per warp and light contended on that
    // address).  Pass 1 counts each warp's jobs, thread 0 scans the warp
    // totals and claims the range, pass 2 writes each warp's jobs light by
    // light (a warp's jobs for one light stay contiguous: nearby origins,
    // one light, so k_shadow's warps trace coherent rays).
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto wants = [&](int l) {
        if (!front) return false;
        const float3 D = shadow_dir(L.l[l], xs);
        return dot3x(n.x, n.y, n.z, D.x, D.y, D.z) > 0.0f;
    };
    unsigned wtot = 0;
    for (int l = 0; l < L.n; ++l) wtot += (unsigned)__popc(__ballot_sync(0xFFFFFFFFu, wants(l)));
    __shared__ unsigned s_w[8], s_base;  // at most 256 threads: 8 warps
    if (lane == 0) s_w[w] = wtot;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (unsigned k = 0; k < (blockDim.x >> 5); ++k) {
            const unsigned c = s_w[k];
            s_w[k] = t;
            t += c;
        }
        s_base = t ? atomicAdd(job_count, t) : 0u;
    }
    __syncthreads();
    unsigned base = s_base + s_w[w];
    for (int l = 0; l < L.n; ++l) {
        const bool want = wants(l);
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, want);
        if (want) {
            const unsigned js = base + __popc(mask & ((1u << lane) - 1u));
            if (js < job_cap) {
                jobs[js] = make_uint4(__float_as_uint(xs.x), __float_as_uint(xs.y), __float_as_uint(xs.z), slot);
                job_light[js] = (uint8_t)l;
            } else {
                atomicOr(V.err, kErrRayRange);
            }
        }
        base += (unsigned)__popc(mask);
    }
}

// Shadow job j (one lane): light l of the job is seen from its origin when
// no triangle blocks the segment (point light) or the ray (sun); then bit l
// of the ray's visibility word is set.
template <bool kLive = false>
__device__ __forceinline__ void shadow_job(const LightSet& L, const SceneDev& S, const uint4* jobs,
                                           const uint8_t* job_light, unsigned long long* vis, unsigned j)
{
    uint4 jb = jobs[j];
    int l = job_light[j];
    const Light& Li = L.l[l];
    float3 xs = make_float3(__uint_as_float(jb.x), __uint_as_float(jb.y), __uint_as_float(jb.z));
    float3 D = shadow_dir(Li, xs);
    float thi = Li.kind == 0 ? 1.0f : __int_as_float(0x7F800000);
    if (!trace_any<kLive>(S, xs, D, 0.0f, thi)) atomicOr(vis + jb.w, 1ull << l);
}

// The shadow jobs [0, min(*job_count, job_cap)) in rounds of 32 consecutive
// jobs, one a lane, with a uniform trip count per warp and an explicit
// reconvergence per round (lanes that finish early wait instead of running
// ahead on their own).  Each warp takes the next round from the counter
// next_round (zero before the launch), so a warp that drew short rays takes
// more rounds and the warps end together.  leader: the one lane that counts
// the jobs.
template <bool kLive = false>
__device__ __forceinline__ void shadow_body(const FrameDev* FD, const SceneDev& S, const uint4* jobs,
                                            const uint8_t* job_light, const unsigned* job_count, unsigned job_cap,
                                            unsigned long long* vis, unsigned long long* shadow_ctr,
                                            unsigned* next_round, bool leader)
{
    const LightSet& L = FD->L;
    const unsigned total = min(*job_count, job_cap);
    if (leader) atomicAdd(shadow_ctr, (unsigned long long)total);
    const unsigned lane = threadIdx.x & 31u, rounds = (total + 31u) / 32u;
    for (;;) {
        unsigned g = 0;
        if (lane == 0) g = atomicAdd(next_round, 1u);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= rounds) break;
        const unsigned j = 32u * g + lane;
        if (j < total) shadow_job<kLive>(L, S, jobs, job_light, vis, j);
        __syncwarp();
    }
}

template <bool kLive>
__device__ __forceinline__ void shade_finish_body(const VolConst& V, const FrameDev* FD, const SceneDev& S,
                                                  const RaySet& Rs, const int2* hit, const unsigned long long* vis,
                                                  const void* __restrict__ irr, const void* __restrict__ dep,
                                                  float4* rec, float* lum, unsigned bx)
{
    const FrameConst& F = FD->F;
    const LightSet& L = FD->L;
    // adaptive rays and samples always carry the multi-bounce term; pilot
    // records are blended (so need it) only on the first frame of a pair
    const int bounce = Rs.mode != 0 || F.even;
    __shared__ int s_lo, s_hi;
    block_range<kLive>(V, Rs, bx, &s_lo, &s_hi);
    const uint32_t idx = bx * blockDim.x + threadIdx.x;
    if (idx >= Rs.n) return;
    const uint32_t r = ray_base<kLive>(V, Rs) + idx;
    uint32_t slot;
    float3 o, d;
    if (Rs.mode == 0 && V.cls[r >> 3] == 0) {  // a culled pilot: a miss with nothing gathered
        rec[r] = make_float4(0.f, 0.f, 0.f, V.depth_max);
        if (lum) lum[r] = 0.0f;
        return;
    }
    if (Rs.mode == 2) {  // a sample outside V_in: dropped, an empty record
        const int p = __float_as_int(__ldg(Rs.sf + r).w);
        if (p >= 0 && p < V.P && V.cls[p] != 2) {
            rec[r] = make_float4(0.f, 0.f, 0.f, V.depth_max);
            return;
        }
    }
    if (!ray_of<kLive>(V, F, Rs, r, s_lo, s_hi, slot, o, d)) return;  // flagged by the trace kernel
    int2 hv = hit[slot];
    uint32_t h = (uint32_t)hv.x;
    float4 out;
    float lo = 0.0f;
    if (h == kMiss) {
        lo = fa(fa(fm(kLumR, F.sky[0]), fm(kLumG, F.sky[1])), fm(kLumB, F.sky[2]));
        out = make_float4(F.sky[0], F.sky[1], F.sky[2], V.depth_max);
    } else {
        float t = __int_as_float(hv.y);
        float depth = fminf(t, V.depth_max);
        if (h & kBackBit) {
            out = make_float4(0.f, 0.f, 0.f, depth);
        } else {
            int tri = (int)h;
            float3 n = tri_normal<kLive>(S, tri);
            float3 x = make_float3(fa(o.x, fm(t, d.x)), fa(o.y, fm(t, d.y)), fa(o.z, fm(t, d.z)));
            unsigned long long vm = vis[slot];
            float E0 = 0.f, E1 = 0.f, E2 = 0.f;
            for (int l = 0; l < L.n; ++l) {
                if (!((vm >> l) & 1ull)) continue;
                const Light& Li = L.l[l];
                float g;
                if (Li.kind == 0) {
                    float dx = fs(Li.v[0], x.x), dy = fs(Li.v[1], x.y), dz = fs(Li.v[2], x.z);
                    float d2 = dot3x(dx, dy, dz, dx, dy, dz);
                    float nd = dot3x(n.x, n.y, n.z, dx, dy, dz);
                    g = nd > 0.0f ? fd(nd, fm(d2, fsq(d2))) : 0.0f;
                } else {
                    float ndD = dot3x(n.x, n.y, n.z, -Li.v[0], -Li.v[1], -Li.v[2]);
                    float l2 = dot3x(Li.v[0], Li.v[1], Li.v[2], Li.v[0], Li.v[1], Li.v[2]);
                    g = fd(ndD, fsq(l2));
                }
                E0 = fa(E0, fm(Li.rgb[0], g));
                E1 = fa(E1, fm(Li.rgb[1], g));
                E2 = fa(E2, fm(Li.rgb[2], g));
            }
            const float a0 = __ldg(S.albedo + 3 * (size_t)tri), a1 = __ldg(S.albedo + 3 * (size_t)tri + 1),
                        a2 = __ldg(S.albedo + 3 * (size_t)tri + 2);
            float r0 = fm(fm(a0, kInvPi), E0), r1 = fm(fm(a1, kInvPi), E1), r2 = fm(fm(a2, kInvPi), E2);
            lo = fa(fa(fm(kLumR, r0), fm(kLumG, r1)), fm(kLumB, r2));
            if (bounce) {
                float3 Q = query_irr_hit(V, irr, dep, o, t, d, n);
                r0 += a0 * Q.x;
                r1 += a1 * Q.y;
                r2 += a2 * Q.z;
            }
            out = make_float4(r0, r1, r2, depth);
        }
    }
    rec[slot] = out;
    if (lum) lum[slot] = lo;
}

}  // namespace

}  // namespace adgi
