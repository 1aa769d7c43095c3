// trace.cu -- probe-ray tracing and shading kernels (sm_103a, SIMT FP32).
//
// Wavefront layout: one kernel finds the nearest hit of every ray, a second
// shades the hits (shadow rays to each light, then the multi-bounce term read
// from the previous frame's atlases).  Rays of a probe are contiguous, so a
// warp shares an origin and sweeps a spiral of nearby directions.
#include <algorithm>
#include <atomic>

#include "adgi_internal.cuh"
#include "kernels.cuh"
#include "wave.cuh"

namespace adgi {

namespace {

__global__ void k_set_frame(FrameDev* __restrict__ dst, const __grid_constant__ FrameDev src)
{
    const int* a = reinterpret_cast<const int*>(&src);
    int* b = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(FrameDev) / sizeof(int)); i += blockDim.x) b[i] = a[i];
}

// The two ray kernels run a grid the GPU holds at once; each warp takes the
// next item of 32 rays from the counter *next (zero before the launch), so
// a warp that drew short rays takes more items and the warps end together.
__device__ __forceinline__ unsigned next_item(unsigned* next)
{
    unsigned w = 0;
    if ((threadIdx.x & 31u) == 0) w = atomicAdd(next, 1u);
    return __shfl_sync(0xFFFFFFFFu, w, 0);
}

// item w: launch threads [32 w, 32 w + 32) of the pilot-ray layout
__global__ void __launch_bounds__(256, 4) k_pilot_trace(VolConst V, const FrameDev* __restrict__ FD, SceneDev S,
                                                     int2* __restrict__ hit, unsigned* next, uint32_t items)
{
    for (;;) {
        const unsigned w = next_item(next);
        if (w >= items) break;
        pilot_trace_body(V, FD, S, hit, (int)(32u * w + (threadIdx.x & 31u)));
        __syncwarp();
    }
}

// item w: adaptive rays [off[p_lo] + 32 w, off[p_lo] + 32 w + 32)
__global__ void __launch_bounds__(256, 4) k_main_trace(VolConst V, const FrameDev* __restrict__ FD, SceneDev S,
                                                    const uint32_t* __restrict__ off, const float4* __restrict__ sf,
                                                    uint32_t R, int2* __restrict__ hit, unsigned* next)
{
    const uint32_t rb = __ldg(off + V.p_lo), re = min(__ldg(off + V.p_hi), R);
    const uint32_t items = re > rb ? (re - rb + 31u) / 32u : 0u;
    for (;;) {
        const unsigned w = next_item(next);
        if (w >= items) break;
        main_trace_warp_body<false>(V, FD, S, off, sf, R, hit, w);
        __syncwarp();
    }
}

// Metropolis samples, in grouped order: thread r < n traces sample r along +w
// into hit_pos[r], thread n + r along -w into hit_neg[r] (the visibility ray
// of the texel at -w).
__global__ void __launch_bounds__(256) k_mh_trace(VolConst V, SceneDev S, const float4* __restrict__ smp_g,
                                                  const float4* __restrict__ smp_gn, uint32_t n,
                                                  int2* __restrict__ hit_pos, int2* __restrict__ hit_neg)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n) return;
    const bool neg = r >= n;
    const uint32_t q = neg ? r - n : r;
    int2* dst = neg ? hit_neg : hit_pos;
    const float4 a = __ldg(smp_g + q);
    const int p = __float_as_int(a.w);
    if (p < 0 || p >= V.P) {
        atomicOr(V.err, kErrRayRange);
        dst[q] = make_int2((int)kMiss, 0x7F800000);
        return;
    }
    if (V.cls[p] != 2) {  // a sample outside V_in is dropped
        dst[q] = make_int2((int)kMiss, 0x7F800000);
        return;
    }
    float3 d = make_float3(a.x, a.y, a.z);
    if (neg) {  // the -w ray: its own direction when snapped to a texel centre
        const float4 b = smp_gn ? __ldg(smp_gn + q) : make_float4(-a.x, -a.y, -a.z, 0.f);
        d = make_float3(b.x, b.y, b.z);
    }
    float t;
    uint32_t h;
    trace_closest(S, probe_pos(V, p), d, V.tmin, __int_as_float(0x7F800000), t, h);
    dst[q] = make_int2((int)h, __float_as_int(t));
}

// Dynamic rays (grouped by probe; r beyond this frame's rays does nothing)
__global__ void __launch_bounds__(256) k_dyn_trace(VolConst V, SceneDev S, DynRays R, uint32_t budget,
                                                   int2* __restrict__ hit)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= budget) return;
    int p, t;
    float3 d;
    if (!dyn_ray_of(V, R, r, p, t, d)) return;
    float th;
    uint32_t h;
    trace_closest(S, probe_pos(V, p), d, V.tmin, __int_as_float(0x7F800000), th, h);
    hit[r] = make_int2((int)h, __float_as_int(th));
}

// Re-trace the last update's rays with work counters (roofline accounting).
// Metropolis volumes (smp_g given): the R = 2B rays after the pilots are the
// samples' +w rays (with their shadow rays) and then their -w rays.
__global__ void __launch_bounds__(128) k_count(VolConst V, const FrameDev* __restrict__ FD, SceneDev S,
                                               const uint32_t* __restrict__ off, const float4* __restrict__ sf,
                                               uint32_t R, unsigned long long* __restrict__ out,
                                               const float4* __restrict__ smp_g)
{
    const FrameConst& F = FD->F;
    const LightSet& L = FD->L;
    __shared__ int s_lo, s_hi;
    const uint32_t NP = (uint32_t)V.P * kPilots;
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    // the main-ray part of this block, for the probe search
    uint32_t b0 = blockIdx.x * blockDim.x;
    uint32_t m0r = b0 > NP ? b0 - NP : 0u;
    uint32_t m1r = min(R ? R - 1 : 0u, (b0 + blockDim.x - 1 > NP ? b0 + blockDim.x - 1 - NP : 0u));
    if (R && !smp_g) block_probe_range(off, V.P, m0r, m1r, &s_lo, &s_hi);
    uint32_t cv = 0, ct = 0, sv = 0, st = 0, sblk = 0, sn = 0;
    if (r < NP + R) {
        float3 org, d;
        bool ok = true, shadows = true;
        if (r < NP) {
            int p = r >> 3;
            ok = V.cls[p] != 0;  // no pilots outside V_out
            org = probe_pos(V, p);
            d = pilot_dir(F.pilot_key, (uint32_t)p, r & 7);
        } else if (smp_g) {
            const uint32_t q = r - NP, n = R / 2;
            const bool neg = q >= n;
            const float4 a = __ldg(smp_g + (neg ? q - n : q));
            const int p = __float_as_int(a.w);
            ok = p >= 0 && p < V.P;
            shadows = !neg;
            org = probe_pos(V, ok ? p : 0);
            d = neg ? make_float3(-a.x, -a.y, -a.z) : make_float3(a.x, a.y, a.z);
        } else {
            uint32_t q = r - NP;
            int p = probe_of_ray(off, q, s_lo, s_hi);
            uint32_t base = __ldg(off + p), m = __ldg(off + p + 1) - base;
            ok = q < __ldg(off + V.P) && m <= (uint32_t)(V.rays_max - kPilots) && q - base < m;
            org = probe_pos(V, p);
            uint32_t i;
            if (ok) d = main_dir(F, sf, m, q - base, &i);
        }
        if (ok) {
            float t;
            uint32_t h;
            trace_closest(S, org, d, V.tmin, __int_as_float(0x7F800000), t, h, &cv, &ct);
            if (shadows && h != kMiss && !(h & kBackBit)) {
                int tri = (int)h;
                float4 A = __ldg(S.tri_orig + 3 * (size_t)tri), B = __ldg(S.tri_orig + 3 * (size_t)tri + 1),
                       C = __ldg(S.tri_orig + 3 * (size_t)tri + 2);
                float e1x = fs(B.x, A.x), e1y = fs(B.y, A.y), e1z = fs(B.z, A.z);
                float e2x = fs(C.x, A.x), e2y = fs(C.y, A.y), e2z = fs(C.z, A.z);
                float cx = fs(fm(e1y, e2z), fm(e1z, e2y));
                float cy = fs(fm(e1z, e2x), fm(e1x, e2z));
                float cz = fs(fm(e1x, e2y), fm(e1y, e2x));
                float cl = fsq(dot3x(cx, cy, cz, cx, cy, cz));
                float3 n = cl > 0.0f ? make_float3(fd(cx, cl), fd(cy, cl), fd(cz, cl)) : make_float3(0.f, 0.f, 1.f);
                float3 x = make_float3(fa(org.x, fm(t, d.x)), fa(org.y, fm(t, d.y)), fa(org.z, fm(t, d.z)));
                float3 xs = make_float3(fa(x.x, fm(V.tmin, n.x)), fa(x.y, fm(V.tmin, n.y)), fa(x.z, fm(V.tmin, n.z)));
                for (int l = 0; l < L.n; ++l) {
                    const Light& Li = L.l[l];
                    float3 D = Li.kind == 0 ? make_float3(fs(Li.v[0], xs.x), fs(Li.v[1], xs.y), fs(Li.v[2], xs.z))
                                            : make_float3(-Li.v[0], -Li.v[1], -Li.v[2]);
                    float thi = Li.kind == 0 ? 1.0f : __int_as_float(0x7F800000);
                    if (!(dot3x(n.x, n.y, n.z, D.x, D.y, D.z) > 0.0f)) continue;
                    sblk += trace_any(S, xs, D, 0.0f, thi, &sv, &st) ? 1u : 0u;
                    ++sn;
                }
            }
        }
    }
    const bool main_ray = r >= NP && r < NP + R;
    // SIMT bound of the main rays' traversal: a warp runs as many node visits
    // as its longest ray, so sum(visits) / (32 x sum of warp maxima) is the
    // lane efficiency that the ray lengths alone allow
    {
        const uint32_t mv = __reduce_max_sync(0xFFFFFFFFu, main_ray ? cv : 0u);
        const uint32_t nr = __popc(__ballot_sync(0xFFFFFFFFu, main_ray));
        const uint32_t nb = __reduce_add_sync(0xFFFFFFFFu, main_ray ? sblk : 0u);
        const uint32_t ns = __reduce_add_sync(0xFFFFFFFFu, main_ray ? sn : 0u);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(out + 8, 32ull * mv);
            atomicAdd(out + 9, (unsigned long long)nr);
            atomicAdd(out + 10, (unsigned long long)nb);
            atomicAdd(out + 11, (unsigned long long)ns);
        }
    }
    unsigned long long* o4 = out;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        bool mine = (part == 1) == main_ray;
        unsigned long long a = __reduce_add_sync(0xFFFFFFFFu, mine ? cv : 0u);
        unsigned long long b = __reduce_add_sync(0xFFFFFFFFu, mine ? ct : 0u);
        unsigned long long c = __reduce_add_sync(0xFFFFFFFFu, mine ? sv : 0u);
        unsigned long long e = __reduce_add_sync(0xFFFFFFFFu, mine ? st : 0u);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(o4 + 4 * part + 0, a);
            atomicAdd(o4 + 4 * part + 1, b);
            atomicAdd(o4 + 4 * part + 2, c);
            atomicAdd(o4 + 4 * part + 3, e);
        }
    }
}

__global__ void k_trace_list(SceneDev S, const float* __restrict__ o, const float* __restrict__ d, int n, float tmin,
                             float tmax, float* __restrict__ t_out, int* __restrict__ tri_out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 org = make_float3(o[3 * (size_t)i], o[3 * (size_t)i + 1], o[3 * (size_t)i + 2]);
    float3 dir = make_float3(d[3 * (size_t)i], d[3 * (size_t)i + 1], d[3 * (size_t)i + 2]);
    float t;
    uint32_t h;
    trace_closest(S, org, dir, tmin, tmax, t, h);
    t_out[i] = t;
    tri_out[i] = (int)h;
}

}  // namespace

// kernel-node parameters of k_set_frame (args[0] -> *dst_slot, args[1] -> src)
void set_frame_node_params(FrameDev** dst_slot, const FrameDev* src, cudaKernelNodeParams* kp, void** args)
{
    args[0] = (void*)dst_slot;
    args[1] = (void*)src;
    kp->func = (void*)k_set_frame;
    kp->gridDim = dim3(1, 1, 1);
    kp->blockDim = dim3(256, 1, 1);
    kp->sharedMemBytes = 0;
    kp->kernelParams = args;
    kp->extra = nullptr;
}

cudaError_t launch_set_frame(FrameDev* dst, const FrameDev& src, cudaStream_t s)
{
    k_set_frame<<<1, 256, 0, s>>>(dst, src);
    count_launches(1);
    return cudaGetLastError();
}

// Blocks of b threads (a multiple of 32, at most 256) that the current GPU
// holds at once for kernel `which` (0 pilot, 1 adaptive trace): asked of the
// runtime once per device, kernel and block size, then kept.
static unsigned resident_blocks(int which, int b)
{
    constexpr int kDevs = 16, kSizes = 8;
    static std::atomic<unsigned> cache[kDevs][2][kSizes];
    int dev = 0;
    cudaGetDevice(&dev);
    const int si = b / 32 - 1;
    const bool keep = dev >= 0 && dev < kDevs && si >= 0 && si < kSizes && b % 32 == 0;
    if (keep) {
        const unsigned c = cache[dev][which][si].load(std::memory_order_relaxed);
        if (c) return c;
    }
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (which == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pilot_trace, b, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_main_trace, b, 0);
    if (sms <= 0) sms = 152;
    if (per <= 0) per = 1;
    const unsigned n = (unsigned)(sms * per);
    if (keep) cache[dev][which][si].store(n, std::memory_order_relaxed);
    return n;
}

cudaError_t launch_pilot_trace(const VolConst& V, const FrameDev* FD, const SceneDev& S, int2* hit, unsigned* next,
                               const Tuning& T, cudaStream_t s)
{
    const int n = ((V.p_hi - V.p_lo + 31) / 32) * 32 * kPilots, b = T.trace_block;
    if (n <= 0) return cudaSuccess;
    const uint32_t items = (uint32_t)n / 32u;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const unsigned g = std::min(resident_blocks(0, b), (items * 32u + (unsigned)b - 1u) / (unsigned)b);
    k_pilot_trace<<<g, b, 0, s>>>(V, FD, S, hit, next, items);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_main_trace(const VolConst& V, const FrameDev* FD, const SceneDev& S, const uint32_t* off,
                              const float4* sf, uint32_t R, int2* hit, unsigned* next, const Tuning& T,
                              cudaStream_t s)
{
    if (R == 0) return cudaSuccess;
    const unsigned b = (unsigned)T.trace_block;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const unsigned g = std::min(resident_blocks(1, (int)b), (R + b - 1) / b);
    k_main_trace<<<g, b, 0, s>>>(V, FD, S, off, sf, R, hit, next);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mh_trace(const VolConst& V, const SceneDev& S, const MhBufs& M, int2* hit_pos, int2* hit_neg,
                            const Tuning& T, cudaStream_t s)
{
    const uint32_t n = M.n_samples;
    if (n == 0) return cudaSuccess;
    const unsigned b = (unsigned)T.trace_block;
    k_mh_trace<<<(2 * n + b - 1) / b, b, 0, s>>>(V, S, M.smp_g, M.smp_gn, n, hit_pos, hit_neg);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dyn_trace(const VolConst& V, const SceneDev& S, const DynRays& R, uint32_t budget, int2* hit,
                             const Tuning& T, cudaStream_t s)
{
    if (budget == 0) return cudaSuccess;
    const unsigned b = (unsigned)T.trace_block;
    k_dyn_trace<<<(budget + b - 1) / b, b, 0, s>>>(V, S, R, budget, hit);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count(const VolConst& V, const FrameDev* FD, const SceneDev& S, const uint32_t* off,
                         const float4* sf, uint32_t R, unsigned long long* out, cudaStream_t s, const float4* smp_g)
{
    uint32_t n = (uint32_t)V.P * kPilots + R;
    k_count<<<(n + 127) / 128, 128, 0, s>>>(V, FD, S, off, sf, R, out, smp_g);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trace_list(const SceneDev& S, const float* o, const float* d, int n, float tmin, float tmax,
                              float* t_out, int* tri_out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_trace_list<<<(n + 127) / 128, 128, 0, s>>>(S, o, d, n, tmin, tmax, t_out, tri_out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adgi
