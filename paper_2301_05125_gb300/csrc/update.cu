// update.cu -- heuristics, ray allocation, blend and query kernels (sm_103a).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include <cooperative_groups.h>

#include "adgi_internal.cuh"
#include "kernels.cuh"

namespace adgi {

namespace {

// ============================================================== heuristics
// Sec. 4.1: q_v from the pilot ray of the opposite octant (f_v = exp(-2t/s),
// t = trace(p, -w)); q_r from the direct-light luminance of the octant's own
// pilot ray (f_r = min(r, 5)/5); temporal trigger (Fig. TrCam(a)).
__device__ __forceinline__ uint32_t qr_of(float lum)
{
    float c = lum < 5.0f ? lum : 5.0f;
    if (!(c > 0.0f)) return 0u;
    float q = floorf(fd(fm(c, 1023.0f), 5.0f));
    return q > 1023.0f ? 1023u : (uint32_t)q;
}

__device__ __forceinline__ uint16_t trigger(uint16_t& amp, uint8_t& age, int delta, int theta)
{
    int a = age;
    if (a < theta) a += 1;
    int cur = a < theta ? (int)(((uint32_t)amp * (uint32_t)(theta - a)) / (uint32_t)theta) : 0;
    if (delta > 0 && delta >= cur) {
        amp = (uint16_t)delta;
        a = 0;
        cur = delta;
    }
    age = (uint8_t)(a < theta ? a : theta);
    return (uint16_t)cur;
}

// Clip volumes (Fig. TrCam(b)): with the view-projection M, probe p is in
// the extended frustum |clip_xy| <= L when w > 0 and |c_x|, |c_y| <= L w,
// (c_x, c_y, -, w) = M (p, 1) in FP32 row order; V_in: L = 1.2 and q_c >= 768
// (f_c >= 0.75), V_out: L = 1.4 and q_c >= 512 (f_c >= 0.5).
__device__ __forceinline__ bool in_frustum(const float* m, float3 x, float L)
{
    const float w = fa(fa(fa(fm(m[12], x.x), fm(m[13], x.y)), fm(m[14], x.z)), m[15]);
    const float cx = fa(fa(fa(fm(m[0], x.x), fm(m[1], x.y)), fm(m[2], x.z)), m[3]);
    const float cy = fa(fa(fa(fm(m[4], x.x), fm(m[5], x.y)), fm(m[6], x.z)), m[7]);
    if (!(w > 0.0f)) return false;
    const float lw = fm(L, w);
    return fabsf(cx) <= lw && fabsf(cy) <= lw;
}

__global__ void __launch_bounds__(256) k_classify(VolConst V, const FrameDev* __restrict__ FD,
                                                  const uint16_t* __restrict__ lut_c, uint8_t* __restrict__ cls)
{
    const FrameConst& F = FD->F;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.P) return;
    uint8_t c = 2;
    if (F.has_clip && F.has_camera) {
        const float3 x = probe_pos(V, p);
        const uint32_t qc = qc_of_probe(V, F, lut_c, p);
        c = (qc >= 768u && in_frustum(F.clip, x, 1.2f)) ? 2 : ((qc >= 512u && in_frustum(F.clip, x, 1.4f)) ? 1 : 0);
    }
    cls[p] = c;
}

__global__ void __launch_bounds__(128) k_change_state(VolConst V, const FrameDev* __restrict__ FD, ChangeBufs B)
{
    const FrameConst& F = FD->F;
    int p = V.p_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.p_hi) return;
    uint32_t yv[8], yr[8];
    const uint8_t cl = V.cls[p];
    if (cl == 0) {  // outside V_out: no heuristics this frame; the state waits
        for (int o = 0; o < 8; ++o) {
            const size_t i = (size_t)p * 8 + o;
            B.trv[i] = 0;
            B.trr[i] = 0;
            B.qv[i] = 0;
            B.qr[i] = 0;
            yv[o] = yr[o] = 0u;
        }
        if (F.even) B.vout_even[p] = 0;
        uint4* G4 = reinterpret_cast<uint4*>(B.G + (size_t)p * 8);
        G4[0] = make_uint4(0u, 0u, 0u, 0u);
        G4[1] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const bool gradient = !F.even && F.pair_valid && B.vout_even[p];  // both frames of the pair in V_out
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        size_t i = (size_t)p * 8 + o;
        int2 hopp = B.pil_hit[(size_t)p * 8 + (7 - o)];
        uint32_t qt = 4095u;
        if ((uint32_t)hopp.x != kMiss) {
            float q = fm(__int_as_float(hopp.y), V.qv_scale);
            qt = q < 4095.0f ? (uint32_t)floorf(q) : 4095u;
        }
        uint16_t qv = __ldg(B.lut_v + qt);
        uint16_t qr = (uint16_t)qr_of(B.pil_lum[i]);
        int dv = 0, dr = 0;
        if (gradient) {
            dv = abs((int)qv - (int)B.qv_even[i]);
            dr = abs((int)qr - (int)B.qr_even[i]);
        }
        uint16_t av = B.amp_v[i], ar = B.amp_r[i];
        uint8_t gv = B.age_v[i], gr = B.age_r[i];
        yv[o] = trigger(av, gv, dv, V.theta);
        yr[o] = trigger(ar, gr, dr, V.theta);
        B.amp_v[i] = av;
        B.amp_r[i] = ar;
        B.age_v[i] = gv;
        B.age_r[i] = gr;
        B.trv[i] = (uint16_t)yv[o];
        B.trr[i] = (uint16_t)yr[o];
        B.qv[i] = qv;
        B.qr[i] = qr;
        if (F.even) {
            B.qv_even[i] = qv;
            B.qr_even[i] = qr;
        }
    }
    if (F.even) B.vout_even[p] = 1;
    uint32_t g[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        g[o] = (yv[o] + yv[o ^ 1] + yv[o ^ 2] + yv[o ^ 4]) + 2u * (yr[o] + yr[o ^ 1] + yr[o ^ 2] + yr[o ^ 4]);
    }
    uint4* G4 = reinterpret_cast<uint4*>(B.G + (size_t)p * 8);
    G4[0] = make_uint4(g[0], g[1], g[2], g[3]);
    G4[1] = make_uint4(g[4], g[5], g[6], g[7]);
}

// 5x5x5 box sum of G (clipped to the grid) and composition (Eq. priorDynamic,
// mu = 2, f_c from Eq. cameraD): W_p = min(sum_o (q_c q_v F) >> 20, 2^24-1).
__global__ void __launch_bounds__(128) k_change_weight(VolConst V, const FrameDev* __restrict__ FD, ChangeBufs B)
{
    const FrameConst& F = FD->F;
    int p = V.p_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.p_hi) return;
    const int X = V.dims[0], Y = V.dims[1], Z = V.dims[2];
    int ix = p % X, iy = (p / X) % Y, iz = p / (X * Y);
    uint32_t f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int jz = max(iz - 2, 0); jz <= min(iz + 2, Z - 1); ++jz)
        for (int jy = max(iy - 2, 0); jy <= min(iy + 2, Y - 1); ++jy)
            for (int jx = max(ix - 2, 0); jx <= min(ix + 2, X - 1); ++jx) {
                const uint4* G4 = reinterpret_cast<const uint4*>(B.G + ((size_t)jx + (size_t)X * (jy + (size_t)Y * jz)) * 8);
                uint4 a = __ldg(G4), b = __ldg(G4 + 1);
                f[0] += a.x;
                f[1] += a.y;
                f[2] += a.z;
                f[3] += a.w;
                f[4] += b.x;
                f[5] += b.y;
                f[6] += b.z;
                f[7] += b.w;
            }
    const uint32_t qc = qc_of_probe(V, F, B.lut_c, p);
    uint64_t Wp = 0;
    const bool vin = V.cls[p] == 2;  // only V_in probes take adaptive samples
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const uint64_t qd = vin ? ((uint64_t)qc * (uint64_t)B.qv[(size_t)p * 8 + o] * (uint64_t)f[o]) >> 20 : 0ull;
        if (B.qd) B.qd[(size_t)p * 8 + o] = (uint32_t)(qd < 0xFFFFFFFFull ? qd : 0xFFFFFFFFull);
        Wp += qd;
    }
    B.W[p] = (uint32_t)(Wp < 0xFFFFFFull ? Wp : 0xFFFFFFull);
}

// ============================================================== allocation
// One CTA of 1024 threads; thread t owns the contiguous probe chunk
// [t*chunk, (t+1)*chunk).  Integer water-filling of the extra budget by W,
// capped, then the remainder one ray per probe in index order.
constexpr int kAllocThreads = 1024;
constexpr int kAllocIters = 64;

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t* red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        uint64_t x = lane < (int)(blockDim.x >> 5) ? red[lane] : 0ull;
        x = warp_sum(x);
        if (lane == 0) red[32] = x;
    }
    __syncthreads();
    return red[32];
}

// block sums of two values at once (one round of barriers)
__device__ __forceinline__ void block_sum2(uint64_t& a, uint64_t& b, uint64_t* red)
{
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if (lane == 0) red[w] = a, red[32 + w] = b;
    __syncthreads();
    if (w == 0) {
        uint64_t x = lane < nw ? red[lane] : 0ull, y = lane < nw ? red[32 + lane] : 0ull;
        x = warp_sum(x);
        y = warp_sum(y);
        if (lane == 0) red[64] = x, red[65] = y;
    }
    __syncthreads();
    a = red[64];
    b = red[65];
}

// exclusive prefix of v over threads in index order; *total receives the sum
__device__ __forceinline__ uint64_t block_exscan(uint64_t v, uint64_t* red, uint64_t* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) red[w] = x;
    __syncthreads();
    if (w == 0) {
        uint64_t s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        red[lane] = s;  // inclusive prefix of warp totals
    }
    __syncthreads();
    uint64_t before = (w > 0 ? red[w - 1] : 0ull) + (x - v);
    *total = red[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// With clip volumes (cls given) only V_in probes (cls 2) take adaptive rays:
// floors m0 in V_in, 8 (the pilots) in V_out - V_in, 0 outside; beyond the
// V_in floors E = (avg - 8) P - (m0 - 8) |V_in| is spread over V_in, capped
// at rmax - m0 per probe.  Without cls every probe is in V_in and E =
// (avg - m0) P.
// floor(x / d) for d >= 1 from inv = floor((2^64 - 1) / d): the high word of
// x inv is floor(x / d) or at most two less (the error of inv is below one
// part in d, that of the product below 2), and the remainder check corrects it
__device__ __forceinline__ uint64_t div_by(uint64_t x, uint64_t d, uint64_t inv)
{
    uint64_t q = __umul64hi(x, inv), r = x - q * d;
    if (r >= d) ++q, r -= d;
    if (r >= d) ++q;
    return q;
}

// One block over global memory, for grids beyond what a cluster stages
// (k_allocate_cluster below).  A probe outside V_in starts with its extras
// at the cap and weight 0, so it is never eligible: every test below is
// w > 0 / n < cap.
__global__ void __launch_bounds__(kAllocThreads, 1) k_allocate(const uint32_t* __restrict__ Win, int P, int avg, int m0,
                                                            int rmax, uint32_t* __restrict__ n, uint32_t* __restrict__ off,
                                                            const uint8_t* __restrict__ cls)
{
    __shared__ uint64_t red[66];
    const int chunk = (P + kAllocThreads - 1) / kAllocThreads;
    const int c0 = min(P, (int)threadIdx.x * chunk), c1 = min(P, c0 + chunk);
    const uint32_t cap = (uint32_t)(rmax - m0);
    uint32_t* nx = n;  // extra rays beyond the floor, then the rays
    auto vin = [&](int p) { return !cls || cls[p] == 2; };
    auto w_of = [&](int p) -> uint32_t { return vin(p) ? __ldg(Win + p) : 0u; };
    uint64_t pin = 0, s = 0;
    for (int p = c0; p < c1; ++p) {
        const bool in = vin(p);
        pin += in ? 1u : 0u;
        s += in ? __ldg(Win + p) : 0u;
        nx[p] = in ? 0u : cap;
    }
    uint64_t Pin;
    const uint64_t rank0 = block_exscan(pin, red, &Pin);  // V_in rank of this chunk's first V_in probe
    const uint64_t S = block_sum(s, red);                  // also orders the staging writes before the reads
    uint64_t E = (uint64_t)(avg - 8) * (uint64_t)P - (uint64_t)(m0 - 8) * Pin;
    if (E > Pin * cap) E = Pin * cap;
    if (S == 0) {  // uniform over V_in, the remainder to the lowest V_in ranks
        const uint64_t q = Pin ? E / Pin : 0, r = Pin ? E % Pin : 0;
        uint64_t rank = rank0;
        for (int p = c0; p < c1; ++p) {
            if (!vin(p)) continue;
            nx[p] = (uint32_t)(q + (rank < r ? 1u : 0u));
            ++rank;
        }
    } else {
        // proportional passes: SU = the weight of the probes below their cap
        // (at first every V_in probe: S, unless the cap is 0); the pass that
        // hands out shares also sums SU for the next pass
        uint64_t Erem = E, SU = cap > 0u ? S : 0u;
        for (int it = 0; it < kAllocIters; ++it) {
            if (SU == 0 || Erem == 0) break;
            const uint64_t inv = 0xFFFFFFFFFFFFFFFFull / SU;
            uint64_t G = 0, su = 0;
            for (int p = c0; p < c1; ++p) {
                const uint32_t w = w_of(p), e = nx[p];
                if (w == 0u || e >= cap) continue;
                const uint64_t share = div_by(Erem * (uint64_t)w, SU, inv);
                const uint64_t room = cap - e;
                const uint64_t a = share < room ? share : room;
                nx[p] = e + (uint32_t)a;
                G += a;
                if (a < room) su += w;  // still below the cap after this pass
            }
            block_sum2(G, su, red);
            if (G == 0) break;
            Erem -= G;
            SU = su;
        }
        // remainder: one each, probe-index order, probes with W > 0 first
        for (int guard = 0; Erem > 0 && guard < (1 << 20); ++guard) {
            uint64_t ca = 0;
            for (int p = c0; p < c1; ++p)
                if (w_of(p) > 0u && nx[p] < cap) ++ca;
            const bool modeA = block_sum(ca, red) > 0;
            uint64_t ce = 0;
            for (int p = c0; p < c1; ++p)
                if (nx[p] < cap && (!modeA || w_of(p) > 0u)) ++ce;
            uint64_t tot;
            uint64_t pre = block_exscan(ce, red, &tot);
            if (tot == 0) break;
            for (int p = c0; p < c1; ++p) {
                if (nx[p] < cap && (!modeA || w_of(p) > 0u)) {
                    if (pre < Erem) nx[p] += 1u;
                    ++pre;
                }
            }
            Erem -= tot < Erem ? tot : Erem;
        }
    }
    // rays per probe: the floor plus the extra; adaptive rays = rays - 8 (0 outside V_in)
    auto rays_of = [&](int p) -> uint32_t {
        if (vin(p)) return (uint32_t)m0 + nx[p];
        return cls[p] == 1 ? 8u : 0u;
    };
    uint64_t loc = 0;
    for (int p = c0; p < c1; ++p) {
        const uint32_t np = rays_of(p);
        loc += np > 8u ? np - 8u : 0u;
    }
    uint64_t tot;
    uint64_t pre = block_exscan(loc, red, &tot);
    for (int p = c0; p < c1; ++p) {
        const uint32_t np = rays_of(p);
        off[p] = (uint32_t)pre;
        pre += np > 8u ? np - 8u : 0u;
        n[p] = np;
    }
    if (threadIdx.x == 0) off[P] = (uint32_t)tot;
}

// The same allocation on a cluster of kAllocCluster CTAs, for grids of up
// to kAllocClusterMaxP probes: CTA r stages and works on the r-th slice of
// the probes, so each pass's loops are kAllocCluster times shorter.  A
// cluster-wide sum is the CTAs' block sums, published in their shared
// memory and added by every thread in rank order after a cluster barrier
// (integer sums: the same totals everywhere).  Every loop bound and break
// below depends only on such totals, so all threads pass the same sequence
// of barriers.  The partials are double-buffered: a CTA can run at most one
// reduction ahead of the slowest reader.
namespace cg = cooperative_groups;
constexpr int kAllocCluster = 8;
constexpr int kAllocClusterMaxP = kAllocCluster * 24576;  // 8 B a probe: at most 192 KB of shared memory per CTA

struct ClusterSums {
    uint64_t* slot;  // this CTA's partials: [2 buffers][4]
    int buf;
};

__device__ __forceinline__ void cluster_sum2(cg::cluster_group& cl, ClusterSums& C, uint64_t* red, uint64_t& a,
                                             uint64_t& b)
{
    block_sum2(a, b, red);
    if (threadIdx.x == 0) C.slot[4 * C.buf] = a, C.slot[4 * C.buf + 1] = b;
    cl.sync();
    uint64_t ta = 0, tb = 0;
    for (int r = 0; r < kAllocCluster; ++r) {
        const uint64_t* rs = cl.map_shared_rank(C.slot, r);
        ta += rs[4 * C.buf];
        tb += rs[4 * C.buf + 1];
    }
    C.buf ^= 1;
    a = ta;
    b = tb;
}

__device__ __forceinline__ uint64_t cluster_exscan(cg::cluster_group& cl, ClusterSums& C, uint64_t* red, uint64_t v,
                                                   uint64_t* total)
{
    uint64_t bt;
    const uint64_t pre = block_exscan(v, red, &bt);
    if (threadIdx.x == 0) C.slot[4 * C.buf + 2] = bt;
    cl.sync();
    const int me = (int)cl.block_rank();
    uint64_t below = 0, all = 0;
    for (int r = 0; r < kAllocCluster; ++r) {
        const uint64_t t = cl.map_shared_rank(C.slot, r)[4 * C.buf + 2];
        below += r < me ? t : 0ull;
        all += t;
    }
    C.buf ^= 1;
    *total = all;
    return below + pre;
}

__global__ void __cluster_dims__(kAllocCluster, 1, 1) __launch_bounds__(kAllocThreads, 1)
    k_allocate_cluster(const uint32_t* __restrict__ Win, int P, int avg, int m0, int rmax, uint32_t* __restrict__ n,
                       uint32_t* __restrict__ off, const uint8_t* __restrict__ cls)
{
    cg::cluster_group cl = cg::this_cluster();
    __shared__ uint64_t red[66];
    __shared__ uint64_t slot[8];
    extern __shared__ uint32_t stage[];  // [Pc] weights, then [Pc] extras of this CTA's slice
    ClusterSums C{slot, 0};
    const int rank = (int)cl.block_rank();
    const int Pc = (P + kAllocCluster - 1) / kAllocCluster;
    const int b0 = min(P, rank * Pc), b1 = min(P, b0 + Pc);
    const int chunk = (b1 - b0 + kAllocThreads - 1) / kAllocThreads;
    const int c0 = min(b1, b0 + (int)threadIdx.x * chunk), c1 = min(b1, c0 + chunk);
    const uint32_t cap = (uint32_t)(rmax - m0);
    uint32_t* ws = stage;
    uint32_t* nx = stage + Pc;
    auto vin = [&](int p) { return !cls || cls[p] == 2; };
    uint64_t pin = 0, S = 0, zero = 0;
    for (int p = c0; p < c1; ++p) {
        const bool in = vin(p);
        const uint32_t w = in ? __ldg(Win + p) : 0u;
        pin += in ? 1u : 0u;
        S += w;
        ws[p - b0] = w;
        nx[p - b0] = in ? 0u : cap;
    }
    uint64_t Pin;
    const uint64_t rank0 = cluster_exscan(cl, C, red, pin, &Pin);  // V_in rank of this chunk's first V_in probe
    cluster_sum2(cl, C, red, S, zero);
    uint64_t E = (uint64_t)(avg - 8) * (uint64_t)P - (uint64_t)(m0 - 8) * Pin;
    if (E > Pin * cap) E = Pin * cap;
    if (S == 0) {  // uniform over V_in, the remainder to the lowest V_in ranks
        const uint64_t q = Pin ? E / Pin : 0, r = Pin ? E % Pin : 0;
        uint64_t rk = rank0;
        for (int p = c0; p < c1; ++p) {
            if (!vin(p)) continue;
            nx[p - b0] = (uint32_t)(q + (rk < r ? 1u : 0u));
            ++rk;
        }
    } else {
        uint64_t Erem = E, SU = cap > 0u ? S : 0u;
        for (int it = 0; it < kAllocIters; ++it) {
            if (SU == 0 || Erem == 0) break;
            const uint64_t inv = 0xFFFFFFFFFFFFFFFFull / SU;
            uint64_t G = 0, su = 0;
            for (int p = c0; p < c1; ++p) {
                const uint32_t w = ws[p - b0], e = nx[p - b0];
                if (w == 0u || e >= cap) continue;
                const uint64_t share = div_by(Erem * (uint64_t)w, SU, inv);
                const uint64_t room = cap - e;
                const uint64_t a = share < room ? share : room;
                nx[p - b0] = e + (uint32_t)a;
                G += a;
                if (a < room) su += w;
            }
            cluster_sum2(cl, C, red, G, su);
            if (G == 0) break;
            Erem -= G;
            SU = su;
        }
        for (int guard = 0; Erem > 0 && guard < (1 << 20); ++guard) {
            uint64_t ca = 0;
            for (int p = c0; p < c1; ++p)
                if (ws[p - b0] > 0u && nx[p - b0] < cap) ++ca;
            cluster_sum2(cl, C, red, ca, zero);
            const bool modeA = ca > 0;
            uint64_t ce = 0;
            for (int p = c0; p < c1; ++p)
                if (nx[p - b0] < cap && (!modeA || ws[p - b0] > 0u)) ++ce;
            uint64_t tot;
            uint64_t pre = cluster_exscan(cl, C, red, ce, &tot);
            if (tot == 0) break;
            for (int p = c0; p < c1; ++p) {
                if (nx[p - b0] < cap && (!modeA || ws[p - b0] > 0u)) {
                    if (pre < Erem) nx[p - b0] += 1u;
                    ++pre;
                }
            }
            Erem -= tot < Erem ? tot : Erem;
        }
    }
    auto rays_of = [&](int p) -> uint32_t {
        if (vin(p)) return (uint32_t)m0 + nx[p - b0];
        return cls[p] == 1 ? 8u : 0u;
    };
    uint64_t loc = 0;
    for (int p = c0; p < c1; ++p) {
        const uint32_t np = rays_of(p);
        loc += np > 8u ? np - 8u : 0u;
    }
    uint64_t tot;
    uint64_t pre = cluster_exscan(cl, C, red, loc, &tot);
    for (int p = c0; p < c1; ++p) {
        const uint32_t np = rays_of(p);
        off[p] = (uint32_t)pre;
        pre += np > 8u ? np - 8u : 0u;
        n[p] = np;
    }
    if (rank == 0 && threadIdx.x == 0) off[P] = (uint32_t)tot;
    cl.sync();  // no CTA leaves while another may still read its partials
}

// ============================================================== blend
// Alg. ApproxAlgo + Alg. MovingAvgUpdate, batched per texel, in two kernels.
//  plan  (once per frame, one CTA per row m of the SF table): the rotated
//        directions of row m are binned to their nearest irradiance and depth
//        texels and sorted by texel with a stable counting sort; every probe
//        with m adaptive rays shares this plan, because its directions are
//        the same -- binning is done once per direction, not once per ray;
//  blend (one warp per probe tile): L2 prefetch of the probe's records and
//        old tiles (cp.async.bulk.prefetch); each lane takes whole texels and
//        sums the texel's pilot samples (pilot order) and then its bucket of
//        the plan (SF index order), i.e. in sample order, so the result is
//        deterministic with no floating-point atomics; the texel is blended
//        with w = max(1 - h, k/(n+k)) into shared memory, and every texel --
//        border texels from their octahedral fold partner -- is written back
//        with coalesced stores in texel order.  Shared memory per warp is
//        kept small: the kernel is latency bound, so warps per SM count.

// float -> half with stochastic rounding: round toward zero, then step one
// half ulp away from zero with probability equal to the remaining fraction
// (unbiased in expectation; u is a uniform 32-bit hash).  Round-to-nearest
// cannot move an EMA value by less than half an ulp, so with weight 1-h the
// stored value would stop short of the target by up to ulp/(2(1-h)).
__device__ __forceinline__ __half half_sr(float v, uint32_t u)
{
    __half h = __float2half_rz(v);
    float hf = __half2float(h);
    if (hf == v || !(fabsf(v) < 65504.0f)) return __float2half_rn(v);
    __half n = __ushort_as_half((unsigned short)(__half_as_ushort(h) + 1));
    float nf = __half2float(n);
    float frac = (v - hf) / (nf - hf);
    return (float)u * 2.3283064365386963e-10f < frac ? n : h;
}

__device__ __forceinline__ uint32_t sr_bits(uint64_t key, int p, int t, int c)
{
    return (uint32_t)splitmix(key ^ ((uint64_t)p << 24) ^ ((uint64_t)t << 4) ^ (uint64_t)c);
}





// exclusive scan of cnt[0..n) into beg[0..n] (beg[n] = total) and, in place,
// cnt -> running cursors; by one warp
__device__ __forceinline__ void warp_scan_bins(uint32_t* cnt, uint16_t* beg, int n, int lane)
{
    uint32_t carry = 0;
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int b = b0 + lane;
        uint32_t c = b < n ? cnt[b] : 0u, x = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (b < n) {
            beg[b] = (uint16_t)(carry + x - c);
            cnt[b] = carry + x - c;
        }
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) beg[n] = (uint16_t)carry;
}

// stable scatter of indices 0..n-1 by key (index order kept inside a key), by one warp
__device__ __forceinline__ void warp_stable_scatter(const uint16_t* key, uint32_t* cur, uint16_t* ord, int n,
                                                    int lane)
{
    const uint32_t lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int j = c0 + lane;
        const bool valid = j < n;
        const uint32_t k = valid ? (uint32_t)key[j] : 0x10000u + (uint32_t)lane;  // invalid lanes match nobody
        const uint32_t mask = __match_any_sync(0xffffffffu, k);
        uint32_t pos = 0;
        if (valid) pos = cur[k] + (uint32_t)__popc(mask & lt);
        __syncwarp();
        if (valid) {
            ord[pos] = (uint16_t)j;
            if ((mask & lt) == 0u) cur[k] += (uint32_t)__popc(mask);  // lowest lane of the group advances the cursor
        }
        __syncwarp();
    }
}

// Plan of SF row m = blockIdx.x + 1 for this frame's rotation.
__global__ void __launch_bounds__(256) k_blend_plan(VolConst V, const FrameDev* __restrict__ FD,
                                                    const float4* __restrict__ sf, BlendPlan Pl)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int m = blockIdx.x + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x;
    const int ti2 = V.Ti * V.Ti, td2 = V.Td * V.Td;
    uint32_t* cnt_i = reinterpret_cast<uint32_t*>(smem);
    uint32_t* cnt_d = cnt_i + ti2;
    uint16_t* key_i = reinterpret_cast<uint16_t*>(cnt_d + td2);
    uint16_t* key_d = key_i + m;
    for (int t = tid; t < ti2; t += nthr) cnt_i[t] = 0u;
    for (int t = tid; t < td2; t += nthr) cnt_d[t] = 0u;
    __syncthreads();
    const size_t row = (size_t)m * (m - 1) / 2;
    for (int k = tid; k < m; k += nthr) {  // row position k holds SF index .w
        const float4 s4 = __ldg(sf + row + k);
        const int i = __float_as_int(s4.w);
        if (i < 0 || i >= m) {
            atomicOr(V.err, kErrIndex);
            continue;
        }
        const float2 e = oct_encode_x(rotate(F.R, s4));
        const int ki = texel_of(e, V.n_irr), kd = texel_of(e, V.n_dep);
        key_i[i] = (uint16_t)ki;
        key_d[i] = (uint16_t)kd;
        atomicAdd(cnt_i + ki, 1u);  // integer counts: order-independent
        atomicAdd(cnt_d + kd, 1u);
    }
    __syncthreads();
    uint16_t* beg_i = Pl.beg_i + (size_t)(m - 1) * (ti2 + 1);
    uint16_t* beg_d = Pl.beg_d + (size_t)(m - 1) * (td2 + 1);
    if (warp == 0) {
        warp_scan_bins(cnt_i, beg_i, ti2, lane);
        __syncwarp();
        warp_stable_scatter(key_i, cnt_i, Pl.ord_i + row, m, lane);
    }
    if (warp == (nthr > 32 ? 1 : 0)) {
        warp_scan_bins(cnt_d, beg_d, td2, lane);
        __syncwarp();
        warp_stable_scatter(key_d, cnt_d, Pl.ord_d + row, m, lane);
    }
}

size_t blend_plan_smem(const VolConst& V)
{
    const size_t M = (size_t)(V.rays_max - kPilots);
    return 4 * ((size_t)V.Ti * V.Ti + (size_t)V.Td * V.Td) + 4 * M;
}

// shared memory of one probe (one warp) of k_blend: the pilot records and
// bins, and the updated tiles (kept small: the kernel is latency bound, so
// warps per SM matter more than staging)
struct BlendLayout {
    uint32_t prec, pkey, irr_new, dep_new, dn_new, total;
};

__host__ __device__ inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline BlendLayout blend_layout(int Ti, int Td)
{
    const uint32_t ti2 = (uint32_t)(Ti * Ti), td2 = (uint32_t)(Td * Td);
    BlendLayout L;
    uint32_t o = 0;
    L.prec = o, o += 16 * kPilots;
    L.pkey = o, o += 4 * 2 * kPilots;
    L.irr_new = o, o += al16(16 * ti2);
    L.dep_new = o, o += al16(8 * td2);
    L.dn_new = o, o += al16(td2);
    L.total = o;
    return L;
}

// row of texel t in a tile of width T (t < 1024, T <= 32: the product is
// never within 2^-7 of an integer, so single-precision rounding is harmless)
__device__ __forceinline__ int tile_row(int t, float rT) { return (int)(((float)t + 0.5f) * rT); }

// hint: bring [src, src+bytes) into L2 (16-byte aligned address and size)
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---- packed atlases (the paper's 32-bit codecs): one moving-average step
// per sample (Alg. MovingAvgUpdate, serialised in sample order as the CAS
// loop of Alg. atmMvAvgUpd would), each followed by coding the value again.
constexpr uint32_t kPackNmax = 63u;  // 6-bit sample count

// code of v >= 0: the largest k with tab[k] <= v (tab increasing, tab[0] = 0).
// The log estimate only seeds the search; the thresholds decide.
__device__ __forceinline__ uint32_t code_of(const float* __restrict__ tab, int kmax, float beta, float gamma, float v)
{
    if (!(v > 0.0f)) return 0u;
    const float u = fminf(__logf(fmaf(gamma, v, 1.0f)), beta) * ((float)kmax / beta);
    int k = (int)fminf(fmaxf(u, 0.0f), (float)kmax);
    for (int it = 0; it < 3 && k > 0 && __ldg(tab + k) > v; ++it) --k;
    for (int it = 0; it < 3 && k < kmax && __ldg(tab + k + 1) <= v; ++it) ++k;
    if (__ldg(tab + k) > v || (k < kmax && __ldg(tab + k + 1) <= v)) {  // not bracketed yet: bisect
        int lo = 0, hi = kmax;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(tab + mid) <= v)
                lo = mid;
            else
                hi = mid - 1;
        }
        k = lo;
    }
    return (uint32_t)k;
}

// V = v/(n+1) + (n o)/(n+1), FP32, in this order
__device__ __forceinline__ float mav_step(float o, float v, uint32_t n)
{
    const float n1 = (float)(n + 1u);
    return fa(fd(v, n1), fd(fm((float)n, o), n1));
}

struct PkIrr {
    uint32_t k0, k1, k2, n;
    float o0, o1, o2;
    __device__ __forceinline__ void load(const float* ct, uint32_t c)
    {
        k0 = c & 511u, k1 = (c >> 9) & 511u, k2 = (c >> 18) & 255u, n = c >> 26;
        o0 = __ldg(ct + kCt9 + k0), o1 = __ldg(ct + kCt9 + k1), o2 = __ldg(ct + kCt8 + k2);
    }
    __device__ __forceinline__ void add(const float* ct, float r, float g, float b)
    {
        k0 = code_of(ct + kCt9, 511, 5.0f, 15.0f, mav_step(o0, r, n));
        k1 = code_of(ct + kCt9, 511, 5.0f, 15.0f, mav_step(o1, g, n));
        k2 = code_of(ct + kCt8, 255, 5.0f, 15.0f, mav_step(o2, b, n));
        o0 = __ldg(ct + kCt9 + k0), o1 = __ldg(ct + kCt9 + k1), o2 = __ldg(ct + kCt8 + k2);
        n = min(n + 1u, kPackNmax);
    }
    __device__ __forceinline__ uint32_t code() const { return k0 | (k1 << 9) | (k2 << 18) | (n << 26); }
};

struct PkDep {
    uint32_t km, kq, n;
    float om, oq;
    __device__ __forceinline__ void load(const float* ct, uint32_t c)
    {
        km = c & 8191u, kq = (c >> 13) & 8191u, n = c >> 26;
        om = __ldg(ct + kCtM + km), oq = __ldg(ct + kCtQ + kq);
    }
    __device__ __forceinline__ void add(const float* ct, float x)  // x: distance / cage diagonal
    {
        km = code_of(ct + kCtM, 8191, 5.0f, 15.0f, mav_step(om, x, n));
        kq = code_of(ct + kCtQ, 8191, 8.0f, 20.0f, mav_step(oq, fm(x, x), n));
        om = __ldg(ct + kCtM + km), oq = __ldg(ct + kCtQ + kq);
        n = min(n + 1u, kPackNmax);
    }
    __device__ __forceinline__ uint32_t code() const { return km | (kq << 13) | (n << 26); }
};

// One warp, one probe tile, packed atlases: each lane takes whole texels and
// applies their samples in sample order (pilots, then the plan bucket in SF
// index order); then the border fold and coalesced stores of the codes.
__device__ __forceinline__ void blend_packed(const VolConst& V, const BlendBufs& B, int p, uint32_t m, int npil,
                                             const float4* __restrict__ mrec, const float4* prs, const int* pk_i,
                                             const int* pk_d, const uint16_t* __restrict__ ord_i,
                                             const uint16_t* __restrict__ ord_d, const uint16_t* __restrict__ beg_i,
                                             const uint16_t* __restrict__ beg_d, uint32_t* irr_new, uint32_t* dep_new,
                                             int lane)
{
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const int ti2 = Ti * Ti, td2 = Td * Td;
    const float* ct = V.ctab;
    const uint32_t* girr = reinterpret_cast<const uint32_t*>(B.irr) + (size_t)p * ti2;
    const uint32_t* gdep = reinterpret_cast<const uint32_t*>(B.dep) + (size_t)p * td2;
    const float rni = 1.0f / (float)ni, rnd = 1.0f / (float)nd;
    for (int q = lane; q < ni * ni; q += 32) {
        const int r = (int)(((float)q + 0.5f) * rni), t = (r + 1) * Ti + (q - r * ni) + 1;
        PkIrr x;
        x.load(ct, __ldg(girr + t));
        for (int o = 0; o < npil; ++o)
            if (pk_i[o] == t) x.add(ct, prs[o].x, prs[o].y, prs[o].z);
        if (m) {
            const uint32_t b1 = __ldg(beg_i + t + 1);
            for (uint32_t u = __ldg(beg_i + t); u < b1; ++u) {
                const float4 rc = __ldg(mrec + min((uint32_t)__ldg(ord_i + u), m - 1));
                x.add(ct, rc.x, rc.y, rc.z);
            }
        }
        if (V.cls[p] == 1) x.n = min(x.n, 16u);  // V_out - V_in: counts set down to 16
        irr_new[t] = x.code();
    }
    for (int q = lane; q < nd * nd; q += 32) {
        const int r = (int)(((float)q + 0.5f) * rnd), t = (r + 1) * Td + (q - r * nd) + 1;
        PkDep x;
        x.load(ct, __ldg(gdep + t));
        for (int o = 0; o < npil; ++o)
            if (pk_d[o] == t) x.add(ct, fd(prs[o].w, V.s_f));
        if (m) {
            const uint32_t b1 = __ldg(beg_d + t + 1);
            for (uint32_t u = __ldg(beg_d + t); u < b1; ++u)
                x.add(ct, fd(__ldg(&mrec[min((uint32_t)__ldg(ord_d + u), m - 1)].w), V.s_f));
        }
        if (V.cls[p] == 1) x.n = min(x.n, 16u);
        dep_new[t] = x.code();
    }
    __syncwarp();
    uint32_t* oirr = reinterpret_cast<uint32_t*>(B.irr) + (size_t)p * ti2;
    uint32_t* odep = reinterpret_cast<uint32_t*>(B.dep) + (size_t)p * td2;
    for (int t = lane; t < ti2; t += 32) oirr[t] = irr_new[__ldg(B.src + t)];
    for (int t = lane; t < td2; t += 32) odep[t] = dep_new[__ldg(B.src + ti2 + t)];
}

// One texel of the batched moving average (Alg. ApproxAlgo + Alg.
// MovingAvgUpdate): k samples with sums (sx, sy, sz) update {rgb, count}.
__device__ __forceinline__ float4 irr_texel_blend(float4 v, float sx, float sy, float sz, uint32_t k, float omh)
{
    const float kf = (float)k;
    const float w = fmaxf(omh, __fdividef(kf, v.w + kf));
    const float ik = __frcp_rn(kf);
    v.x += w * (sx * ik - v.x);
    v.y += w * (sy * ik - v.y);
    v.z += w * (sz * ik - v.z);
    v.w = fminf(v.w + kf, 255.0f);
    return v;
}

// The depth texel stores {mean, variance}; with batch mean m and batch
// variance vb of k samples the moving average of {d, d^2} becomes
//   mean' = mean + w (m - mean)
//   var'  = (1-w) var + w vb + w (1-w) (m - mean)^2
// (every term non-negative: no cancellation in storage); c is the count.
// The batch arrives as sums s1, s2 of the samples' offsets d - x0 from a
// shift x0 (the texel's first sample): m = x0 + s1/k, vb = s2/k - (s1/k)^2,
// which cancels only at the scale of the samples' spread, not of d^2.
__device__ __forceinline__ float2 dep_texel_blend(float2 v, uint32_t& c, float x0, float s1, float s2, uint32_t k,
                                                  float omh)
{
    const float kf = (float)k;
    const float w = fmaxf(omh, __fdividef(kf, (float)c + kf));
    const float ik = __frcp_rn(kf);
    const float mo = s1 * ik;
    const float mb = x0 + mo;
    const float vb = fmaxf(s2 * ik - mo * mo, 0.0f);
    const float dm = mb - v.x;
    v.y = (1.0f - w) * v.y + w * vb + w * (1.0f - w) * dm * dm;
    v.x += w * dm;
    c = (uint32_t)fminf((float)c + kf, 255.0f);
    return v;
}

// Every texel of probe p's updated tiles (a border texel from its octahedral
// fold partner src[t]) in the storage format, stored in texel order
// (coalesced), by one warp.
__device__ __forceinline__ void store_tiles(const VolConst& V, const FrameConst& F, void* irr, void* dep,
                                            uint8_t* dep_n, const uint16_t* __restrict__ src, int p,
                                            const float4* irr_new, const float2* dep_new, const uint8_t* dn_new,
                                            int lane)
{
    const int ti2 = V.Ti * V.Ti, td2 = V.Td * V.Td;
    const size_t io = (size_t)p * ti2, dof = (size_t)p * td2;
    const uint64_t srkey = F.pilot_key ^ (F.even ? 0x5352ull : 0x5353ull);
    for (int t = lane; t < ti2; t += 32) {
        const float4 v = irr_new[__ldg(src + t)];
        if (V.fp16 == 2) {
            __half2* h = reinterpret_cast<__half2*>(irr) + 2 * (io + t);
            const __half2 h0 = __halves2half2(half_sr(v.x, sr_bits(srkey, p, t, 0)), half_sr(v.y, sr_bits(srkey, p, t, 1)));
            const __half2 h1 = __halves2half2(half_sr(v.z, sr_bits(srkey, p, t, 2)), __float2half_rn(v.w));
            *reinterpret_cast<uint2*>(h) = make_uint2(*reinterpret_cast<const uint32_t*>(&h0),
                                                     *reinterpret_cast<const uint32_t*>(&h1));
        } else if (V.fp16) {
            __half2* h = reinterpret_cast<__half2*>(irr) + 2 * (io + t);
            const __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
            *reinterpret_cast<uint2*>(h) = make_uint2(*reinterpret_cast<const uint32_t*>(&h0),
                                                     *reinterpret_cast<const uint32_t*>(&h1));
        } else {
            reinterpret_cast<float4*>(irr)[io + t] = v;
        }
    }
    for (int t = lane; t < td2; t += 32) {
        const int st = __ldg(src + ti2 + t);
        const float2 v = dep_new[st];
        if (V.fp16 == 2)
            reinterpret_cast<__half2*>(dep)[dof + t] =
                __halves2half2(half_sr(v.x, sr_bits(srkey, p, t, 4)), half_sr(v.y, sr_bits(srkey, p, t, 5)));
        else if (V.fp16)
            reinterpret_cast<__half2*>(dep)[dof + t] = __floats2half2_rn(v.x, v.y);
        else
            reinterpret_cast<float2*>(dep)[dof + t] = v;
        dep_n[dof + t] = dn_new[st];
    }
}

__global__ void __launch_bounds__(128) k_blend(VolConst V, const FrameDev* __restrict__ FD, BlendBufs B)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int p = V.p_lo + blockIdx.x * (blockDim.x >> 5) + wib;
    if (p >= V.p_hi) return;  // the whole warp
    const uint32_t base = __ldg(B.off + p);
    uint32_t m = __ldg(B.off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || base > V.R_main || m > V.R_main - base) {
        if (lane == 0) atomicOr(V.err, kErrRayRange);
        m = 0;
    }
    const uint8_t cl = V.cls[p];
    const int npil = (F.even && cl >= 1) ? kPilots : 0;  // pilots exist inside V_out only
    if ((int)m + npil == 0 && cl != 1) return;  // untouched tile (V_out - V_in tiles get the count catch-up)
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const int ti2 = Ti * Ti, td2 = Td * Td;
    const BlendLayout L = blend_layout(Ti, Td);
    unsigned char* ws = smem + (size_t)wib * L.total;
    float4* prs = reinterpret_cast<float4*>(ws + L.prec);
    int* pk_i = reinterpret_cast<int*>(ws + L.pkey);
    int* pk_d = pk_i + kPilots;
    float4* irr_new = reinterpret_cast<float4*>(ws + L.irr_new);
    float2* dep_new = reinterpret_cast<float2*>(ws + L.dep_new);
    uint8_t* dn_new = ws + L.dn_new;
    const size_t io = (size_t)p * ti2, dof = (size_t)p * td2;
    const float4* mrec = B.main_rec + base;
    if (lane == 0) {  // L2 prefetch of the records and the old tiles, gathered below
        if (m) prefetch_l2(mrec, 16u * m);
        const uint32_t irr_b = (uint32_t)ti2 * (V.fp16 == 3 ? 4u : V.fp16 ? 8u : 16u);
        const uint32_t dep_b = (uint32_t)td2 * (V.fp16 == 3 ? 4u : V.fp16 ? 4u : 8u);
        if ((irr_b % 16u) == 0u) prefetch_l2(reinterpret_cast<const unsigned char*>(B.irr) + (size_t)p * irr_b, irr_b);
        if ((dep_b % 16u) == 0u) prefetch_l2(reinterpret_cast<const unsigned char*>(B.dep) + (size_t)p * dep_b, dep_b);
        if (V.fp16 != 3 && (td2 % 16) == 0) prefetch_l2(B.dep_n + dof, (uint32_t)td2);
    }
    // pilot samples: records and bins (pilots come first in every texel's sum)
    if (npil && lane < kPilots) {
        prs[lane] = __ldg(B.pil_rec + (size_t)p * kPilots + lane);
        const float2 e = oct_encode_x(pilot_dir(F.pilot_key, (uint32_t)p, lane));
        pk_i[lane] = texel_of(e, ni);
        pk_d[lane] = texel_of(e, nd);
    }
    const uint16_t* ord_i = B.plan.ord_i + (m ? (size_t)m * (m - 1) / 2 : 0);
    const uint16_t* ord_d = B.plan.ord_d + (m ? (size_t)m * (m - 1) / 2 : 0);
    const uint16_t* beg_i = B.plan.beg_i + (size_t)(m ? m - 1 : 0) * (ti2 + 1);
    const uint16_t* beg_d = B.plan.beg_d + (size_t)(m ? m - 1 : 0) * (td2 + 1);
    __syncwarp();
    if (V.fp16 == 3) {
        blend_packed(V, B, p, m, npil, mrec, prs, pk_i, pk_d, ord_i, ord_d, beg_i, beg_d,
                     reinterpret_cast<uint32_t*>(irr_new), reinterpret_cast<uint32_t*>(dep_new), lane);
        return;
    }
    // each lane sums whole texels: the pilots of the texel in pilot order,
    // then the texel's bucket of the plan in SF index order (the sample
    // order), and blends the texel
    const float omh = 1.0f - V.hyst;
    const float rni = 1.0f / (float)ni, rnd = 1.0f / (float)nd;
    for (int q = lane; q < ni * ni; q += 32) {
        const int r = tile_row(q, rni), t = (r + 1) * Ti + (q - r * ni) + 1;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        uint32_t k = 0;
        for (int o = 0; o < npil; ++o)
            if (pk_i[o] == t) {
                const float4 x = prs[o];
                sx += x.x;
                sy += x.y;
                sz += x.z;
                ++k;
            }
        float4 v = irr_load(V, B.irr, io + t);  // issued early: independent of the sums
        if (m) {
            const uint32_t b0 = __ldg(beg_i + t), b1 = __ldg(beg_i + t + 1);
            uint32_t u = b0;
            for (; u + 4 <= b1; u += 4) {  // four gathers in flight, added in order
                uint32_t i4[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) i4[z] = min((uint32_t)__ldg(ord_i + u + z), m - 1);
                float4 x4[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) x4[z] = __ldg(mrec + i4[z]);
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                    sx += x4[z].x;
                    sy += x4[z].y;
                    sz += x4[z].z;
                }
            }
            for (; u < b1; ++u) {
                const float4 x = __ldg(mrec + min((uint32_t)__ldg(ord_i + u), m - 1));
                sx += x.x;
                sy += x.y;
                sz += x.z;
            }
            k += b1 - b0;
        }
        if (k) v = irr_texel_blend(v, sx, sy, sz, k, omh);
        if (cl == 1) v.w = fminf(v.w, 16.0f);  // V_out - V_in: counts set down to 16 (catch-up)
        irr_new[t] = v;
    }
    for (int q = lane; q < nd * nd; q += 32) {
        const int r = tile_row(q, rnd), t = (r + 1) * Td + (q - r * nd) + 1;
        // sums of the offsets from the texel's first sample x0
        float x0 = 0.f, s1 = 0.f, s2 = 0.f;
        uint32_t k = 0;
        for (int o = 0; o < npil; ++o)
            if (pk_d[o] == t) {
                const float x = prs[o].w;
                if (k == 0) x0 = x;
                const float dx = x - x0;
                s1 += dx;
                s2 += dx * dx;
                ++k;
            }
        float2 v = dep_load(V, B.dep, dof + t);  // issued early: independent of the sums
        uint32_t c = B.dep_n[dof + t];
        if (m) {
            const uint32_t b0 = __ldg(beg_d + t), b1 = __ldg(beg_d + t + 1);
            if (k == 0 && b0 < b1) x0 = __ldg(&mrec[min((uint32_t)__ldg(ord_d + b0), m - 1)].w);
            uint32_t u = b0;
            for (; u + 2 <= b1; u += 2) {  // two gathers in flight, added in order
                const uint32_t i0 = min((uint32_t)__ldg(ord_d + u), m - 1), i1 = min((uint32_t)__ldg(ord_d + u + 1), m - 1);
                const float d0 = __ldg(&mrec[i0].w) - x0, d1 = __ldg(&mrec[i1].w) - x0;
                s1 += d0;
                s2 += d0 * d0;
                s1 += d1;
                s2 += d1 * d1;
            }
            if (u < b1) {
                const float dx = __ldg(&mrec[min((uint32_t)__ldg(ord_d + u), m - 1)].w) - x0;
                s1 += dx;
                s2 += dx * dx;
            }
            k += b1 - b0;
        }
        if (k) v = dep_texel_blend(v, c, x0, s1, s2, k, omh);
        if (cl == 1) c = min(c, 16u);
        dep_new[t] = v;
        dn_new[t] = (uint8_t)c;
    }
    __syncwarp();
    store_tiles(V, F, B.irr, B.dep, B.dep_n, B.src, p, irr_new, dep_new, dn_new, lane);
}

// ---- DDGI cosine gather (blend_mode = 1, Sec. 3.1): every ray of the probe
// feeds every texel of its hemisphere.  Texel t with centre direction n_t
// (FP32 decode of the texel centre) and ray direction w, c = n_t . w: the
// test c > 0 is exact FP32 ((x x' + y y') + z z'), the irradiance texel
// takes the c-weighted mean radiance, the visibility texel the c^50-weighted
// mean of {d, d^2} (weights taken relative to the texel's largest c); the number of rays with c > 0 is the batch count of the
// moving average.  One warp per probe; rays are staged 32 at a time in
// shared memory; each lane holds 4 texels per pass over the rays (one pass
// for the irradiance tile, two for the 14 x 14 depth interior).
constexpr int kCosPer = 4;

struct CosLayout {
    uint32_t ray_d, ray_r, irr_new, dep_new, dn_new, total;
};

__host__ __device__ inline CosLayout cos_layout(int Ti, int Td)
{
    const uint32_t ti2 = (uint32_t)(Ti * Ti), td2 = (uint32_t)(Td * Td);
    CosLayout L;
    uint32_t o = 0;
    L.ray_d = o, o += 16 * 32;  // a chunk of ray directions
    L.ray_r = o, o += 16 * 32;  // and records {r, g, b, depth}
    L.irr_new = o, o += al16(16 * ti2);
    L.dep_new = o, o += al16(8 * td2);
    L.dn_new = o, o += al16(td2);
    L.total = o;
    return L;
}

__device__ __forceinline__ float pow50(float c)
{
    const float c2 = c * c, c4 = c2 * c2, c8 = c4 * c4, c16 = c8 * c8, c32 = c16 * c16;
    return c32 * c16 * c2;
}

__global__ void __launch_bounds__(128) k_blend_cos(VolConst V, const FrameDev* __restrict__ FD, BlendBufs B)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int p = V.p_lo + blockIdx.x * (blockDim.x >> 5) + wib;
    if (p >= V.p_hi) return;  // the whole warp
    const uint32_t base = __ldg(B.off + p);
    uint32_t m = __ldg(B.off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || base > V.R_main || m > V.R_main - base) {
        if (lane == 0) atomicOr(V.err, kErrRayRange);
        m = 0;
    }
    const uint8_t cl = V.cls[p];
    const int npil = (F.even && cl >= 1) ? kPilots : 0;
    if ((int)m + npil == 0 && cl != 1) return;  // untouched tile
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const CosLayout L = cos_layout(Ti, Td);
    unsigned char* ws = smem + (size_t)wib * L.total;
    float4* rd = reinterpret_cast<float4*>(ws + L.ray_d);
    float4* rr = reinterpret_cast<float4*>(ws + L.ray_r);
    float4* irr_new = reinterpret_cast<float4*>(ws + L.irr_new);
    float2* dep_new = reinterpret_cast<float2*>(ws + L.dep_new);
    uint8_t* dn_new = ws + L.dn_new;
    const size_t io = (size_t)p * Ti * Ti, dof = (size_t)p * Td * Td;
    const float4* sfrow = B.sf + (m ? (size_t)m * (m - 1) / 2 : 0);
    const float4* mrec = B.main_rec + base;
    const int nrays = npil + (int)m;
    const float omh = 1.0f - V.hyst;
    // passes: 0 the irradiance interior, then the depth interior in groups of 32 * kCosPer texels
    const int ngi = (ni * ni + 32 * kCosPer - 1) / (32 * kCosPer), ngd = (nd * nd + 32 * kCosPer - 1) / (32 * kCosPer);
    for (int pass = 0; pass < ngi + ngd; ++pass) {
        const bool depth = pass >= ngi;
        const int n = depth ? nd : ni, g = depth ? pass - ngi : pass;
        float3 nt[kCosPer];
        float s0[kCosPer], s1[kCosPer], s2[kCosPer], sw[kCosPer], cm[kCosPer];
        uint32_t k[kCosPer];
#pragma unroll
        for (int j = 0; j < kCosPer; ++j) {
            const int q = (g * kCosPer + j) * 32 + lane;
            nt[j] = q < n * n ? texel_centre_dir(q % n, q / n, n) : make_float3(0.f, 0.f, 0.f);
            s0[j] = s1[j] = s2[j] = sw[j] = cm[j] = 0.f;
            k[j] = 0u;
        }
        for (int c0 = 0; c0 < nrays; c0 += 32) {
            const int j = c0 + lane;
            if (j < nrays) {
                float3 d;
                float4 r;
                if (j < npil) {
                    d = pilot_dir(F.pilot_key, (uint32_t)p, j);
                    r = __ldg(B.pil_rec + (size_t)p * kPilots + j);
                } else {
                    const float4 sfp = __ldg(sfrow + (j - npil));
                    const uint32_t i = min((uint32_t)__float_as_int(sfp.w), m - 1);
                    d = rotate(F.R, sfp);
                    r = __ldg(mrec + i);
                }
                rd[lane] = make_float4(d.x, d.y, d.z, 0.f);
                rr[lane] = r;
            }
            __syncwarp();
            const int cnt = min(32, nrays - c0);
            for (int u = 0; u < cnt; ++u) {
                const float4 d = rd[u], r = rr[u];
#pragma unroll
                for (int jj = 0; jj < kCosPer; ++jj) {
                    const float c = dot3x(nt[jj].x, nt[jj].y, nt[jj].z, d.x, d.y, d.z);
                    if (c > 0.0f) {
                        k[jj] += 1u;
                        if (!depth) {
                            sw[jj] += c;
                            s0[jj] = fmaf(c, r.x, s0[jj]);
                            s1[jj] = fmaf(c, r.y, s1[jj]);
                            s2[jj] = fmaf(c, r.z, s2[jj]);
                        } else {
                            // weights (c / c_max)^50 relative to the largest c so far (the
                            // mean is scale-free; c^50 itself underflows FP32 at grazing c):
                            // a new maximum rescales the weight sum and the second moment.
                            // Weighted running mean s0 and sum of squared deviations s1
                            // (West's update of Welford's method): no cancellation between
                            // the mean of d^2 and the square of the mean of d
                            if (c > cm[jj]) {
                                const float sc = cm[jj] > 0.0f ? pow50(cm[jj] / c) : 0.0f;
                                sw[jj] *= sc;
                                s1[jj] *= sc;
                                cm[jj] = c;
                            }
                            const float wgt = pow50(c / cm[jj]);
                            sw[jj] += wgt;
                            const float dx = r.w - s0[jj];
                            s0[jj] = fmaf(dx, __fdividef(wgt, sw[jj]), s0[jj]);
                            s1[jj] = fmaf(wgt * dx, r.w - s0[jj], s1[jj]);
                        }
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < kCosPer; ++j) {
            const int q = (g * kCosPer + j) * 32 + lane;
            if (q >= n * n) continue;
            const int row = q / n, t = (row + 1) * (n + 2) + (q - row * n) + 1;
            const bool ok = k[j] > 0u && sw[j] > 0.0f;
            const float kf = (float)k[j], inv = ok ? kf / sw[j] : 0.0f;  // sums of the k-sample batch: mean * k
            if (!depth) {
                float4 v = irr_load(V, B.irr, io + t);
                if (ok) v = irr_texel_blend(v, s0[j] * inv, s1[j] * inv, s2[j] * inv, k[j], omh);
                if (cl == 1) v.w = fminf(v.w, 16.0f);
                irr_new[t] = v;
            } else {
                float2 v = dep_load(V, B.dep, dof + t);
                uint32_t c = B.dep_n[dof + t];
                // the batch as mean s0 with zero offset sum and k x its variance s1 / sw
                if (ok) v = dep_texel_blend(v, c, s0[j], 0.0f, s1[j] * inv, k[j], omh);
                if (cl == 1) c = min(c, 16u);
                dep_new[t] = v;
                dn_new[t] = (uint8_t)c;
            }
        }
    }
    __syncwarp();
    store_tiles(V, F, B.irr, B.dep, B.dep_n, B.src, p, irr_new, dep_new, dn_new, lane);
}

// ---- Metropolis samples (sampler.cu): one warp per probe tile.  The
// samples of probe p are contiguous in grouped order (sample order inside the
// probe).  Sample s adds its +w radiance to the irradiance texel of w and the
// distance along -w to the visibility texel of -w (the extra ray of the
// static adaptive sampling); the pilots come first on the first frame of a
// pair.  Per texel the sums run in that order (a chunk's samples of one
// texel summed first, in order); then the batched moving average and the
// stores of k_blend.
struct MhLayout {
    uint32_t acc_i, acc_d, cnt_d, sh_d, dn, e_rec, dacc_i, dacc_d, dcnt_d, dsh_d, total;
};

__host__ __device__ inline MhLayout mh_layout(int Ti, int Td, bool dyn)
{
    const uint32_t ti2 = (uint32_t)(Ti * Ti), td2 = (uint32_t)(Td * Td);
    MhLayout L;
    uint32_t o = 0;
    L.acc_i = o, o += al16(16 * ti2);  // {sum r, g, b, count}, then the updated texel
    L.acc_d = o, o += al16(8 * td2);   // {sum d - x0, sum (d - x0)^2}, then the updated texel
    L.cnt_d = o, o += al16(4 * td2);
    L.sh_d = o, o += al16(4 * td2);    // x0: the texel's first sample (the shift of the sums)
    L.dn = o, o += al16(td2);
    L.e_rec = o, o += 16 * 32;  // one chunk of samples: {r, g, b, depth}
    L.dacc_i = L.dacc_d = L.dcnt_d = L.dsh_d = o;
    if (dyn) {  // the dynamic rays' sums: a second batch step
        L.dacc_i = o, o += al16(16 * ti2);
        L.dacc_d = o, o += al16(8 * td2);
        L.dcnt_d = o, o += al16(4 * td2);
        L.dsh_d = o, o += al16(4 * td2);
    }
    L.total = o;
    return L;
}

// Add a chunk of samples, one per lane (lane j holds sample j of the chunk
// with its texels ki, kd; -1 for none): the lanes of one texel form a group
// (match_any) whose lowest lane sums the group's records in lane order and
// adds the sum to the texel.  Texels are distinct across groups, so the
// adds do not race; per texel the chunks are added in order.
__device__ __forceinline__ void mh_accumulate(const float4* e_rec, int ki, int kd, float4* acc_i, float2* acc_d,
                                              uint32_t* cnt_d, float* sh_d, int lane)
{
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t gi = __match_any_sync(0xFFFFFFFFu, ki), gd = __match_any_sync(0xFFFFFFFFu, kd);
    if (ki >= 0 && (gi & below) == 0u) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (uint32_t m = gi; m; m &= m - 1u) {
            const float4 r = e_rec[__ffs(m) - 1];
            sx += r.x;
            sy += r.y;
            sz += r.z;
        }
        float4 t = acc_i[ki];
        t.x += sx;
        t.y += sy;
        t.z += sz;
        t.w += (float)__popc(gi);
        acc_i[ki] = t;
    }
    if (kd >= 0 && (gd & below) == 0u) {
        // offsets from the texel's first sample (this group's first when the
        // texel has none yet)
        if (cnt_d[kd] == 0u) sh_d[kd] = e_rec[__ffs(gd) - 1].w;
        const float x0 = sh_d[kd];
        float s1 = 0.f, s2 = 0.f;
        for (uint32_t m = gd; m; m &= m - 1u) {
            const float dx = e_rec[__ffs(m) - 1].w - x0;
            s1 += dx;
            s2 += dx * dx;
        }
        float2 t = acc_d[kd];
        t.x += s1;
        t.y += s2;
        acc_d[kd] = t;
        cnt_d[kd] += (uint32_t)__popc(gd);
    }
}

__global__ void __launch_bounds__(128) k_mh_blend(VolConst V, const FrameDev* __restrict__ FD, MhBlendBufs B)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int p = blockIdx.x * (blockDim.x >> 5) + wib;
    if (p >= V.P) return;  // the whole warp
    const uint32_t b0 = __ldg(B.off + p);
    uint32_t b1 = __ldg(B.off + p + 1);
    if (b1 < b0 || b1 > B.n) {
        if (lane == 0) atomicOr(V.err, kErrRayRange);
        b1 = b0;
    }
    const uint8_t cl = V.cls[p];
    if (cl != 2) b1 = b0;  // samples outside V_in are dropped
    const int npil = (F.even && cl >= 1) ? kPilots : 0;
    const uint32_t r0 = V.dyn ? __ldg(B.dyn.off + p) : 0u, r1 = V.dyn ? __ldg(B.dyn.off + p + 1) : 0u;
    if (b1 == b0 && npil == 0 && r1 <= r0 && cl != 1) return;  // untouched tile
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const int ti2 = Ti * Ti, td2 = Td * Td;
    const MhLayout L = mh_layout(Ti, Td, V.dyn != 0);
    unsigned char* ws = smem + (size_t)wib * L.total;
    float4* acc_i = reinterpret_cast<float4*>(ws + L.acc_i);
    float2* acc_d = reinterpret_cast<float2*>(ws + L.acc_d);
    uint32_t* cnt_d = reinterpret_cast<uint32_t*>(ws + L.cnt_d);
    float* sh_d = reinterpret_cast<float*>(ws + L.sh_d);
    uint8_t* dn = ws + L.dn;
    float4* e_rec = reinterpret_cast<float4*>(ws + L.e_rec);
    for (int t = lane; t < ti2; t += 32) acc_i[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = lane; t < td2; t += 32) {
        acc_d[t] = make_float2(0.f, 0.f);
        cnt_d[t] = 0u;
    }
    float4* dacc_i = reinterpret_cast<float4*>(ws + L.dacc_i);
    float2* dacc_d = reinterpret_cast<float2*>(ws + L.dacc_d);
    uint32_t* dcnt_d = reinterpret_cast<uint32_t*>(ws + L.dcnt_d);
    float* dsh_d = reinterpret_cast<float*>(ws + L.dsh_d);
    if (V.dyn) {
        for (int t = lane; t < ti2; t += 32) dacc_i[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t = lane; t < td2; t += 32) {
            dacc_d[t] = make_float2(0.f, 0.f);
            dcnt_d[t] = 0u;
        }
    }
    __syncwarp();
    if (npil) {
        int ki = -1, kd = -1;
        if (lane < kPilots) {
            e_rec[lane] = __ldg(B.pil_rec + (size_t)p * kPilots + lane);
            const float2 e = oct_encode_x(pilot_dir(F.pilot_key, (uint32_t)p, lane));
            ki = texel_of(e, ni);
            kd = texel_of(e, nd);
        }
        __syncwarp();
        mh_accumulate(e_rec, ki, kd, acc_i, acc_d, cnt_d, sh_d, lane);
        __syncwarp();
    }
    // chunks of 32 samples, one per lane; the next chunk's loads are issued
    // before the current chunk is added (two chunks in flight per warp)
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), x = a;
    int2 hn = make_int2((int)kMiss, 0);
    if (b0 + lane < b1) {
        a = __ldg(B.smp_g + b0 + lane);
        x = __ldg(B.rec + b0 + lane);
        hn = __ldg(B.hit_neg + b0 + lane);
    }
    for (uint32_t c0 = b0; c0 < b1; c0 += 32) {
        int ki = -1, kd = -1;
        if (c0 + lane < b1) {
            const float dep = (uint32_t)hn.x == kMiss ? V.depth_max : fminf(__int_as_float(hn.y), V.depth_max);
            e_rec[lane] = make_float4(x.x, x.y, x.z, dep);
            ki = texel_of(oct_encode_x(make_float3(a.x, a.y, a.z)), ni);
            const float4 an = B.smp_gn ? __ldg(B.smp_gn + c0 + lane) : make_float4(-a.x, -a.y, -a.z, 0.f);
            kd = texel_of(oct_encode_x(make_float3(an.x, an.y, an.z)), nd);
        }
        __syncwarp();
        const uint32_t qn = c0 + 32 + lane;
        if (qn < b1) {
            a = __ldg(B.smp_g + qn);
            x = __ldg(B.rec + qn);
            hn = __ldg(B.hit_neg + qn);
        }
        mh_accumulate(e_rec, ki, kd, acc_i, acc_d, cnt_d, sh_d, lane);
        __syncwarp();
    }
    // the dynamic rays of the probe (each at its own texel centre): sums of
    // the second batch step
    for (uint32_t c0 = r0; c0 < r1; c0 += 32) {
        int ki = -1, kd = -1;
        if (c0 + lane < r1) {
            int pp, t;
            float3 d;
            if (dyn_ray_of(V, B.dyn, c0 + lane, pp, t, d) && pp == p) {
                e_rec[lane] = __ldg(B.drec + c0 + lane);
                ki = t;
                kd = texel_of(oct_encode_x(d), nd);
            } else {
                atomicOr(V.err, kErrRayRange);
            }
        }
        __syncwarp();
        mh_accumulate(e_rec, ki, kd, dacc_i, dacc_d, dcnt_d, dsh_d, lane);
        __syncwarp();
    }
    const float omh = 1.0f - V.hyst;
    const float rni = 1.0f / (float)ni, rnd = 1.0f / (float)nd;
    const size_t io = (size_t)p * ti2, dof = (size_t)p * td2;
    for (int q = lane; q < ni * ni; q += 32) {
        const int r = tile_row(q, rni), t = (r + 1) * Ti + (q - r * ni) + 1;
        const float4 sum = acc_i[t];
        float4 v = irr_load(V, B.irr, io + t);
        if (sum.w > 0.0f) v = irr_texel_blend(v, sum.x, sum.y, sum.z, (uint32_t)sum.w, omh);
        if (V.dyn) {
            const float4 ds = dacc_i[t];
            if (ds.w > 0.0f) v = irr_texel_blend(v, ds.x, ds.y, ds.z, (uint32_t)ds.w, 1.0f - V.hyst_dyn);
        }
        if (cl == 1) v.w = fminf(v.w, 16.0f);
        acc_i[t] = v;
    }
    for (int q = lane; q < nd * nd; q += 32) {
        const int r = tile_row(q, rnd), t = (r + 1) * Td + (q - r * nd) + 1;
        const float2 sum = acc_d[t];
        const uint32_t k = cnt_d[t];
        float2 v = dep_load(V, B.dep, dof + t);
        uint32_t c = B.dep_n[dof + t];
        if (k) v = dep_texel_blend(v, c, sh_d[t], sum.x, sum.y, k, omh);
        if (V.dyn) {
            const uint32_t kd2 = dcnt_d[t];
            const float2 ds = dacc_d[t];
            if (kd2) v = dep_texel_blend(v, c, dsh_d[t], ds.x, ds.y, kd2, 1.0f - V.hyst_dyn);
        }
        if (cl == 1) c = min(c, 16u);
        acc_d[t] = v;
        dn[t] = (uint8_t)c;
    }
    __syncwarp();
    store_tiles(V, F, B.irr, B.dep, B.dep_n, B.src, p, acc_i, acc_d, dn, lane);
}

// ============================================================== query
__global__ void __launch_bounds__(128) k_query(VolConst V, const void* __restrict__ irr, const void* __restrict__ dep,
                                               const float* __restrict__ pos, const float* __restrict__ nrm, int n,
                                               float* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 x = make_float3(pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]);
    float3 nn = make_float3(nrm[3 * (size_t)i], nrm[3 * (size_t)i + 1], nrm[3 * (size_t)i + 2]);
    float3 e = query_irr(V, irr, dep, x, nn);
    out[3 * (size_t)i] = e.x;
    out[3 * (size_t)i + 1] = e.y;
    out[3 * (size_t)i + 2] = e.z;
}

}  // namespace

size_t blend_plan_bytes(int M, int Ti, int Td)
{
    const size_t m = (size_t)(M > 0 ? M : 0), tri = m * (m + 1) / 2;
    return sizeof(uint16_t) * (2 * tri + m * ((size_t)Ti * Ti + 1) + m * ((size_t)Td * Td + 1) + 8);
}

BlendPlan carve_blend_plan(void* base, int M, int Ti, int Td)
{
    const size_t m = (size_t)(M > 0 ? M : 0), tri = m * (m + 1) / 2;
    uint16_t* b = reinterpret_cast<uint16_t*>(base);
    BlendPlan P;
    P.ord_i = b;
    P.ord_d = b + tri;
    P.beg_i = b + 2 * tri;
    P.beg_d = P.beg_i + m * ((size_t)Ti * Ti + 1);
    return P;
}

// shared memory of one probe (one warp) of k_blend
size_t blend_smem_bytes(const VolConst& V) { return blend_layout(V.Ti, V.Td).total; }

cudaError_t launch_change(const VolConst& V, const FrameDev* FD, const ChangeBufs& B, cudaStream_t s, int parts)
{
    const int n = V.p_hi - V.p_lo;
    if (n <= 0) return cudaSuccess;
    if (parts & 1) {
        k_change_state<<<(n + 127) / 128, 128, 0, s>>>(V, FD, B);
        count_launches(1);
    }
    if (parts & 2) {
        k_change_weight<<<(n + 127) / 128, 128, 0, s>>>(V, FD, B);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_classify(const VolConst& V, const FrameDev* FD, const uint16_t* lut_c, uint8_t* cls,
                            cudaStream_t s)
{
    k_classify<<<(V.P + 255) / 256, 256, 0, s>>>(V, FD, lut_c, cls);
    count_launches(1);
    return cudaGetLastError();
}

// The dynamic shared-memory limit of a kernel is one attribute per device,
// shared by every launch in the process, graphs captured earlier included.
// It is only ever raised: lowering it for a small volume could invalidate a
// launch or a graph made for a larger one.
static cudaError_t raise_smem_limit(const void* func, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

cudaError_t launch_allocate(const uint32_t* W, int P, int avg, int m0, int rmax, uint32_t* n_out, uint32_t* off_out,
                            cudaStream_t s, const uint8_t* cls)
{
    if (P <= kAllocClusterMaxP) {
        const int sm = 8 * ((P + kAllocCluster - 1) / kAllocCluster);
        // the limit for the largest grid the cluster kernel takes, set once
        cudaError_t e = raise_smem_limit((const void*)k_allocate_cluster, 8 * (kAllocClusterMaxP / kAllocCluster));
        if (e != cudaSuccess) return e;
        k_allocate_cluster<<<kAllocCluster, kAllocThreads, sm, s>>>(W, P, avg, m0, rmax, n_out, off_out, cls);
    } else {
        k_allocate<<<1, kAllocThreads, 0, s>>>(W, P, avg, m0, rmax, n_out, off_out, cls);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend_plan(const VolConst& V, const FrameDev* FD, const float4* sf, const BlendPlan& plan,
                              cudaStream_t s)
{
    const int M = V.rays_max - kPilots;
    if (M <= 0) return cudaSuccess;
    const size_t ps = blend_plan_smem(V);
    {
        cudaError_t e = raise_smem_limit((const void*)k_blend_plan, ps);
        if (e != cudaSuccess) return e;
    }
    k_blend_plan<<<M, 256, ps, s>>>(V, FD, sf, plan);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s)
{
    // probes per CTA (one warp each), as many as the tuning asks and 227 KB allow
    const size_t per = blend_smem_bytes(V);
    const int wpb = std::max(1, std::min(T.blend_block / 32, (int)((227u * 1024u) / per)));
    const size_t sm = per * (size_t)wpb;
    {
        cudaError_t e = raise_smem_limit((const void*)k_blend, sm);
        if (e != cudaSuccess) return e;
    }
    const int np = V.p_hi - V.p_lo;
    if (np <= 0) return cudaSuccess;
    k_blend<<<(np + wpb - 1) / wpb, 32 * wpb, sm, s>>>(V, FD, B);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend_cos(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s)
{
    (void)T;
    const size_t per = cos_layout(V.Ti, V.Td).total;
    const int wpb = std::max(1, std::min(4, (int)((227u * 1024u) / per)));
    const size_t sm = per * (size_t)wpb;
    {
        cudaError_t e = raise_smem_limit((const void*)k_blend_cos, sm);
        if (e != cudaSuccess) return e;
    }
    const int np = V.p_hi - V.p_lo;
    if (np <= 0) return cudaSuccess;
    k_blend_cos<<<(np + wpb - 1) / wpb, 32 * wpb, sm, s>>>(V, FD, B);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mh_blend(const VolConst& V, const FrameDev* FD, const MhBlendBufs& B, cudaStream_t s)
{
    const size_t per = mh_layout(V.Ti, V.Td, V.dyn != 0).total;
    const int wpb = std::max(1, std::min(4, (int)((227u * 1024u) / per)));
    const size_t sm = per * (size_t)wpb;
    {
        cudaError_t e = raise_smem_limit((const void*)k_mh_blend, sm);
        if (e != cudaSuccess) return e;
    }
    k_mh_blend<<<(V.P + wpb - 1) / wpb, 32 * wpb, sm, s>>>(V, FD, B);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_query(const VolConst& V, const void* irr, const void* dep, const float* pos, const float* nrm, int n,
                         float* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_query<<<(n + 127) / 128, 128, 0, s>>>(V, irr, dep, pos, nrm, n, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adgi
