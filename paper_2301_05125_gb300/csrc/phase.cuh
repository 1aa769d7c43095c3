// phase.cuh -- device bodies of the update's per-probe phases (sm_103a):
// clip classes, change measure, blend plan and blend, plus the block-wide
// sums of the allocation.  The ordinary kernels (update.cu) and the
// persistent batched tick (tick.cu) run the same bodies.
#pragma once
#include <cuda_fp16.h>

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

__device__ __forceinline__ void classify_body(const VolConst& V, const FrameDev* FD, const uint16_t* __restrict__ lut_c,
                                              uint8_t* cls, unsigned bx)
{
    const FrameConst& F = FD->F;
    const int p = bx * blockDim.x + threadIdx.x;
    if (p >= V.P) return;
    uint8_t c = 2;
    if (F.has_clip && F.has_camera) {
        const float3 x = probe_pos(V, p);
        const uint32_t qc = qc_of_probe(V, F, lut_c, p);
        c = (qc >= 768u && in_frustum(F.clip, x, 1.2f)) ? 2 : ((qc >= 512u && in_frustum(F.clip, x, 1.4f)) ? 1 : 0);
    }
    cls[p] = c;
}

__device__ __forceinline__ void change_state_body(const VolConst& V, const FrameDev* FD, const ChangeBufs& B, unsigned bx)
{
    const FrameConst& F = FD->F;
    int p = V.p_lo + bx * blockDim.x + threadIdx.x;
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
template <bool kLive>
__device__ __forceinline__ void change_weight_body(const VolConst& V, const FrameDev* FD, const ChangeBufs& B,
                                                   unsigned bx)
{
    const FrameConst& F = FD->F;
    int p = V.p_lo + bx * blockDim.x + threadIdx.x;
    if (p >= V.p_hi) return;
    const int X = V.dims[0], Y = V.dims[1], Z = V.dims[2];
    int ix = p % X, iy = (p / X) % Y, iz = p / (X * Y);
    uint32_t f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int jz = max(iz - 2, 0); jz <= min(iz + 2, Z - 1); ++jz)
        for (int jy = max(iy - 2, 0); jy <= min(iy + 2, Y - 1); ++jy)
            for (int jx = max(ix - 2, 0); jx <= min(ix + 2, X - 1); ++jx) {
                const uint4* G4 = reinterpret_cast<const uint4*>(B.G + ((size_t)jx + (size_t)X * (jy + (size_t)Y * jz)) * 8);
                uint4 a = ldl<kLive>(G4), b = ldl<kLive>(G4 + 1);
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

// Plan of SF row m = bx + 1 for this frame's rotation.
__device__ __forceinline__ void blend_plan_body(const VolConst& V, const FrameDev* FD, const float4* __restrict__ sf,
                                                const BlendPlan& Pl, unsigned bx)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int m = (int)bx + 1;
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
template <bool kLive>
__device__ __forceinline__ void blend_packed(const VolConst& V, const BlendBufs& B, int p, uint32_t m, int npil,
                                             const float4* mrec, const float4* prs, const int* pk_i, const int* pk_d,
                                             const uint16_t* ord_i, const uint16_t* ord_d, const uint16_t* beg_i,
                                             const uint16_t* beg_d, uint32_t* irr_new, uint32_t* dep_new, int lane)
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
            const uint32_t b1 = ldl<kLive>(beg_i + t + 1);
            for (uint32_t u = ldl<kLive>(beg_i + t); u < b1; ++u) {
                const float4 rc = ldl<kLive>(mrec + min((uint32_t)ldl<kLive>(ord_i + u), m - 1));
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
            const uint32_t b1 = ldl<kLive>(beg_d + t + 1);
            for (uint32_t u = ldl<kLive>(beg_d + t); u < b1; ++u)
                x.add(ct, fd(ldl<kLive>(&mrec[min((uint32_t)ldl<kLive>(ord_d + u), m - 1)].w), V.s_f));
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

template <bool kLive>
// bx: the item of wpb probe tiles (one warp each) that this block works on
__device__ __forceinline__ void blend_body(const VolConst& V, const FrameDev* FD, const BlendBufs& B, unsigned bx,
                                           int wpb)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int p = V.p_lo + bx * wpb + wib;
    if (wib >= wpb || p >= V.p_hi) return;  // the whole warp
    const uint32_t base = ldl<kLive>(B.off + p);
    uint32_t m = ldl<kLive>(B.off + p + 1) - base;
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
        prs[lane] = ldl<kLive>(B.pil_rec + (size_t)p * kPilots + lane);
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
        blend_packed<kLive>(V, B, p, m, npil, mrec, prs, pk_i, pk_d, ord_i, ord_d, beg_i, beg_d,
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
            const uint32_t b0 = ldl<kLive>(beg_i + t), b1 = ldl<kLive>(beg_i + t + 1);
            uint32_t u = b0;
            for (; u + 4 <= b1; u += 4) {  // four gathers in flight, added in order
                uint32_t i4[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) i4[z] = min((uint32_t)ldl<kLive>(ord_i + u + z), m - 1);
                float4 x4[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) x4[z] = ldl<kLive>(mrec + i4[z]);
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                    sx += x4[z].x;
                    sy += x4[z].y;
                    sz += x4[z].z;
                }
            }
            for (; u < b1; ++u) {
                const float4 x = ldl<kLive>(mrec + min((uint32_t)ldl<kLive>(ord_i + u), m - 1));
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
            const uint32_t b0 = ldl<kLive>(beg_d + t), b1 = ldl<kLive>(beg_d + t + 1);
            if (k == 0 && b0 < b1) x0 = ldl<kLive>(&mrec[min((uint32_t)ldl<kLive>(ord_d + b0), m - 1)].w);
            uint32_t u = b0;
            for (; u + 2 <= b1; u += 2) {  // two gathers in flight, added in order
                const uint32_t i0 = min((uint32_t)ldl<kLive>(ord_d + u), m - 1), i1 = min((uint32_t)ldl<kLive>(ord_d + u + 1), m - 1);
                const float d0 = ldl<kLive>(&mrec[i0].w) - x0, d1 = ldl<kLive>(&mrec[i1].w) - x0;
                s1 += d0;
                s2 += d0 * d0;
                s1 += d1;
                s2 += d1 * d1;
            }
            if (u < b1) {
                const float dx = ldl<kLive>(&mrec[min((uint32_t)ldl<kLive>(ord_d + u), m - 1)].w) - x0;
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

}  // namespace

}  // namespace adgi
