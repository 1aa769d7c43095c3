// update.cu -- heuristics, ray allocation, blend and query kernels (sm_103a).
#include <algorithm>

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

__global__ void __launch_bounds__(128) k_change_state(VolConst V, const FrameDev* __restrict__ FD, ChangeBufs B)
{
    const FrameConst& F = FD->F;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.P) return;
    uint32_t yv[8], yr[8];
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
        if (!F.even && F.pair_valid) {
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
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.P) return;
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
    uint32_t qc = 1023u;
    if (F.has_camera) {
        float3 pp = probe_pos(V, p);
        float dx = fs(pp.x, F.cam[0]), dy = fs(pp.y, F.cam[1]), dz = fs(pp.z, F.cam[2]);
        float dist = fsq(dot3x(dx, dy, dz, dx, dy, dz));
        if (!(dist < F.cam_k)) {
            float q = fm(fs(dist, F.cam_k), V.qc_scale);
            uint32_t i = q < 4095.0f ? (uint32_t)floorf(q) : 4095u;
            qc = __ldg(B.lut_c + i);
        }
    }
    uint64_t Wp = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o) Wp += ((uint64_t)qc * (uint64_t)B.qv[(size_t)p * 8 + o] * (uint64_t)f[o]) >> 20;
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

__global__ void __launch_bounds__(kAllocThreads) k_allocate(const uint32_t* __restrict__ W, int P, int avg, int m0,
                                                            int rmax, uint32_t* __restrict__ n, uint32_t* __restrict__ off)
{
    __shared__ uint64_t red[33];
    const int chunk = (P + kAllocThreads - 1) / kAllocThreads;
    const int c0 = min(P, (int)threadIdx.x * chunk), c1 = min(P, c0 + chunk);
    const uint64_t E = (uint64_t)(avg - m0) * (uint64_t)P;
    const uint32_t cap = (uint32_t)(rmax - m0);
    uint64_t s = 0;
    for (int p = c0; p < c1; ++p) s += W[p];
    const uint64_t S = block_sum(s, red);
    if (S == 0) {
        const uint64_t q = E / (uint64_t)P, r = E % (uint64_t)P;
        for (int p = c0; p < c1; ++p) n[p] = (uint32_t)(q + ((uint64_t)p < r ? 1u : 0u));
    } else {
        for (int p = c0; p < c1; ++p) n[p] = 0u;
        uint64_t Erem = E;
        for (int it = 0; it < kAllocIters; ++it) {
            uint64_t su = 0;
            for (int p = c0; p < c1; ++p) {
                uint32_t w = W[p];
                if (w > 0u && n[p] < cap) su += w;
            }
            const uint64_t SU = block_sum(su, red);
            if (SU == 0 || Erem == 0) break;
            uint64_t given = 0;
            for (int p = c0; p < c1; ++p) {
                uint32_t w = W[p], e = n[p];
                if (w == 0u || e >= cap) continue;
                uint64_t share = Erem * (uint64_t)w / SU;
                uint64_t room = cap - e;
                uint64_t a = share < room ? share : room;
                n[p] = e + (uint32_t)a;
                given += a;
            }
            const uint64_t G = block_sum(given, red);
            if (G == 0) break;
            Erem -= G;
        }
        // remainder: one each, probe-index order, probes with W > 0 first
        for (int guard = 0; Erem > 0 && guard < (1 << 20); ++guard) {
            uint64_t ca = 0;
            for (int p = c0; p < c1; ++p)
                if (W[p] > 0u && n[p] < cap) ++ca;
            const bool modeA = block_sum(ca, red) > 0;
            uint64_t ce = 0;
            for (int p = c0; p < c1; ++p)
                if (n[p] < cap && (!modeA || W[p] > 0u)) ++ce;
            uint64_t tot;
            uint64_t pre = block_exscan(ce, red, &tot);
            if (tot == 0) break;
            for (int p = c0; p < c1; ++p) {
                if (n[p] < cap && (!modeA || W[p] > 0u)) {
                    if (pre < Erem) n[p] += 1u;
                    ++pre;
                }
            }
            Erem -= tot < Erem ? tot : Erem;
        }
    }
    uint64_t loc = 0;
    for (int p = c0; p < c1; ++p) loc += (uint64_t)(m0 - 8) + n[p];
    uint64_t tot;
    uint64_t pre = block_exscan(loc, red, &tot);
    for (int p = c0; p < c1; ++p) {
        off[p] = (uint32_t)pre;
        uint32_t np = (uint32_t)m0 + n[p];
        pre += np - 8u;
        n[p] = np;
    }
    if (threadIdx.x == 0) off[P] = (uint32_t)tot;
}

// ============================================================== blend
// Alg. ApproxAlgo + Alg. MovingAvgUpdate, batched per texel, in two kernels.
//  plan  (once per frame): the irradiance and depth texel of every point of
//        every row of the SF table under this frame's rotation -- every probe
//        with m adaptive rays shares row m, so binning is done once per
//        direction, not once per ray;
//  blend (one warp per probe tile): the probe's ray records stream through
//        shared memory 32 at a time (cp.async, double buffered) and the old
//        tiles are staged beside them; within each group of 32 samples, the
//        lanes that fall in the same texel are found with match_any and the
//        group's lowest lane adds them in lane order, so every texel sums its
//        samples in sample order (pilots, then SF index order): the result is
//        deterministic, with no floating-point atomics.  Touched texels are
//        blended with w = max(1 - h, k/(n+k)), and every texel -- border
//        texels from their octahedral fold partner -- is written back with
//        coalesced stores in texel order.

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




// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Plan of this frame: thread e handles entry e of the flat table (row m,
// SF index i).
__global__ void __launch_bounds__(256) k_blend_plan(VolConst V, const FrameDev* __restrict__ FD,
                                                    const float4* __restrict__ sf, BlendPlan Pl, uint32_t n_entries)
{
    const FrameConst& F = FD->F;
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_entries) return;
    // row m holds SF indices in a spatial order; position e - row start is
    // SF index .w of that point
    const uint32_t m = (uint32_t)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);  // first guess of the row
    uint32_t mm = m;
    while (mm > 1 && (size_t)mm * (mm - 1) / 2 > e) --mm;  // m(m-1)/2 <= e < m(m+1)/2
    while ((size_t)(mm + 1) * mm / 2 <= e) ++mm;
    const size_t row = (size_t)mm * (mm - 1) / 2;
    const float4 s4 = __ldg(sf + e);
    const uint32_t i = (uint32_t)__float_as_int(s4.w);
    if (i >= mm) {
        atomicOr(V.err, kErrIndex);
        return;
    }
    const float2 oe = oct_encode_x(rotate(F.R, s4));
    Pl.key_i[row + i] = (uint16_t)texel_of(oe, V.n_irr);
    Pl.key_d[row + i] = (uint16_t)texel_of(oe, V.n_dep);
}

// shared memory of one probe (one warp) of k_blend: two 32-record buffers,
// the pilot records and bins, the old tiles as stored, per-texel running
// sums and counts, and the updated depth counts
struct BlendLayout {
    uint32_t rb, prec, pkey, irr_raw, dep_raw, dn_raw, acc_i, acc_d, cnt_d, dn_new, total;
};

__host__ __device__ inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline BlendLayout blend_layout(int Ti, int Td)
{
    const uint32_t ti2 = (uint32_t)(Ti * Ti), td2 = (uint32_t)(Td * Td);
    BlendLayout L;
    uint32_t o = 0;
    L.rb = o, o += 2 * 32 * 16;
    L.prec = o, o += 16 * kPilots;
    L.pkey = o, o += 4 * 2 * kPilots;
    L.irr_raw = o, o += al16(16 * ti2);
    L.dep_raw = o, o += al16(8 * td2);
    L.dn_raw = o, o += al16(td2);
    L.acc_i = o, o += al16(16 * ti2);
    L.acc_d = o, o += al16(8 * td2);
    L.cnt_d = o, o += al16(2 * td2);
    L.dn_new = o, o += al16(td2);
    L.total = o;
    return L;
}

// row of texel t in a tile of width T (t < 1024, T <= 32: the product is
// never within 2^-7 of an integer, so single-precision rounding is harmless)
__device__ __forceinline__ int tile_row(int t, float rT) { return (int)(((float)t + 0.5f) * rT); }

__global__ void __launch_bounds__(256) k_blend(VolConst V, const FrameDev* __restrict__ FD, BlendBufs B)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int p = blockIdx.x * (blockDim.x >> 5) + wib;
    if (p >= V.P) return;  // the whole warp
    const uint32_t base = __ldg(B.off + p);
    uint32_t m = __ldg(B.off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || base > V.R_main || m > V.R_main - base) {
        if (lane == 0) atomicOr(V.err, kErrRayRange);
        m = 0;
    }
    const int npil = F.even ? kPilots : 0;
    if ((int)m + npil == 0) return;  // untouched tile: nothing to read or write
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const int ti2 = Ti * Ti, td2 = Td * Td;
    const BlendLayout L = blend_layout(Ti, Td);
    unsigned char* ws = smem + (size_t)wib * L.total;
    float4* rb = reinterpret_cast<float4*>(ws + L.rb);  // [2][32]
    float4* prs = reinterpret_cast<float4*>(ws + L.prec);
    int* pk_i = reinterpret_cast<int*>(ws + L.pkey);
    int* pk_d = pk_i + kPilots;
    unsigned char* irr_raw = ws + L.irr_raw;
    unsigned char* dep_raw = ws + L.dep_raw;
    uint8_t* dn_raw = ws + L.dn_raw;
    float4* acc_i = reinterpret_cast<float4*>(ws + L.acc_i);
    float2* acc_d = reinterpret_cast<float2*>(ws + L.acc_d);
    uint16_t* cnt_d = reinterpret_cast<uint16_t*>(ws + L.cnt_d);
    uint8_t* dn_new = ws + L.dn_new;
    const size_t io = (size_t)p * ti2, dof = (size_t)p * td2;
    const float4* mrec = B.main_rec + base;
    // old tiles: asynchronous copies when the tile sizes are 16-byte multiples
    const uint32_t irr_b = (uint32_t)ti2 * (V.fp16 ? 8u : 16u), dep_b = (uint32_t)td2 * (V.fp16 ? 4u : 8u);
    const uint32_t dn_b = (uint32_t)td2;
    const bool tiles_async = (irr_b % 16u) == 0u && (dep_b % 16u) == 0u && (dn_b % 16u) == 0u;
    const unsigned char* g_irr = reinterpret_cast<const unsigned char*>(B.irr) + (size_t)p * irr_b;
    const unsigned char* g_dep = reinterpret_cast<const unsigned char*>(B.dep) + (size_t)p * dep_b;
    const uint8_t* g_dn = B.dep_n + dof;
    if (tiles_async) {
        for (uint32_t c = lane; c < irr_b / 16u; c += 32) cp_async16(irr_raw + 16 * c, g_irr + 16 * c);
        for (uint32_t c = lane; c < dep_b / 16u; c += 32) cp_async16(dep_raw + 16 * c, g_dep + 16 * c);
        for (uint32_t c = lane; c < dn_b / 16u; c += 32) cp_async16(dn_raw + 16 * c, g_dn + 16 * c);
    } else {
        for (uint32_t c = lane; c < irr_b / 4u; c += 32)
            reinterpret_cast<uint32_t*>(irr_raw)[c] = reinterpret_cast<const uint32_t*>(g_irr)[c];
        for (uint32_t c = lane; c < dep_b / 4u; c += 32)
            reinterpret_cast<uint32_t*>(dep_raw)[c] = reinterpret_cast<const uint32_t*>(g_dep)[c];
        for (uint32_t c = lane; c < dn_b; c += 32) dn_raw[c] = g_dn[c];
    }
    cp_async_commit();  // group: tiles
    // records of rounds 0 and 1 (32 samples each)
    const uint32_t rounds = (m + 31u) / 32u;
    if (lane < m) cp_async16(rb + lane, mrec + lane);
    cp_async_commit();  // group: round 0
    if (32u + lane < m) cp_async16(rb + 32 + lane, mrec + 32 + lane);
    cp_async_commit();  // group: round 1
    // pilot samples (first in every texel's sum, in pilot order): records and
    // bins, added by one lane
    if (npil && lane < kPilots) {
        prs[lane] = __ldg(B.pil_rec + (size_t)p * kPilots + lane);
        const float2 e = oct_encode_x(pilot_dir(F.pilot_key, (uint32_t)p, lane));
        pk_i[lane] = texel_of(e, ni);
        pk_d[lane] = texel_of(e, nd);
    }
    for (int t = lane; t < ti2; t += 32) acc_i[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = lane; t < td2; t += 32) {
        acc_d[t] = make_float2(0.f, 0.f);
        cnt_d[t] = 0;
    }
    __syncwarp();
    if (lane == 0)
        for (int o = 0; o < npil; ++o) {
            const float4 r = prs[o];
            float4& ai = acc_i[pk_i[o]];
            ai.x += r.x;
            ai.y += r.y;
            ai.z += r.z;
            ai.w += 1.0f;
            float2& ad = acc_d[pk_d[o]];
            ad.x += r.w;
            ad.y += r.w * r.w;
            cnt_d[pk_d[o]] += 1;
        }
    // adaptive samples, 32 per round in SF index order
    const size_t row = m ? (size_t)m * (m - 1) / 2 : 0;
    uint32_t ki = 0, kd = 0;
    if (lane < m) {
        ki = __ldg(B.plan.key_i + row + lane);
        kd = __ldg(B.plan.key_d + row + lane);
    }
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t j = 32u * r + lane;
        const bool valid = j < m;
        uint32_t ki_n = 0, kd_n = 0;  // next round's bins, loaded early
        if (j + 32u < m) {
            ki_n = __ldg(B.plan.key_i + row + j + 32u);
            kd_n = __ldg(B.plan.key_d + row + j + 32u);
        }
        cp_async_wait<1>();  // this round's records have landed (the next round's may be in flight)
        __syncwarp();
        const float4* cur = rb + 32 * (r & 1u);
        const uint32_t gi = __match_any_sync(0xffffffffu, valid ? ki : 0x10000u + lane);
        if (valid && (gi & lt) == 0u) {  // lowest lane of its group: add the group in lane order
            float4& a = acc_i[ki];
            for (uint32_t g = gi; g; g &= g - 1u) {
                const float4 x = cur[__ffs(g) - 1];
                a.x += x.x;
                a.y += x.y;
                a.z += x.z;
            }
            a.w += (float)__popc(gi);
        }
        const uint32_t gd = __match_any_sync(0xffffffffu, valid ? kd : 0x10000u + lane);
        if (valid && (gd & lt) == 0u) {
            float2& a = acc_d[kd];
            for (uint32_t g = gd; g; g &= g - 1u) {
                const float x = cur[__ffs(g) - 1].w;
                a.x += x;
                a.y += x * x;
            }
            cnt_d[kd] += (uint16_t)__popc(gd);
        }
        __syncwarp();
        // refill the buffer just consumed with round r + 2
        const uint32_t j2 = j + 64u;
        if (j2 < m) cp_async16(rb + 32 * (r & 1u) + lane, mrec + j2);
        cp_async_commit();
        ki = ki_n;
        kd = kd_n;
    }
    cp_async_wait<0>();
    __syncwarp();
    // blend the interior texels in place (untouched ones keep their value)
    const float omh = 1.0f - V.hyst;
    const float rni = 1.0f / (float)ni, rnd = 1.0f / (float)nd;
    for (int q = lane; q < ni * ni; q += 32) {
        const int r = tile_row(q, rni), t = (r + 1) * Ti + (q - r * ni) + 1;
        const float4 a = acc_i[t];
        float4 v = irr_load(irr_raw, (size_t)t, V.fp16);
        if (a.w > 0.0f) {
            const float kf = a.w;
            const float w = fmaxf(omh, __fdividef(kf, v.w + kf));
            const float ik = __frcp_rn(kf);
            v.x += w * (a.x * ik - v.x);
            v.y += w * (a.y * ik - v.y);
            v.z += w * (a.z * ik - v.z);
            v.w = fminf(v.w + kf, 255.0f);
        }
        acc_i[t] = v;
    }
    for (int q = lane; q < nd * nd; q += 32) {
        const int r = tile_row(q, rnd), t = (r + 1) * Td + (q - r * nd) + 1;
        const float2 a = acc_d[t];
        float2 v = dep_load(dep_raw, (size_t)t, V.fp16);
        uint32_t c = dn_raw[t];
        const uint32_t k = cnt_d[t];
        if (k) {
            // the texel stores {mean, variance}; with batch mean m and batch
            // variance vb the moving average of {d, d^2} becomes
            //   mean' = mean + w (m - mean)
            //   var'  = (1-w) var + w vb + w (1-w) (m - mean)^2
            // (every term non-negative: no cancellation in storage)
            const float kf = (float)k;
            const float w = fmaxf(omh, __fdividef(kf, (float)c + kf));
            const float ik = __frcp_rn(kf);
            const float mb = a.x * ik;
            const float vb = fmaxf(a.y * ik - mb * mb, 0.0f);
            const float dm = mb - v.x;
            v.y = (1.0f - w) * v.y + w * vb + w * (1.0f - w) * dm * dm;
            v.x += w * dm;
            c = (uint32_t)fminf((float)c + kf, 255.0f);
        }
        acc_d[t] = v;
        dn_new[t] = (uint8_t)c;
    }
    __syncwarp();
    // every texel (a border texel from its octahedral fold partner) in the
    // storage format, stored in texel order (coalesced)
    const uint64_t srkey = F.pilot_key ^ (F.even ? 0x5352ull : 0x5353ull);
    for (int t = lane; t < ti2; t += 32) {
        const float4 v = acc_i[__ldg(B.src + t)];
        if (V.fp16 == 2) {
            __half2* h = reinterpret_cast<__half2*>(B.irr) + 2 * (io + t);
            const __half2 h0 = __halves2half2(half_sr(v.x, sr_bits(srkey, p, t, 0)), half_sr(v.y, sr_bits(srkey, p, t, 1)));
            const __half2 h1 = __halves2half2(half_sr(v.z, sr_bits(srkey, p, t, 2)), __float2half_rn(v.w));
            *reinterpret_cast<uint2*>(h) = make_uint2(*reinterpret_cast<const uint32_t*>(&h0),
                                                     *reinterpret_cast<const uint32_t*>(&h1));
        } else if (V.fp16) {
            __half2* h = reinterpret_cast<__half2*>(B.irr) + 2 * (io + t);
            const __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
            *reinterpret_cast<uint2*>(h) = make_uint2(*reinterpret_cast<const uint32_t*>(&h0),
                                                     *reinterpret_cast<const uint32_t*>(&h1));
        } else {
            reinterpret_cast<float4*>(B.irr)[io + t] = v;
        }
    }
    for (int t = lane; t < td2; t += 32) {
        const int src = __ldg(B.src + ti2 + t);
        const float2 v = acc_d[src];
        if (V.fp16 == 2)
            reinterpret_cast<__half2*>(B.dep)[dof + t] =
                __halves2half2(half_sr(v.x, sr_bits(srkey, p, t, 4)), half_sr(v.y, sr_bits(srkey, p, t, 5)));
        else if (V.fp16)
            reinterpret_cast<__half2*>(B.dep)[dof + t] = __floats2half2_rn(v.x, v.y);
        else
            reinterpret_cast<float2*>(B.dep)[dof + t] = v;
        B.dep_n[dof + t] = dn_new[src];
    }
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

size_t blend_plan_elems(int M)
{
    const size_t m = (size_t)(M > 0 ? M : 0);
    return 2 * (m * (m + 1) / 2) + 8;
}

BlendPlan carve_blend_plan(uint16_t* base, int M)
{
    const size_t m = (size_t)(M > 0 ? M : 0), tri = m * (m + 1) / 2;
    BlendPlan P;
    P.key_i = base;
    P.key_d = base + tri;
    return P;
}

// shared memory of one probe (one warp) of k_blend
size_t blend_smem_bytes(const VolConst& V) { return blend_layout(V.Ti, V.Td).total; }

cudaError_t launch_change(const VolConst& V, const FrameDev* FD, const ChangeBufs& B, cudaStream_t s)
{
    k_change_state<<<(V.P + 127) / 128, 128, 0, s>>>(V, FD, B);
    count_launches(1);
    k_change_weight<<<(V.P + 127) / 128, 128, 0, s>>>(V, FD, B);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_allocate(const uint32_t* W, int P, int avg, int m0, int rmax, uint32_t* n_out, uint32_t* off_out,
                            cudaStream_t s)
{
    k_allocate<<<1, kAllocThreads, 0, s>>>(W, P, avg, m0, rmax, n_out, off_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend_plan(const VolConst& V, const FrameDev* FD, const float4* sf, const BlendPlan& plan,
                              cudaStream_t s)
{
    const int M = V.rays_max - kPilots;
    if (M <= 0) return cudaSuccess;
    const uint32_t n = (uint32_t)((size_t)M * (M + 1) / 2);
    k_blend_plan<<<(n + 255) / 256, 256, 0, s>>>(V, FD, sf, plan, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s)
{
    // probes per CTA (one warp each), as many as the tuning asks and 227 KB allow
    const size_t per = blend_smem_bytes(V);
    const int wpb = std::max(1, std::min(T.blend_block / 32, (int)((227u * 1024u) / per)));
    const size_t sm = per * (size_t)wpb;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_blend, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_blend<<<(V.P + wpb - 1) / wpb, 32 * wpb, sm, s>>>(V, FD, B);
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
