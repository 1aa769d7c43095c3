// update.cu -- heuristics, ray allocation, blend and query kernels (sm_103a).
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
// One CTA per probe tile (Alg. ApproxAlgo + Alg. MovingAvgUpdate, batched).
//  1. one thread stages the probe's ray records and its old atlas tiles into
//     shared memory with bulk asynchronous copies (cp.async.bulk, completion
//     counted on an mbarrier) while the CTA bins every sample direction to its
//     nearest irradiance and depth texel;
//  2. a stable counting sort in shared memory groups the samples of each
//     texel in sample order, so each texel's sum is taken by one thread in a
//     fixed order: the blend is deterministic (no floating-point atomics);
//  3. touched texels are blended with w = max(1 - h, k/(n+k)), the octahedral
//     border is refreshed from the updated interior, and the tiles are
//     written back with coalesced 16-byte stores.

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

__device__ __forceinline__ void border_src(int i, int j, int n, int& si, int& sj)
{
    if (i == 0 && j == 0) {
        si = n;
        sj = n;
    } else if (i == 0 && j == n + 1) {
        si = n;
        sj = 1;
    } else if (i == n + 1 && j == 0) {
        si = 1;
        sj = n;
    } else if (i == n + 1 && j == n + 1) {
        si = 1;
        sj = 1;
    } else if (i == 0) {
        si = 1;
        sj = n + 1 - j;
    } else if (i == n + 1) {
        si = n;
        sj = n + 1 - j;
    } else if (j == 0) {
        si = n + 1 - i;
        sj = 1;
    } else {
        si = n + 1 - i;
        sj = n;
    }
}


constexpr int kErrWait = 16;  // a bulk copy did not complete within the wait limit

// shared-memory layout of k_blend for samples <= smax (byte offsets, 16-aligned)
struct BlendLayout {
    uint32_t rec, irr_raw, dep_raw, dn_raw, irr_new, dep_new, dn_new, key_i, key_d, ord_i, ord_d, beg_i, beg_d, cur_i,
        cur_d, total;
};

__host__ __device__ inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline BlendLayout blend_layout(int smax, int Ti, int Td)
{
    const uint32_t ti2 = (uint32_t)(Ti * Ti), td2 = (uint32_t)(Td * Td), S = (uint32_t)smax;
    BlendLayout L;
    uint32_t o = 16;  // mbarrier
    L.rec = o, o += al16(16 * S);
    L.irr_raw = o, o += al16(16 * ti2);
    L.dep_raw = o, o += al16(8 * td2);
    L.dn_raw = o, o += al16(td2);
    L.irr_new = o, o += al16(16 * ti2);
    L.dep_new = o, o += al16(8 * td2);
    L.dn_new = o, o += al16(td2);
    L.key_i = o, o += al16(2 * S);
    L.key_d = o, o += al16(2 * S);
    L.ord_i = o, o += al16(2 * S);
    L.ord_d = o, o += al16(2 * S);
    L.beg_i = o, o += al16(4 * (ti2 + 1));
    L.beg_d = o, o += al16(4 * (td2 + 1));
    L.cur_i = o, o += al16(4 * ti2);
    L.cur_d = o, o += al16(4 * td2);
    L.total = o;
    return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// exclusive scan of cnt[0..n) into beg[0..n] (beg[n] = total) and cur, by one warp
__device__ __forceinline__ void warp_scan_bins(const uint32_t* cnt, uint32_t* beg, uint32_t* cur, int n, int lane)
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
            beg[b] = carry + x - c;
            cur[b] = carry + x - c;
        }
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) beg[n] = carry;
}

// stable scatter of sample indices by key (sample order kept inside a key), by one warp
__device__ __forceinline__ void warp_stable_scatter(const uint16_t* key, uint32_t* cur, uint16_t* ord, int total,
                                                    int lane)
{
    const uint32_t lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < total; c0 += 32) {
        const int j = c0 + lane;
        const bool valid = j < total;
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

__global__ void __launch_bounds__(256) k_blend(VolConst V, const FrameDev* __restrict__ FD, BlendBufs B)
{
    const FrameConst& F = FD->F;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = blockIdx.x;
    const uint32_t base = __ldg(B.off + p);
    uint32_t m = __ldg(B.off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || base > V.R_main || m > V.R_main - base) {
        if (tid == 0) atomicOr(V.err, kErrRayRange);
        m = 0;
    }
    const int npil = F.even ? kPilots : 0;
    const int total = (int)m + npil;
    if (total == 0) return;  // untouched tile: nothing to read or write
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const int ti2 = Ti * Ti, td2 = Td * Td;
    const BlendLayout L = blend_layout(V.rays_max, Ti, Td);
    float4* rec = reinterpret_cast<float4*>(smem + L.rec);
    unsigned char* irr_raw = smem + L.irr_raw;
    unsigned char* dep_raw = smem + L.dep_raw;
    uint8_t* dn_raw = smem + L.dn_raw;
    float4* irr_new = reinterpret_cast<float4*>(smem + L.irr_new);
    float2* dep_new = reinterpret_cast<float2*>(smem + L.dep_new);
    uint8_t* dn_new = smem + L.dn_new;
    uint16_t* key_i = reinterpret_cast<uint16_t*>(smem + L.key_i);
    uint16_t* key_d = reinterpret_cast<uint16_t*>(smem + L.key_d);
    uint16_t* ord_i = reinterpret_cast<uint16_t*>(smem + L.ord_i);
    uint16_t* ord_d = reinterpret_cast<uint16_t*>(smem + L.ord_d);
    uint32_t* beg_i = reinterpret_cast<uint32_t*>(smem + L.beg_i);
    uint32_t* beg_d = reinterpret_cast<uint32_t*>(smem + L.beg_d);
    uint32_t* cur_i = reinterpret_cast<uint32_t*>(smem + L.cur_i);
    uint32_t* cur_d = reinterpret_cast<uint32_t*>(smem + L.cur_d);
    const uint32_t bar = smem_u32(smem);

    // 1. stage records (always 16-byte multiples) and, when their sizes allow
    //    16-byte bulk copies, the old tiles
    const uint32_t irr_b = (uint32_t)ti2 * (V.fp16 ? 8u : 16u), dep_b = (uint32_t)td2 * (V.fp16 ? 4u : 8u);
    const uint32_t dn_b = (uint32_t)td2;
    const bool tiles_bulk = (irr_b % 16u) == 0u && (dep_b % 16u) == 0u && (dn_b % 16u) == 0u;
    const unsigned char* g_irr = reinterpret_cast<const unsigned char*>(B.irr) + (size_t)p * irr_b;
    const unsigned char* g_dep = reinterpret_cast<const unsigned char*>(B.dep) + (size_t)p * dep_b;
    const uint8_t* g_dn = B.dep_n + (size_t)p * dn_b;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int t = tid; t < ti2; t += nthr) cur_i[t] = 0u;
    for (int t = tid; t < td2; t += nthr) cur_d[t] = 0u;
    __syncthreads();
    if (tid == 0) {
        const uint32_t tx = 16u * (uint32_t)total + (tiles_bulk ? irr_b + dep_b + dn_b : 0u);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
        if (npil) bulk_g2s(rec, B.pil_rec + (size_t)p * kPilots, 16u * kPilots, bar);
        if (m) bulk_g2s(rec + npil, B.main_rec + base, 16u * m, bar);
        if (tiles_bulk) {
            bulk_g2s(irr_raw, g_irr, irr_b, bar);
            bulk_g2s(dep_raw, g_dep, dep_b, bar);
            bulk_g2s(dn_raw, g_dn, dn_b, bar);
        }
    }
    if (!tiles_bulk) {  // odd tile sizes: plain loads (4-byte words; the counts bytewise)
        for (uint32_t t = tid; t < irr_b / 4u; t += nthr)
            reinterpret_cast<uint32_t*>(irr_raw)[t] = reinterpret_cast<const uint32_t*>(g_irr)[t];
        for (uint32_t t = tid; t < dep_b / 4u; t += nthr)
            reinterpret_cast<uint32_t*>(dep_raw)[t] = reinterpret_cast<const uint32_t*>(g_dep)[t];
        for (uint32_t t = tid; t < dn_b; t += nthr) dn_raw[t] = g_dn[t];
    }
    // sample directions -> nearest texels (the copies are in flight meanwhile)
    const float4* sfm = B.sf + (size_t)m * (m - 1) / 2;
    for (int j = tid; j < total; j += nthr) {
        float3 d = j < npil ? pilot_dir(F.pilot_key, (uint32_t)p, j) : rotate(F.R, __ldg(sfm + (j - npil)));
        float2 e = oct_encode_x(d);
        const int ki = texel_of(e, ni), kd = texel_of(e, nd);
        key_i[j] = (uint16_t)ki;
        key_d[j] = (uint16_t)kd;
        atomicAdd(cur_i + ki, 1u);  // integer counts: order-independent
        atomicAdd(cur_d + kd, 1u);
    }
    __syncthreads();
    // 2. per-texel buckets in sample order
    const int wd = nthr > 32 ? 1 : 0;  // the warp that sorts the depth keys
    if (warp == 0) warp_scan_bins(cur_i, beg_i, cur_i, ti2, lane);
    if (warp == wd) warp_scan_bins(cur_d, beg_d, cur_d, td2, lane);
    __syncthreads();
    if (warp == 0) warp_stable_scatter(key_i, cur_i, ord_i, total, lane);
    if (warp == wd) warp_stable_scatter(key_d, cur_d, ord_d, total, lane);
    // the staged data must have landed (bounded wait; on time-out the CTA
    // flags the volume and leaves the tiles as they were)
    bool ok = false;
    for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(bar, 0u);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(V.err, kErrWait);
        for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(bar, 0u);
        return;
    }
    // 3. blend the touched interior texels
    const float omh = 1.0f - V.hyst;
    for (int t = tid; t < ti2; t += nthr) {
        const int i = t / Ti, jj = t - i * Ti;
        if (i < 1 || i > ni || jj < 1 || jj > ni) continue;
        float4 v;
        if (V.fp16) {
            const __half2* h = reinterpret_cast<const __half2*>(irr_raw) + 2 * t;
            float2 a = __half22float2(h[0]), b2 = __half22float2(h[1]);
            v = make_float4(a.x, a.y, b2.x, b2.y);
        } else {
            v = reinterpret_cast<const float4*>(irr_raw)[t];
        }
        const uint32_t b0 = beg_i[t], b1 = beg_i[t + 1];
        if (b1 > b0) {
            float sx = 0.f, sy = 0.f, sz = 0.f;
            for (uint32_t q = b0; q < b1; ++q) {
                const float4 r = rec[ord_i[q]];
                sx += r.x;
                sy += r.y;
                sz += r.z;
            }
            const float k = (float)(b1 - b0);
            const float w = fmaxf(omh, k / (v.w + k));
            const float ik = 1.0f / k;
            v.x += w * (sx * ik - v.x);
            v.y += w * (sy * ik - v.y);
            v.z += w * (sz * ik - v.z);
            v.w = fminf(v.w + k, 255.0f);
        }
        irr_new[t] = v;
    }
    for (int t = tid; t < td2; t += nthr) {
        const int i = t / Td, jj = t - i * Td;
        if (i < 1 || i > nd || jj < 1 || jj > nd) continue;
        float2 v = V.fp16 ? __half22float2(reinterpret_cast<const __half2*>(dep_raw)[t])
                          : reinterpret_cast<const float2*>(dep_raw)[t];
        uint32_t c = dn_raw[t];
        const uint32_t b0 = beg_d[t], b1 = beg_d[t + 1];
        if (b1 > b0) {
            // the texel stores {mean, variance}; with batch mean m and batch
            // variance vb the moving average of {d, d^2} becomes
            //   mean' = mean + w (m - mean)
            //   var'  = (1-w) var + w vb + w (1-w) (m - mean)^2
            // (every term non-negative: no cancellation in storage)
            float s1 = 0.f, s2 = 0.f;
            for (uint32_t q = b0; q < b1; ++q) {
                const float d = rec[ord_d[q]].w;
                s1 += d;
                s2 += d * d;
            }
            const float k = (float)(b1 - b0);
            const float w = fmaxf(omh, k / ((float)c + k));
            const float ik = 1.0f / k;
            const float mb = s1 * ik;
            const float vb = fmaxf(s2 * ik - mb * mb, 0.0f);
            const float dm = mb - v.x;
            v.y = (1.0f - w) * v.y + w * vb + w * (1.0f - w) * dm * dm;
            v.x += w * dm;
            c = (uint32_t)fminf((float)c + k, 255.0f);
        }
        dep_new[t] = v;
        dn_new[t] = (uint8_t)c;
    }
    __syncthreads();
    // 4. every texel (border ones from their octahedral fold partner) in the
    //    storage format, into the staging buffers
    const uint64_t srkey = F.pilot_key ^ (F.even ? 0x5352ull : 0x5353ull);
    for (int t = tid; t < ti2; t += nthr) {
        const int i = t / Ti, jj = t - i * Ti;
        int src = t;
        if (i < 1 || i > ni || jj < 1 || jj > ni) {
            int si, sj;
            border_src(i, jj, ni, si, sj);
            src = si * Ti + sj;
        }
        const float4 v = irr_new[src];
        if (V.fp16 == 2) {
            __half2* h = reinterpret_cast<__half2*>(irr_raw) + 2 * t;
            h[0] = __halves2half2(half_sr(v.x, sr_bits(srkey, p, t, 0)), half_sr(v.y, sr_bits(srkey, p, t, 1)));
            h[1] = __halves2half2(half_sr(v.z, sr_bits(srkey, p, t, 2)), __float2half_rn(v.w));
        } else if (V.fp16) {
            __half2* h = reinterpret_cast<__half2*>(irr_raw) + 2 * t;
            h[0] = __floats2half2_rn(v.x, v.y);
            h[1] = __floats2half2_rn(v.z, v.w);
        } else {
            reinterpret_cast<float4*>(irr_raw)[t] = v;
        }
    }
    for (int t = tid; t < td2; t += nthr) {
        const int i = t / Td, jj = t - i * Td;
        int src = t;
        if (i < 1 || i > nd || jj < 1 || jj > nd) {
            int si, sj;
            border_src(i, jj, nd, si, sj);
            src = si * Td + sj;
        }
        const float2 v = dep_new[src];
        if (V.fp16 == 2)
            reinterpret_cast<__half2*>(dep_raw)[t] =
                __halves2half2(half_sr(v.x, sr_bits(srkey, p, t, 4)), half_sr(v.y, sr_bits(srkey, p, t, 5)));
        else if (V.fp16)
            reinterpret_cast<__half2*>(dep_raw)[t] = __floats2half2_rn(v.x, v.y);
        else
            reinterpret_cast<float2*>(dep_raw)[t] = v;
        dn_raw[t] = dn_new[src];
    }
    __syncthreads();
    // 5. coalesced write-back: 16-byte stores when the tile sizes allow
    unsigned char* o_irr = reinterpret_cast<unsigned char*>(B.irr) + (size_t)p * irr_b;
    unsigned char* o_dep = reinterpret_cast<unsigned char*>(B.dep) + (size_t)p * dep_b;
    uint8_t* o_dn = B.dep_n + (size_t)p * dn_b;
    if (tiles_bulk) {
        for (uint32_t t = tid; t < irr_b / 16u; t += nthr)
            reinterpret_cast<uint4*>(o_irr)[t] = reinterpret_cast<const uint4*>(irr_raw)[t];
        for (uint32_t t = tid; t < dep_b / 16u; t += nthr)
            reinterpret_cast<uint4*>(o_dep)[t] = reinterpret_cast<const uint4*>(dep_raw)[t];
        for (uint32_t t = tid; t < dn_b / 16u; t += nthr)
            reinterpret_cast<uint4*>(o_dn)[t] = reinterpret_cast<const uint4*>(dn_raw)[t];
    } else {
        for (uint32_t t = tid; t < irr_b / 4u; t += nthr)
            reinterpret_cast<uint32_t*>(o_irr)[t] = reinterpret_cast<const uint32_t*>(irr_raw)[t];
        for (uint32_t t = tid; t < dep_b / 4u; t += nthr)
            reinterpret_cast<uint32_t*>(o_dep)[t] = reinterpret_cast<const uint32_t*>(dep_raw)[t];
        for (uint32_t t = tid; t < dn_b; t += nthr) o_dn[t] = dn_raw[t];
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

size_t blend_smem_bytes(const VolConst& V) { return blend_layout(V.rays_max, V.Ti, V.Td).total; }

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

cudaError_t launch_blend(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s)
{
    size_t sm = blend_smem_bytes(V);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_blend, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_blend<<<V.P, T.blend_block, sm, s>>>(V, FD, B);
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
