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
// One CTA per probe tile (Alg. ApproxAlgo + Alg. MovingAvgUpdate, batched):
// the probe's samples are binned to their nearest texel in shared memory, the
// touched texels are blended with w = max(1 - h, k/(n+k)), the octahedral
// border is refreshed, and the tiles are written back with coalesced stores.

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

__global__ void __launch_bounds__(256) k_blend(VolConst V, const FrameDev* __restrict__ FD, BlendBufs B)
{
    const FrameConst& F = FD->F;
    const int nthr = blockDim.x;
    extern __shared__ float4 smem4[];
    const int p = blockIdx.x;
    const uint32_t base = __ldg(B.off + p);
    uint32_t m = __ldg(B.off + p + 1) - base;
    if (m > (uint32_t)(V.rays_max - kPilots) || base > V.R_main || m > V.R_main - base) {
        if (threadIdx.x == 0) atomicOr(V.err, kErrRayRange);
        m = 0;
    }
    const int npil = F.even ? kPilots : 0;
    const int total = (int)m + npil;
    if (total == 0) return;  // untouched tile: nothing to read or write
    const int Ti = V.Ti, Td = V.Td, ni = V.n_irr, nd = V.n_dep;
    const int ti2 = Ti * Ti, td2 = Td * Td;
    float4* tile_i = smem4;                                        // [ti2]
    float4* acc_i = tile_i + ti2;                                  // [ti2] sum rgb, k
    float2* tile_d = reinterpret_cast<float2*>(acc_i + ti2);       // [td2]
    float* acc_d = reinterpret_cast<float*>(tile_d + td2);         // [td2*3]
    uint32_t* cnt_d = reinterpret_cast<uint32_t*>(acc_d + 3 * td2);  // [td2]
    const int tid = threadIdx.x;
    for (int t = tid; t < ti2; t += nthr) acc_i[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = tid; t < 3 * td2; t += nthr) acc_d[t] = 0.f;
    __syncthreads();
    for (int j = tid; j < total; j += nthr) {
        float3 d;
        float4 rec;
        if (j < npil) {
            d = pilot_dir(F.pilot_key, (uint32_t)p, j);
            rec = B.pil_rec[(size_t)p * kPilots + j];
        } else {
            uint32_t i = (uint32_t)(j - npil);
            float4 s = __ldg(B.sf + (size_t)m * (m - 1) / 2 + i);
            d = rotate(F.R, s);
            rec = B.main_rec[base + i];
        }
        float2 e = oct_encode_x(d);
        int ti = texel_of(e, ni);
        int td = texel_of(e, nd);
        float* ai = reinterpret_cast<float*>(acc_i + ti);
        atomicAdd(ai + 0, rec.x);
        atomicAdd(ai + 1, rec.y);
        atomicAdd(ai + 2, rec.z);
        atomicAdd(ai + 3, 1.0f);
        atomicAdd(acc_d + 3 * td + 0, rec.w);
        atomicAdd(acc_d + 3 * td + 1, rec.w * rec.w);
        atomicAdd(acc_d + 3 * td + 2, 1.0f);
    }
    // stage the old tiles
    const size_t io = (size_t)p * ti2, dof = (size_t)p * td2;
    for (int t = tid; t < ti2; t += nthr) tile_i[t] = irr_load(B.irr, io + t, V.fp16);
    for (int t = tid; t < td2; t += nthr) {
        tile_d[t] = dep_load(B.dep, dof + t, V.fp16);
        cnt_d[t] = B.dep_n[dof + t];
    }
    __syncthreads();
    const float omh = 1.0f - V.hyst;
    for (int t = tid; t < ti2; t += nthr) {
        float4 a = acc_i[t];
        if (a.w > 0.f) {
            float4 v = tile_i[t];
            float w = fmaxf(omh, a.w / (v.w + a.w));
            float ik = 1.0f / a.w;
            v.x += w * (a.x * ik - v.x);
            v.y += w * (a.y * ik - v.y);
            v.z += w * (a.z * ik - v.z);
            v.w = fminf(v.w + a.w, 255.0f);
            tile_i[t] = v;
        }
    }
    for (int t = tid; t < td2; t += nthr) {
        float k = acc_d[3 * t + 2];
        if (k > 0.f) {
            // the texel stores {mean, variance}; with batch mean m and batch
            // variance vb the moving average of {d, d^2} becomes
            //   mean' = mean + w (m - mean)
            //   var'  = (1-w) var + w vb + w (1-w) (m - mean)^2
            // (every term non-negative: no cancellation in storage)
            float2 v = tile_d[t];
            float c = (float)cnt_d[t];
            float w = fmaxf(omh, k / (c + k));
            float ik = 1.0f / k;
            float m = acc_d[3 * t] * ik;
            float vb = fmaxf(acc_d[3 * t + 1] * ik - m * m, 0.0f);
            float dm = m - v.x;
            v.y = (1.0f - w) * v.y + w * vb + w * (1.0f - w) * dm * dm;
            v.x += w * dm;
            tile_d[t] = v;
            cnt_d[t] = (uint32_t)fminf(c + k, 255.0f);
        }
    }
    __syncthreads();
    // border texels copy their octahedral fold partners (interior, updated)
    for (int t = tid; t < ti2; t += nthr) {
        int i = t / Ti, j = t - i * Ti;
        if (i >= 1 && i <= ni && j >= 1 && j <= ni) continue;
        int si, sj;
        border_src(i, j, ni, si, sj);
        tile_i[t] = tile_i[si * Ti + sj];
    }
    for (int t = tid; t < td2; t += nthr) {
        int i = t / Td, j = t - i * Td;
        if (i >= 1 && i <= nd && j >= 1 && j <= nd) continue;
        int si, sj;
        border_src(i, j, nd, si, sj);
        tile_d[t] = tile_d[si * Td + sj];
        cnt_d[t] = cnt_d[si * Td + sj];
    }
    __syncthreads();
    if (V.fp16 == 2) {  // stochastic rounding, seeded by the frame, probe, texel and channel
        const uint64_t key = F.pilot_key ^ (F.even ? 0x5352ull : 0x5353ull);
        __half2* hi = reinterpret_cast<__half2*>(B.irr) + 2 * io;
        for (int t = tid; t < ti2; t += nthr) {
            float4 v = tile_i[t];
            hi[2 * t] = __halves2half2(half_sr(v.x, sr_bits(key, p, t, 0)), half_sr(v.y, sr_bits(key, p, t, 1)));
            hi[2 * t + 1] = __halves2half2(half_sr(v.z, sr_bits(key, p, t, 2)), __float2half_rn(v.w));
        }
        __half2* hd = reinterpret_cast<__half2*>(B.dep) + dof;
        for (int t = tid; t < td2; t += nthr)
            hd[t] = __halves2half2(half_sr(tile_d[t].x, sr_bits(key, p, t, 4)), half_sr(tile_d[t].y, sr_bits(key, p, t, 5)));
    } else if (V.fp16) {
        __half2* hi = reinterpret_cast<__half2*>(B.irr) + 2 * io;
        for (int t = tid; t < ti2; t += nthr) {
            float4 v = tile_i[t];
            hi[2 * t] = __floats2half2_rn(v.x, v.y);
            hi[2 * t + 1] = __floats2half2_rn(v.z, v.w);
        }
        __half2* hd = reinterpret_cast<__half2*>(B.dep) + dof;
        for (int t = tid; t < td2; t += nthr) hd[t] = __floats2half2_rn(tile_d[t].x, tile_d[t].y);
    } else {
        float4* gi = reinterpret_cast<float4*>(B.irr) + io;
        for (int t = tid; t < ti2; t += nthr) gi[t] = tile_i[t];
        float2* gd = reinterpret_cast<float2*>(B.dep) + dof;
        for (int t = tid; t < td2; t += nthr) gd[t] = tile_d[t];
    }
    for (int t = tid; t < td2; t += nthr) B.dep_n[dof + t] = (uint8_t)cnt_d[t];
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

size_t blend_smem_bytes(const VolConst& V)
{
    size_t ti2 = (size_t)V.Ti * V.Ti, td2 = (size_t)V.Td * V.Td;
    return ti2 * 16 * 2 + td2 * 8 + td2 * 12 + td2 * 4;
}

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
