// update.cu -- heuristics, ray allocation, blend and query kernels (sm_103a).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include <cooperative_groups.h>

#include "adgi_internal.cuh"
#include "kernels.cuh"
#include "phase.cuh"

namespace adgi {

namespace {


__global__ void __launch_bounds__(256) k_classify(VolConst V, const FrameDev* __restrict__ FD,
                                                  const uint16_t* __restrict__ lut_c, uint8_t* __restrict__ cls)
{
    classify_body(V, FD, lut_c, cls, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_change_state(VolConst V, const FrameDev* __restrict__ FD, ChangeBufs B)
{
    change_state_body(V, FD, B, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_change_weight(VolConst V, const FrameDev* __restrict__ FD, ChangeBufs B)
{
    change_weight_body<false>(V, FD, B, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_blend_plan(VolConst V, const FrameDev* __restrict__ FD,
                                                    const float4* __restrict__ sf, BlendPlan Pl)
{
    blend_plan_body(V, FD, sf, Pl, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_blend(VolConst V, const FrameDev* __restrict__ FD, BlendBufs B)
{
    blend_body<false>(V, FD, B, blockIdx.x, blockDim.x >> 5);
}

// ============================================================== allocation
// One CTA of 1024 threads; thread t owns the contiguous probe chunk
// [t*chunk, (t+1)*chunk).  Integer water-filling of the extra budget by W,
// capped, then the remainder one ray per probe in index order.
constexpr int kAllocThreads = 1024;
constexpr int kAllocIters = 64;


// With clip volumes (cls given) only V_in probes (cls 2) take adaptive rays:
// floors m0 in V_in, 8 (the pilots) in V_out - V_in, 0 outside; beyond the
// V_in floors E = (avg - 8) P - (m0 - 8) |V_in| is spread over V_in, capped
// at rmax - m0 per probe.  Without cls every probe is in V_in and E =
// (avg - m0) P.

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
cudaError_t raise_smem_limit(const void* func, size_t bytes)
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
