// sampler.cu -- Metropolis sampling of the adaptive rays (sm_103a).
//
// The static form of the paper's adaptive sampling (Sec. "Adaptive sampling -
// static", Alg. MetropolisStep): instead of a ray count per probe, chains of
// a random walk over (probe position, direction) draw the frame's B =
// (rays_avg - 8) * P adaptive samples from the guide
//     h(x) = exp(min(alpha * g(x) / f_s(x), 1)) * f_s(x),
//     f_s = q_c(probe) * q_v(probe, octant of w) / 1023^2,
// g = luminance of the cached irradiance texel of w (previous atlas).
// A state x = (g, u): g continuous grid coordinates in [0, dims-1]^3 (the
// probe is the nearest grid point), u octahedral coordinates in [-1, 1]^2.
// Each frame every chain takes M = 8 steps; a step proposes g + 0.5 N(0,1)
// per axis and u + sqrt(pi/256) N(0,1) per coordinate, both mirrored into
// the domain, and accepts when eps <= h(x')/h(x) (always when h(x) = 0).
// The states after steps K+1..M-1 (K = 2) are the frame's samples.
//
// Random numbers: the SplitMix64 counter hash of the pilot rays, keyed by
// (seed, frame) and counted by (chain, step, component); N(0,1) comes from a
// table of 4096 quantiles indexed by the top 12 bits, exp from a table of
// 1024 values at r = floor(1023 r) / 1023.  Every decision is exact FP32, so
// with the same atlas the chains follow the same path on any correct
// implementation.
#include "adgi_internal.cuh"
#include "bvh.cuh"
#include "kernels.cuh"

namespace adgi {

namespace {

constexpr float kLumR = 0.2126f, kLumG = 0.7152f, kLumB = 0.0722f;
constexpr float kStepG = 0.5f;          // proposal sigma in grid units
constexpr float kStepU = 0.11077321f;   // proposal sigma in octahedral units: sqrt(pi / 256)
constexpr float k2m24 = 5.9604644775390625e-08f;

__device__ __forceinline__ uint64_t mh_hash(uint64_t key, uint32_t chain, int step, int comp)
{
    return splitmix(key ^ (((uint64_t)chain * (kMhSteps + 1) + (uint64_t)step) * 8u + (uint64_t)comp));
}

__device__ __forceinline__ float mh_unif(uint64_t h) { return fm(__uint2float_rn((uint32_t)(h >> 40)), k2m24); }

// mirror x at the ends of [lo, hi], then clamp
__device__ __forceinline__ float mh_mirror(float x, float lo, float hi)
{
    if (x < lo) x = fa(lo, fs(lo, x));
    if (x > hi) x = fs(hi, fs(x, hi));
    return fminf(fmaxf(x, lo), hi);
}

// Morton index of the direction's cell in a 16 x 16 grid over the
// octahedral square: the grouping key below the probe, so that the rays of a
// probe run in a spatially coherent direction order
__device__ __forceinline__ uint32_t mh_dir_cell(float3 w)
{
    const float2 e = oct_encode_x(w);
    const uint32_t cx = (uint32_t)min(max((int)floorf(fm(fm(fa(e.x, 1.0f), 0.5f), 16.0f)), 0), 15);
    const uint32_t cy = (uint32_t)min(max((int)floorf(fm(fm(fa(e.y, 1.0f), 0.5f), 16.0f)), 0), 15);
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) m |= (((cx >> b) & 1u) << (2 * b)) | (((cy >> b) & 1u) << (2 * b + 1));
    return m;
}

// nearest probe of grid coordinates g
__device__ __forceinline__ int mh_probe_of(const VolConst& V, float gx, float gy, float gz)
{
    const int ix = min(max((int)floorf(fa(gx, 0.5f)), 0), V.dims[0] - 1);
    const int iy = min(max((int)floorf(fa(gy, 0.5f)), 0), V.dims[1] - 1);
    const int iz = min(max((int)floorf(fa(gz, 0.5f)), 0), V.dims[2] - 1);
    return ix + V.dims[0] * (iy + V.dims[1] * iz);
}

// unit direction of octahedral coordinates (ux, uy)
__device__ __forceinline__ float3 mh_oct_dir(float ux, float uy)
{
    float x = ux, y = uy;
    const float z = fs(fs(1.0f, fabsf(x)), fabsf(y));
    if (z < 0.0f) {
        const float fx = fm(fs(1.0f, fabsf(uy)), sgnf(ux));
        const float fy = fm(fs(1.0f, fabsf(ux)), sgnf(uy));
        x = fx;
        y = fy;
    }
    const float l = fsq(dot3x(x, y, z, x, y, z));
    return make_float3(fd(x, l), fd(y, l), fd(z, l));
}

// guide h at state (g, u); also returns the probe and the direction
__device__ __forceinline__ float mh_guide(const VolConst& V, const FrameConst& F, const MhBufs& M, float gx, float gy,
                                          float gz, float ux, float uy, int* probe, float3* dir)
{
    const int p = mh_probe_of(V, gx, gy, gz);
    const float3 w = mh_oct_dir(ux, uy);
    *probe = p;
    *dir = w;
    if (V.cls[p] != 2) return 0.0f;  // adaptive samples only inside V_in
    const int o = (w.x < 0.0f ? 1 : 0) | (w.y < 0.0f ? 2 : 0) | (w.z < 0.0f ? 4 : 0);
    const uint32_t q = qc_of_probe(V, F, M.lut_c, p) * (uint32_t)__ldg(M.qv + (size_t)p * 8 + o);
    const float f_s = fm(__uint2float_rn(q), M.inv_q2);
    if (!(f_s > 0.0f)) return 0.0f;
    const int t = texel_of(oct_encode_x(w), V.n_irr);
    const float4 e = irr_load(V, M.irr, (size_t)p * V.Ti * V.Ti + t);
    const float g = fa(fa(fm(kLumR, e.x), fm(kLumG, e.y)), fm(kLumB, e.z));
    float r = fd(fm(M.alpha, g), f_s);
    if (!(r < 1.0f)) r = 1.0f;
    if (r < 0.0f) r = 0.0f;
    const int k = (int)floorf(fm(r, 1023.0f));
    return fm(__ldg(M.ex + k), f_s);
}

// first states: uniform over the domain, from the volume's first frame seed
__global__ void __launch_bounds__(128) k_mh_init(VolConst V, MhBufs M, uint64_t key)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= M.n_chains) return;
    float4 a;
    a.x = fm(mh_unif(mh_hash(key, c, kMhSteps, 0)), (float)(V.dims[0] - 1));
    a.y = fm(mh_unif(mh_hash(key, c, kMhSteps, 1)), (float)(V.dims[1] - 1));
    a.z = fm(mh_unif(mh_hash(key, c, kMhSteps, 2)), (float)(V.dims[2] - 1));
    a.w = fs(fm(mh_unif(mh_hash(key, c, kMhSteps, 3)), 2.0f), 1.0f);
    const float uy = fs(fm(mh_unif(mh_hash(key, c, kMhSteps, 4)), 2.0f), 1.0f);
    M.chain[c] = a;
    M.chain[M.n_chains + c] = make_float4(uy, 0.f, 0.f, 0.f);
}

// One chain per thread: this frame's M steps and its samples
__global__ void __launch_bounds__(128) k_mh_chain(VolConst V, const FrameDev* __restrict__ FD, MhBufs M)
{
    const FrameConst& F = FD->F;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= M.n_chains) return;
    const float4 a = M.chain[c];
    float gx = a.x, gy = a.y, gz = a.z, ux = a.w, uy = M.chain[M.n_chains + c].x;
    const float hx = (float)(V.dims[0] - 1), hy = (float)(V.dims[1] - 1), hz = (float)(V.dims[2] - 1);
    int p;
    float3 w;
    float y = mh_guide(V, F, M, gx, gy, gz, ux, uy, &p, &w);
    for (int i = 0; i < kMhSteps; ++i) {
        const float gx2 = mh_mirror(fa(gx, fm(kStepG, __ldg(M.nq + (mh_hash(F.mh_key, c, i, 0) >> 52)))), 0.0f, hx);
        const float gy2 = mh_mirror(fa(gy, fm(kStepG, __ldg(M.nq + (mh_hash(F.mh_key, c, i, 1) >> 52)))), 0.0f, hy);
        const float gz2 = mh_mirror(fa(gz, fm(kStepG, __ldg(M.nq + (mh_hash(F.mh_key, c, i, 2) >> 52)))), 0.0f, hz);
        const float ux2 = mh_mirror(fa(ux, fm(kStepU, __ldg(M.nq + (mh_hash(F.mh_key, c, i, 3) >> 52)))), -1.0f, 1.0f);
        const float uy2 = mh_mirror(fa(uy, fm(kStepU, __ldg(M.nq + (mh_hash(F.mh_key, c, i, 4) >> 52)))), -1.0f, 1.0f);
        int p2;
        float3 w2;
        const float y2 = mh_guide(V, F, M, gx2, gy2, gz2, ux2, uy2, &p2, &w2);
        bool take = true;
        if (y > 0.0f) {
            const float ratio = fd(y2, y);
            take = !(ratio < 1.0f && mh_unif(mh_hash(F.mh_key, c, i, 5)) > ratio);
        }
        if (take) {
            gx = gx2, gy = gy2, gz = gz2, ux = ux2, uy = uy2, y = y2, p = p2, w = w2;
        }
        if (i > kMhBurn) {
            const uint32_t sidx = c * kMhPer + (uint32_t)(i - kMhBurn - 1);
            if (sidx < M.n_samples) {
                M.smp[sidx] = make_float4(w.x, w.y, w.z, __int_as_float(p));
                M.keys[0][sidx] = ((uint64_t)p << kMhCellBits) | mh_dir_cell(w);
                M.vals[0][sidx] = sidx;
            }
        }
    }
    M.chain[c] = make_float4(gx, gy, gz, ux);
    M.chain[M.n_chains + c] = make_float4(uy, 0.f, 0.f, 0.f);
}

// off[p] = first grouped position whose probe is >= p (keys sorted by probe,
// then direction cell), p in [0, P]
__global__ void k_mh_offsets(const uint64_t* __restrict__ keys, uint32_t n, int P, uint32_t* __restrict__ off)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P) return;
    const uint64_t key = (uint64_t)p << kMhCellBits;
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(keys + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[p] = lo;
}

// direction through the centre of tile texel t of an n x n interior:
// u = (c + 1/2)/n * 2 - 1 per axis in FP32, decoded like a chain state
__device__ __forceinline__ float3 mh_texel_centre(int t, int n)
{
    const int T = n + 2, cx = t % T - 1, cy = t / T - 1;
    const float fn = (float)n;
    return mh_oct_dir(fs(fm(fd(fa((float)cx, 0.5f), fn), 2.0f), 1.0f), fs(fm(fd(fa((float)cy, 0.5f), fn), 2.0f), 1.0f));
}

__device__ __forceinline__ int mh_octant(float3 w) { return (w.x < 0.0f ? 1 : 0) | (w.y < 0.0f ? 2 : 0) | (w.z < 0.0f ? 4 : 0); }

// the samples in grouped order: smp_g[q] = smp[ord[q]] (one gather, after
// which the traces, the shading and the blend read them contiguously).
// With the dynamic chains on (qd given), a sample whose probe and octant
// have q_d > 0 traces through texel centres: +w through the centre of its
// irradiance texel, -w through the centre of the visibility texel of -w;
// smp_gn then holds the -w ray direction.
__global__ void k_mh_permute(VolConst V, const float4* __restrict__ smp, const uint32_t* __restrict__ ord, uint32_t n,
                             float4* __restrict__ smp_g, float4* __restrict__ smp_gn, const uint32_t* __restrict__ qd)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t s = __ldg(ord + q);
    if (s >= n) {
        atomicOr(V.err, kErrRayRange);
        smp_g[q] = make_float4(0.f, 0.f, 1.f, __int_as_float(-1));
        if (smp_gn) smp_gn[q] = make_float4(0.f, 0.f, -1.f, __int_as_float(-1));
        return;
    }
    const float4 a = __ldg(smp + s);
    if (!qd) {
        smp_g[q] = a;
        return;
    }
    const int p = __float_as_int(a.w);
    const float3 w = make_float3(a.x, a.y, a.z), wn = make_float3(-a.x, -a.y, -a.z);
    float3 dp = w, dn = wn;
    if (p >= 0 && p < V.P && __ldg(qd + (size_t)p * 8 + mh_octant(w)) > 0u) {
        dp = mh_texel_centre(texel_of(oct_encode_x(w), V.n_irr), V.n_irr);
        dn = mh_texel_centre(texel_of(oct_encode_x(wn), V.n_dep), V.n_dep);
    }
    smp_g[q] = make_float4(dp.x, dp.y, dp.z, a.w);
    smp_gn[q] = make_float4(dn.x, dn.y, dn.z, a.w);
}

// ---------------------------------------------------------------- dynamic chains
// Sec. "Adaptive sampling - dynamic": proxies of 3x3x3 probes, target = max
// of q_d over the proxy in the octant (alpha = 0), steps 3x (position) and 6x
// (direction) the static ones; a sample marks its cell once per frame;
// marked cells in first-sample order are traced while the running ray count
// stays within the budget, one ray per probe of the proxy through the centre
// of every irradiance texel of the octant.
constexpr float kDynStepG = 0.5f;         // proxy units (1.5 probe spacings)
constexpr float kDynStepU = 0.66463926f;  // 6 sqrt(pi / 256)

__global__ void k_dyn_tables(VolConst V, DynBufs D)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int n = V.n_irr, T = n + 2, nn = n * n;
    for (int o = 0; o < 8; ++o) D.ntex[o] = 0;
    for (int cy = 0; cy < n; ++cy)
        for (int cx = 0; cx < n; ++cx) {
            const int t = (cy + 1) * T + (cx + 1);
            const float3 w = mh_texel_centre(t, n);
            const int o = mh_octant(w), j = D.ntex[o]++;
            D.tex_t[o * nn + j] = t;
            D.tex_dir[o * nn + j] = make_float4(w.x, w.y, w.z, 0.f);
        }
}

__global__ void __launch_bounds__(128) k_dyn_init(DynBufs D, uint64_t key)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n_chains) return;
    float4 a;
    a.x = fm(mh_unif(mh_hash(key, c, kMhSteps, 0)), (float)(D.dp[0] - 1));
    a.y = fm(mh_unif(mh_hash(key, c, kMhSteps, 1)), (float)(D.dp[1] - 1));
    a.z = fm(mh_unif(mh_hash(key, c, kMhSteps, 2)), (float)(D.dp[2] - 1));
    a.w = fs(fm(mh_unif(mh_hash(key, c, kMhSteps, 3)), 2.0f), 1.0f);
    const float uy = fs(fm(mh_unif(mh_hash(key, c, kMhSteps, 4)), 2.0f), 1.0f);
    D.chain[c] = a;
    D.chain[D.n_chains + c] = make_float4(uy, 0.f, 0.f, 0.f);
}

// target table (max of q_d over each proxy, per octant); resets the marks
__global__ void __launch_bounds__(256) k_dyn_target(VolConst V, DynBufs D)
{
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= D.pp * 8) return;
    const int q = cell >> 3, o = cell & 7;
    const int qx = q % D.dp[0], qy = (q / D.dp[0]) % D.dp[1], qz = q / (D.dp[0] * D.dp[1]);
    uint32_t m = 0, nin = 0;
    for (int z = 3 * qz; z < min(3 * qz + 3, V.dims[2]); ++z)
        for (int y = 3 * qy; y < min(3 * qy + 3, V.dims[1]); ++y)
            for (int x = 3 * qx; x < min(3 * qx + 3, V.dims[0]); ++x) {
                const size_t pi = (size_t)x + (size_t)V.dims[0] * ((size_t)y + (size_t)V.dims[1] * z);
                m = max(m, __ldg(D.qd + pi * 8 + o));
                nin += V.cls[pi] == 2;
            }
    D.val[cell] = m;
    if (o == 0) D.npin[q] = nin;  // probes of the proxy inside V_in (they alone send dynamic rays)
    D.first[cell] = 0xFFFFFFFFu;
    D.incl[cell] = 0;
}

__device__ __forceinline__ int dyn_proxy_of(const DynBufs& D, float gx, float gy, float gz)
{
    const int ix = min(max((int)floorf(fa(gx, 0.5f)), 0), D.dp[0] - 1);
    const int iy = min(max((int)floorf(fa(gy, 0.5f)), 0), D.dp[1] - 1);
    const int iz = min(max((int)floorf(fa(gz, 0.5f)), 0), D.dp[2] - 1);
    return ix + D.dp[0] * (iy + D.dp[1] * iz);
}

__global__ void __launch_bounds__(128) k_dyn_chain(const FrameDev* __restrict__ FD, DynBufs D)
{
    const FrameConst& F = FD->F;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n_chains) return;
    const float4 a = D.chain[c];
    float gx = a.x, gy = a.y, gz = a.z, ux = a.w, uy = D.chain[D.n_chains + c].x;
    const float hx = (float)(D.dp[0] - 1), hy = (float)(D.dp[1] - 1), hz = (float)(D.dp[2] - 1);
    int q = dyn_proxy_of(D, gx, gy, gz);
    float3 w = mh_oct_dir(ux, uy);
    float y = (float)__ldg(D.val + q * 8 + mh_octant(w));
    for (int i = 0; i < kMhSteps; ++i) {
        const float gx2 = mh_mirror(fa(gx, fm(kDynStepG, __ldg(D.nq + (mh_hash(F.dyn_key, c, i, 0) >> 52)))), 0.0f, hx);
        const float gy2 = mh_mirror(fa(gy, fm(kDynStepG, __ldg(D.nq + (mh_hash(F.dyn_key, c, i, 1) >> 52)))), 0.0f, hy);
        const float gz2 = mh_mirror(fa(gz, fm(kDynStepG, __ldg(D.nq + (mh_hash(F.dyn_key, c, i, 2) >> 52)))), 0.0f, hz);
        const float ux2 = mh_mirror(fa(ux, fm(kDynStepU, __ldg(D.nq + (mh_hash(F.dyn_key, c, i, 3) >> 52)))), -1.0f, 1.0f);
        const float uy2 = mh_mirror(fa(uy, fm(kDynStepU, __ldg(D.nq + (mh_hash(F.dyn_key, c, i, 4) >> 52)))), -1.0f, 1.0f);
        const int q2 = dyn_proxy_of(D, gx2, gy2, gz2);
        const float3 w2 = mh_oct_dir(ux2, uy2);
        const float y2 = (float)__ldg(D.val + q2 * 8 + mh_octant(w2));
        bool take = true;
        if (y > 0.0f) {
            const float ratio = fd(y2, y);
            take = !(ratio < 1.0f && mh_unif(mh_hash(F.dyn_key, c, i, 5)) > ratio);
        }
        if (take) {
            gx = gx2, gy = gy2, gz = gz2, ux = ux2, uy = uy2, y = y2, q = q2, w = w2;
        }
        if (i > kMhBurn) {
            const uint32_t sidx = c * kMhPer + (uint32_t)(i - kMhBurn - 1);
            if (sidx < D.n_samples) {
                const int cell = y > 0.0f ? q * 8 + mh_octant(w) : -1;
                D.smp[sidx] = make_float4(w.x, w.y, w.z, __int_as_float(q));
                D.cell[sidx] = cell;
                if (cell >= 0) atomicMin(D.first + cell, sidx);  // the first sample marks the cell
            }
        }
    }
    D.chain[c] = make_float4(gx, gy, gz, ux);
    D.chain[D.n_chains + c] = make_float4(uy, 0.f, 0.f, 0.f);
}

// sort keys of the cells: first sample (n_samples when unmarked)
__global__ void k_dyn_keys(DynBufs D)
{
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= D.pp * 8) return;
    D.keys[0][cell] = (uint64_t)min(D.first[cell], D.n_samples);
    D.vals[0][cell] = (uint32_t)cell;
}

// One block: the marked cells in first-sample order are traced while the
// running ray count stays within the budget.
__global__ void __launch_bounds__(1024) k_dyn_budget(VolConst V, DynBufs D, const uint64_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ cells)
{
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry_s;
    __shared__ unsigned marked_s, traced_s;
    const int n = D.pp * 8, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        carry_s = 0ull;
        marked_s = 0u;
        traced_s = 0u;
    }
    __syncthreads();
    for (int b = 0; b < n; b += blockDim.x) {
        const int i = b + threadIdx.x;
        bool marked = false;
        int cell = 0;
        unsigned long long rays = 0ull;
        if (i < n) {
            marked = keys[i] < (uint64_t)D.n_samples;
            cell = (int)cells[i];
            if (marked) rays = (unsigned long long)D.npin[cell >> 3] * (unsigned)__ldg(D.ntex + (cell & 7));
        }
        unsigned long long x = rays;  // inclusive scan in the block
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yv = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += yv;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned long long before = carry_s, all = 0ull;
        for (int w2 = 0; w2 < nw; ++w2) {
            if (w2 < warp) before += wsum[w2];
            all += wsum[w2];
        }
        const unsigned long long prefix = before + x;
        if (i < n && marked) {
            atomicAdd(&marked_s, 1u);
            if (prefix <= (unsigned long long)D.budget) {
                D.incl[cell] = 1;
                atomicAdd(&traced_s, 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        D.info[0] = marked_s;
        D.info[1] = traced_s;
    }
}

// dynamic rays of each probe (off[P] = 0 for the exclusive scan)
__global__ void k_dyn_count(VolConst V, DynBufs D)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > V.P) return;
    if (p == V.P) {
        D.off[p] = 0u;
        return;
    }
    const int ix = p % V.dims[0], iy = (p / V.dims[0]) % V.dims[1], iz = p / (V.dims[0] * V.dims[1]);
    const int q = ix / 3 + D.dp[0] * (iy / 3 + D.dp[1] * (iz / 3));
    uint32_t c = 0;
    if (V.cls[p] == 2)  // dynamic rays only from V_in probes
        for (int o = 0; o < 8; ++o)
            if (D.incl[q * 8 + o]) c += (uint32_t)__ldg(D.ntex + o);
    D.off[p] = c;
}

}  // namespace

cudaError_t launch_mh_init(const VolConst& V, const MhBufs& M, uint64_t init_key, cudaStream_t s)
{
    if (M.n_chains == 0) return cudaSuccess;
    k_mh_init<<<(M.n_chains + 127) / 128, 128, 0, s>>>(V, M, init_key);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mh_chain(const VolConst& V, const FrameDev* FD, const MhBufs& M, cudaStream_t s)
{
    if (M.n_chains == 0) return cudaSuccess;
    k_mh_chain<<<(M.n_chains + 127) / 128, 128, 0, s>>>(V, FD, M);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mh_group(const VolConst& V, const MhBufs& M, cudaStream_t s, const uint32_t** ord)
{
    int bits = kMhCellBits;
    while (bits < 40 && ((uint64_t)1 << bits) < ((uint64_t)V.P << kMhCellBits)) ++bits;
    int cur = 0;
    cudaError_t e = radix_sort_pairs(M.keys, M.vals, M.hist, (int)M.n_samples, bits, s, &cur, M.part);
    if (e != cudaSuccess) return e;
    *ord = M.vals[cur];
    k_mh_offsets<<<(V.P + 1 + 255) / 256, 256, 0, s>>>(M.keys[cur], M.n_samples, V.P, M.off);
    count_launches(1);
    if (M.n_samples) {
        k_mh_permute<<<(M.n_samples + 255) / 256, 256, 0, s>>>(V, M.smp, M.vals[cur], M.n_samples, M.smp_g, M.smp_gn,
                                                             M.qd);
        count_launches(1);
    }
    return cudaGetLastError();
}

DynRays dyn_rays_of(const DynBufs& D)
{
    DynRays R{};
    R.off = D.off;
    R.incl = D.incl;
    R.ntex = D.ntex;
    R.tex_t = D.tex_t;
    R.tex_dir = D.tex_dir;
    for (int k = 0; k < 3; ++k) R.dp[k] = D.dp[k];
    return R;
}

cudaError_t launch_dyn_tables(const VolConst& V, const DynBufs& D, cudaStream_t s)
{
    k_dyn_tables<<<1, 32, 0, s>>>(V, D);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dyn_init(const VolConst& V, const DynBufs& D, uint64_t init_key, cudaStream_t s)
{
    (void)V;
    if (D.n_chains == 0) return cudaSuccess;
    k_dyn_init<<<(D.n_chains + 127) / 128, 128, 0, s>>>(D, init_key);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dyn_plan(const VolConst& V, const FrameDev* FD, const DynBufs& D, cudaStream_t s)
{
    const int cells = D.pp * 8;
    k_dyn_target<<<(cells + 255) / 256, 256, 0, s>>>(V, D);
    count_launches(1);
    if (D.n_chains) {
        k_dyn_chain<<<(D.n_chains + 127) / 128, 128, 0, s>>>(FD, D);
        count_launches(1);
    }
    k_dyn_keys<<<(cells + 255) / 256, 256, 0, s>>>(D);
    count_launches(1);
    int bits = 0;
    while (bits < 40 && ((uint64_t)1 << bits) <= (uint64_t)D.n_samples) ++bits;
    int cur = 0;
    cudaError_t e = radix_sort_pairs(D.keys, D.vals, D.hist, cells, bits, s, &cur);
    if (e != cudaSuccess) return e;
    k_dyn_budget<<<1, 1024, 0, s>>>(V, D, D.keys[cur], D.vals[cur]);
    k_dyn_count<<<(V.P + 1 + 255) / 256, 256, 0, s>>>(V, D);
    count_launches(2);
    return scan_exclusive_u32(D.off, V.P + 1, D.part, s);
}

}  // namespace adgi
