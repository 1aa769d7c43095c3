// shade.cu -- shading of probe rays as a three-kernel wavefront (sm_103a).
//
//   prep:    per ray, for a front-face hit: exact FP32 normal, hit point and
//            biased shadow origin; every light passing the exact lit test
//            appends one shadow job {origin, ray, light} (warp-aggregated);
//   shadow:  a persistent grid walks the compacted jobs, one any-hit
//            traversal per job, and sets the light's bit in the ray's
//            visibility mask when nothing blocks it;
//   finish:  per ray, direct light of the visible lights (exact FP32, light
//            order fixed), the multi-bounce term albedo * Q_{t-1}(x, n) and the
//            ray record {rgb, depth}.
// Splitting the shadow rays out keeps SIMT lanes busy: a thread no longer
// loops over lights while its neighbours missed the scene or faced away.
#include "adgi_internal.cuh"
#include "kernels.cuh"
#include "wave.cuh"

namespace adgi {

namespace {

__global__ void __launch_bounds__(256) k_shade_prep(VolConst V, const FrameDev* __restrict__ FD, SceneDev S,
                                                    RaySet Rs, const int2* __restrict__ hit,
                                                    unsigned long long* __restrict__ vis, uint4* __restrict__ jobs,
                                                    uint8_t* __restrict__ job_light, unsigned* __restrict__ job_count,
                                                    unsigned job_cap)
{
    shade_prep_body<false>(V, FD, S, Rs, hit, vis, jobs, job_light, job_count, job_cap, blockIdx.x);
}

__global__ void __launch_bounds__(128, 8) k_shadow(const FrameDev* __restrict__ FD, SceneDev S,
                                                const uint4* __restrict__ jobs, const uint8_t* __restrict__ job_light,
                                                const unsigned* __restrict__ job_count, unsigned job_cap,
                                                unsigned long long* __restrict__ vis, unsigned long long* shadow_ctr,
                                                unsigned* next_round)
{
    shadow_body(FD, S, jobs, job_light, job_count, job_cap, vis, shadow_ctr, next_round,
                blockIdx.x == 0 && threadIdx.x == 0);
}

__global__ void __launch_bounds__(256, 4) k_shade_finish(VolConst V, const FrameDev* __restrict__ FD, SceneDev S,
                                                      RaySet Rs, const int2* __restrict__ hit,
                                                      const unsigned long long* __restrict__ vis,
                                                      const void* __restrict__ irr, const void* __restrict__ dep,
                                                      float4* __restrict__ rec, float* __restrict__ lum)
{
    shade_finish_body<false>(V, FD, S, Rs, hit, vis, irr, dep, rec, lum, blockIdx.x);
}

}  // namespace

unsigned shadow_grid_blocks(int mult)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_shadow, 128, 0);
    if (sms <= 0) sms = 152;
    if (per <= 0) per = 4;
    if (mult > 0 && mult < per) per = mult;
    return (unsigned)(sms * per);
}

cudaError_t launch_shade(const VolConst& V, const FrameDev* FD, const SceneDev& S, int mode, uint32_t n_rays,
                         const uint32_t* off, const float4* sf, const void* irr, const void* dep, const int2* hit,
                         float4* rec, float* lum, const ShadeWork& W, const Tuning& T, cudaStream_t s,
                         cudaEvent_t* ev_shadow, const DynRays* dyn)
{
    if (n_rays == 0) return cudaSuccess;
    RaySet Rs{mode, n_rays, off, sf, dyn ? *dyn : DynRays{}};
    const unsigned b = (unsigned)T.shade_block;
    const unsigned nb = (n_rays + b - 1) / b;
    cudaError_t e = cudaMemsetAsync(W.job_count, 0, 2 * sizeof(unsigned), s);  // the count and the round counter
    if (e != cudaSuccess) return e;
    k_shade_prep<<<nb, b, 0, s>>>(V, FD, S, Rs, hit, W.vis, W.jobs, W.job_light, W.job_count, W.job_cap);
    count_launches(1);
    if (ev_shadow && (e = cudaEventRecord(ev_shadow[0], s)) != cudaSuccess) return e;
    k_shadow<<<W.shadow_blocks, 128, 0, s>>>(FD, S, W.jobs, W.job_light, W.job_count, W.job_cap, W.vis,
                                             W.shadow_ctr, W.job_count + 1);
    count_launches(1);
    if (ev_shadow && (e = cudaEventRecord(ev_shadow[1], s)) != cudaSuccess) return e;
    k_shade_finish<<<nb, b, 0, s>>>(V, FD, S, Rs, hit, W.vis, irr, dep, rec, lum);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adgi
