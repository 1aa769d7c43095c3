// kernels.cuh -- launch wrappers of the update's kernels (host side).
#pragma once
#include <cuda_runtime.h>

#include "adgi_internal.cuh"

namespace adgi {

// process-wide count of kernels launched by this library (launch wrappers add to it)
void count_launches(unsigned n);
unsigned long long kernels_launched();

struct LightSet {
    int n;
    Light l[kMaxLights];
};

struct ChangeBufs {
    const int2* pil_hit;
    const float* pil_lum;
    const uint16_t* lut_v;
    const uint16_t* lut_c;
    uint16_t* qv;
    uint16_t* qr;
    uint16_t* qv_even;
    uint16_t* qr_even;
    uint16_t* amp_v;
    uint16_t* amp_r;
    uint8_t* age_v;
    uint8_t* age_r;
    uint16_t* trv;
    uint16_t* trr;
    uint32_t* G;  // per (probe, octant): octant-neighbourhood sum of trv + 2 trr
    uint32_t* W;
};

// work buffers of the shading wavefront (shade.cu)
struct ShadeWork {
    unsigned long long* vis;  // per ray: bit l = light l visible
    uint4* jobs;              // shadow jobs {origin xyz, ray}
    uint8_t* job_light;       // light of each job
    unsigned* job_count;
    unsigned job_cap;
    unsigned shadow_blocks;   // persistent grid of the shadow kernel
    unsigned long long* shadow_ctr;
};

struct BlendBufs {
    const uint32_t* off;
    const float4* sf;
    const float4* pil_rec;
    const float4* main_rec;
    void* irr;
    void* dep;
    uint8_t* dep_n;
};

cudaError_t launch_pilot_trace(const VolConst& V, const FrameConst& F, const SceneDev& S, int2* hit, cudaStream_t s);
cudaError_t launch_main_trace(const VolConst& V, const FrameConst& F, const SceneDev& S, const uint32_t* off,
                              const float4* sf, uint32_t R, int2* hit, cudaStream_t s);
cudaError_t launch_shade(const VolConst& V, const FrameConst& F, const LightSet& L, const SceneDev& S, int mode,
                         uint32_t n_rays, const uint32_t* off, const float4* sf, const void* irr, const void* dep,
                         const int2* hit, float4* rec, float* lum, int bounce, const ShadeWork& W, cudaStream_t s);
unsigned shadow_grid_blocks();
cudaError_t launch_count(const VolConst& V, const FrameConst& F, const LightSet& L, const SceneDev& S,
                         const uint32_t* off, const float4* sf, uint32_t R, unsigned long long* out, cudaStream_t s);
cudaError_t launch_trace_list(const SceneDev& S, const float* o, const float* d, int n, float tmin, float tmax,
                              float* t_out, int* tri_out, cudaStream_t s);

cudaError_t launch_change(const VolConst& V, const FrameConst& F, const ChangeBufs& B, cudaStream_t s);
cudaError_t launch_allocate(const uint32_t* W, int P, int avg, int m0, int rmax, uint32_t* n_out, uint32_t* off_out,
                            cudaStream_t s);
cudaError_t launch_blend(const VolConst& V, const FrameConst& F, const BlendBufs& B, cudaStream_t s);
cudaError_t launch_query(const VolConst& V, const void* irr, const void* dep, const float* pos, const float* nrm, int n,
                         float* out, cudaStream_t s);

}  // namespace adgi
