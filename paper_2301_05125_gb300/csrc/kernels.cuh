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

// Per-frame inputs of one update, kept in device memory so that a captured
// graph of the update reads each tick's values (written by k_set_frame).
struct FrameDev {
    FrameConst F;
    LightSet L;
};

// Block shapes of the launch wrappers (picked per volume by the autotuner).
struct Tuning {
    int trace_block = 128;   // pilot/adaptive nearest-hit kernels
    int shade_block = 128;   // shading prep/finish kernels
    int shadow_mult = 0;     // shadow-ray grid: blocks per SM (0: occupancy)
    int blend_block = 64;    // blend kernel threads per CTA: one warp per probe tile
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

// Per-frame blend plan, shared by every probe with the same adaptive ray
// count m: for row m of the SF table, its SF indices sorted by the texel
// their point falls in under this frame's rotation (stable: index order
// within a texel), and each texel's bucket start.  ord_* [M(M+1)/2] (row m
// at m(m-1)/2); beg_i [M][Ti^2+1], beg_d [M][Td^2+1] (row m at m-1).
struct BlendPlan {
    uint16_t* ord_i;
    uint16_t* ord_d;
    uint16_t* beg_i;
    uint16_t* beg_d;
};
size_t blend_plan_bytes(int M, int Ti, int Td);
BlendPlan carve_blend_plan(void* base, int M, int Ti, int Td);

struct BlendBufs {
    const uint32_t* off;
    const float4* sf;
    const float4* pil_rec;
    const float4* main_rec;
    void* irr;
    void* dep;
    uint8_t* dep_n;
    BlendPlan plan;
    const uint16_t* src;  // [Ti^2 + Td^2]: the texel each texel copies (itself, or a border's fold partner)
};

cudaError_t launch_set_frame(FrameDev* dst, const FrameDev& src, cudaStream_t s);
void set_frame_node_params(FrameDev** dst_slot, const FrameDev* src, cudaKernelNodeParams* kp, void** args);
cudaError_t launch_pilot_trace(const VolConst& V, const FrameDev* FD, const SceneDev& S, int2* hit, const Tuning& T,
                               cudaStream_t s);
cudaError_t launch_main_trace(const VolConst& V, const FrameDev* FD, const SceneDev& S, const uint32_t* off,
                              const float4* sf, uint32_t R, int2* hit, const Tuning& T, cudaStream_t s);
cudaError_t launch_shade(const VolConst& V, const FrameDev* FD, const SceneDev& S, int mode, uint32_t n_rays,
                         const uint32_t* off, const float4* sf, const void* irr, const void* dep, const int2* hit,
                         float4* rec, float* lum, const ShadeWork& W, const Tuning& T, cudaStream_t s,
                         cudaEvent_t* ev_shadow = nullptr);
unsigned shadow_grid_blocks(int mult);
cudaError_t launch_count(const VolConst& V, const FrameDev* FD, const SceneDev& S, const uint32_t* off,
                         const float4* sf, uint32_t R, unsigned long long* out, cudaStream_t s);
cudaError_t launch_trace_list(const SceneDev& S, const float* o, const float* d, int n, float tmin, float tmax,
                              float* t_out, int* tri_out, cudaStream_t s);

cudaError_t launch_change(const VolConst& V, const FrameDev* FD, const ChangeBufs& B, cudaStream_t s);
cudaError_t launch_allocate(const uint32_t* W, int P, int avg, int m0, int rmax, uint32_t* n_out, uint32_t* off_out,
                            cudaStream_t s);
// this frame's blend plan (needs only the frame rotation: may run beside the traces)
cudaError_t launch_blend_plan(const VolConst& V, const FrameDev* FD, const float4* sf, const BlendPlan& plan,
                              cudaStream_t s);
// the tiles (after the plan and every read of the previous atlases)
cudaError_t launch_blend(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s);
cudaError_t launch_query(const VolConst& V, const void* irr, const void* dep, const float* pos, const float* nrm, int n,
                         float* out, cudaStream_t s);

}  // namespace adgi
