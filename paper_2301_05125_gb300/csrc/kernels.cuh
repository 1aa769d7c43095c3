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
    int trace_block = 64;    // pilot/adaptive nearest-hit kernels (resident grid: 64, 128, 256 measured equal)
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
    uint32_t* qd; // per (probe, octant): the dynamic weight q_d summed into W (null: not kept)
    uint8_t* vout_even;  // [P] 1: the probe was in V_out on the last first-of-pair frame
};

// work buffers of the shading wavefront (shade.cu)
struct ShadeWork {
    unsigned long long* vis;  // per ray: bit l = light l visible
    uint4* jobs;              // shadow jobs {origin xyz, ray}
    uint8_t* job_light;       // light of each job
    unsigned* job_count;      // [4]: the jobs written, the next round of 32 jobs for the shadow kernel,
                              // the next item of the pilot and of the adaptive trace
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

// Metropolis sampling of the adaptive rays (sampler.cu): the chains' state
// and this frame's samples, grouped by probe.
constexpr int kMhSteps = 8;                        // M: random-walk steps per chain per frame
constexpr int kMhBurn = 2;                         // K: leading steps whose states are not used
constexpr int kMhPer = kMhSteps - kMhBurn - 1;     // samples per chain per frame (steps K+1..M-1)
constexpr int kMhNq = 4096;                        // normal quantile table entries
constexpr int kMhEx = 1024;                        // exp table entries
constexpr int kMhCellBits = 8;                     // direction cell below the probe in the grouping key

struct MhBufs {
    uint32_t n_samples;       // B = (rays_avg - 8) * P
    uint32_t n_chains;        // ceil(B / kMhPer)
    float alpha;              // confidence of the cached irradiance in the guide
    float inv_q2;             // 1 / 1023^2 (FP32)
    const float* nq;          // [4096] Phi^-1((i + 0.5) / 4096)
    const float* ex;          // [1024] exp(k / 1023)
    float4* chain;            // [2C]: {g.xyz, u.x} then {u.y, -, -, -}
    float4* smp;              // [B] sample direction xyz, probe (int bits) in .w, chain order
    float4* smp_g;            // [B] the same, in grouped order
    uint64_t* keys[2];        // radix sort of the samples by probe
    uint32_t* vals[2];
    uint32_t* hist;
    uint32_t* part;           // [1024] partial sums of the histogram scan
    uint32_t* off;            // [P+1] first grouped sample of each probe
    const uint16_t* lut_c;
    const uint16_t* qv;       // this frame's q_v per (probe, octant)
    const void* irr;          // previous irradiance atlas (the cache term of the guide)
    const uint32_t* qd;       // dynamic chains on: q_d per (probe, octant), else null
    float4* smp_gn;           // dynamic chains on: [B] the -w ray direction in grouped order, else null
};

// Dynamic chains over virtual proxies of 3x3x3 probes (sampler.cu).
struct DynBufs {
    uint32_t n_chains;        // ceil(C_s / dyn_ratio)
    uint32_t n_samples;       // 5 per chain
    uint32_t budget;          // dynamic rays per frame at most
    int dp[3];                // proxy grid: ceil(dims / 3)
    int pp;                   // proxies
    const float* nq;          // normal quantile table (shared with the static chains)
    const uint32_t* qd;       // [P][8] this frame's q_d
    float4* chain;            // [2Cd] states: {g.xyz, u.x}, then {u.y, ...}
    float4* smp;              // [Bd] sample direction, proxy (int bits) in .w
    int* cell;                // [Bd] proxy*8 + octant, -1 where the target is 0
    uint32_t* val;            // [Pp*8] coarsened target: max q_d over the proxy
    uint32_t* npin;           // [Pp] probes of each proxy inside V_in
    uint32_t* first;          // [Pp*8] first sample marking each cell (UINT32_MAX: none)
    uint64_t* keys[2];        // sort of the cells by first sample
    uint32_t* vals[2];
    uint32_t* hist;
    uint8_t* incl;            // [Pp*8] traced this frame
    uint32_t* off;            // [P+1] dynamic rays of each probe (counts, then offsets)
    uint32_t* part;           // [1024] partial sums of the offsets scan
    uint32_t* info;           // [2] marked cells, traced cells
    int* ntex;                // [8]
    int* tex_t;               // [8][n_irr^2]
    float4* tex_dir;          // [8][n_irr^2]
};
DynRays dyn_rays_of(const DynBufs& D);
// the per-octant texel-centre table (once per volume)
cudaError_t launch_dyn_tables(const VolConst& V, const DynBufs& D, cudaStream_t s);
cudaError_t launch_dyn_init(const VolConst& V, const DynBufs& D, uint64_t init_key, cudaStream_t s);
// target table, chain steps and marks, the budget and the per-probe ray offsets
cudaError_t launch_dyn_plan(const VolConst& V, const FrameDev* FD, const DynBufs& D, cudaStream_t s);
cudaError_t launch_dyn_trace(const VolConst& V, const SceneDev& S, const DynRays& R, uint32_t budget, int2* hit,
                             const Tuning& T, cudaStream_t s);

cudaError_t launch_mh_init(const VolConst& V, const MhBufs& M, uint64_t init_key, cudaStream_t s);
cudaError_t launch_mh_chain(const VolConst& V, const FrameDev* FD, const MhBufs& M, cudaStream_t s);
// group the samples by probe, then by direction cell (stable: sample order
// inside a cell); *ord receives the order, M.smp_g the samples in that order
cudaError_t launch_mh_group(const VolConst& V, const MhBufs& M, cudaStream_t s, const uint32_t** ord);
// the +w rays to hit_pos[0..B), the -w rays to hit_neg[0..B), in grouped order
cudaError_t launch_mh_trace(const VolConst& V, const SceneDev& S, const MhBufs& M, int2* hit_pos, int2* hit_neg,
                            const Tuning& T, cudaStream_t s);

struct MhBlendBufs {
    uint32_t n;               // samples
    const uint32_t* off;      // [P+1] grouped sample ranges
    const float4* smp_g;      // [B] samples, grouped order (the +w ray direction)
    const float4* rec;        // [B] +w records, grouped order
    const int2* hit_neg;      // [B] -w hits, grouped order
    const float4* pil_rec;
    void* irr;
    void* dep;
    uint8_t* dep_n;
    const uint16_t* src;      // border fold table (as BlendBufs::src)
    const float4* smp_gn;     // [B] the -w ray direction (dynamic chains on), else null: -smp_g
    DynRays dyn;              // dynamic rays (dynamic chains on)
    const float4* drec;       // [budget] dynamic ray records
};
cudaError_t launch_mh_blend(const VolConst& V, const FrameDev* FD, const MhBlendBufs& B, cudaStream_t s);

cudaError_t launch_set_frame(FrameDev* dst, const FrameDev& src, cudaStream_t s);
void set_frame_node_params(FrameDev** dst_slot, const FrameDev* src, cudaKernelNodeParams* kp, void** args);
// next: one device word, the work counter of the launch (cleared by it)
cudaError_t launch_pilot_trace(const VolConst& V, const FrameDev* FD, const SceneDev& S, int2* hit, unsigned* next,
                               const Tuning& T, cudaStream_t s);
cudaError_t launch_main_trace(const VolConst& V, const FrameDev* FD, const SceneDev& S, const uint32_t* off,
                              const float4* sf, uint32_t R, int2* hit, unsigned* next, const Tuning& T,
                              cudaStream_t s);
// mode 0 pilot rays, 1 adaptive rays (off, sf), 2 Metropolis samples (sf = the
// grouped samples), 3 dynamic rays (dyn; n_rays = the budget)
cudaError_t launch_shade(const VolConst& V, const FrameDev* FD, const SceneDev& S, int mode, uint32_t n_rays,
                         const uint32_t* off, const float4* sf, const void* irr, const void* dep, const int2* hit,
                         float4* rec, float* lum, const ShadeWork& W, const Tuning& T, cudaStream_t s,
                         cudaEvent_t* ev_shadow = nullptr, const DynRays* dyn = nullptr);
unsigned shadow_grid_blocks(int mult);
// smp_g: the Metropolis samples in grouped order (then R = 2B), else null
cudaError_t launch_count(const VolConst& V, const FrameDev* FD, const SceneDev& S, const uint32_t* off,
                         const float4* sf, uint32_t R, unsigned long long* out, cudaStream_t s,
                         const float4* smp_g = nullptr);
cudaError_t launch_trace_list(const SceneDev& S, const float* o, const float* d, int n, float tmin, float tmax,
                              float* t_out, int* tri_out, cudaStream_t s);

// clip volume of every probe for this frame (V.cls; 2 everywhere without a matrix)
cudaError_t launch_classify(const VolConst& V, const FrameDev* FD, const uint16_t* lut_c, uint8_t* cls,
                            cudaStream_t s);
// parts: 1 the change state (q, pair gradient, Tr, G), 2 the weights (the
// 5x5x5 sum of G -> q_d, W), 3 both; over probes [V.p_lo, V.p_hi)
cudaError_t launch_change(const VolConst& V, const FrameDev* FD, const ChangeBufs& B, cudaStream_t s, int parts = 3);
// cls: clip volumes (null: every probe in V_in, the plain rule)
cudaError_t launch_allocate(const uint32_t* W, int P, int avg, int m0, int rmax, uint32_t* n_out, uint32_t* off_out,
                            cudaStream_t s, const uint8_t* cls = nullptr);
// this frame's blend plan (needs only the frame rotation: may run beside the traces)
cudaError_t launch_blend_plan(const VolConst& V, const FrameDev* FD, const float4* sf, const BlendPlan& plan,
                              cudaStream_t s);
// the tiles (after the plan and every read of the previous atlases)
cudaError_t launch_blend(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s);
// the DDGI cosine-gather variant of the blend (blend_mode = 1; no plan needed)
cudaError_t launch_blend_cos(const VolConst& V, const FrameDev* FD, const BlendBufs& B, const Tuning& T, cudaStream_t s);
cudaError_t launch_query(const VolConst& V, const void* irr, const void* dep, const float* pos, const float* nrm, int n,
                         float* out, cudaStream_t s);

// ---- the batched update as one persistent launch per tick (tick.cu)

// The part of a tick's volume that the ray phases (traces, shadow rays)
// read; each warp keeps its own copy in shared memory (tick.cu).
struct TickWave {
    VolConst V;
    SceneDev S;
    const FrameDev* FD;
    const uint32_t* off;      // [P+1] adaptive-ray offsets
    const float4* sf;         // SF table
    int2* pil_hit;
    int2* m_hit;
    ShadeWork Wk;
    uint32_t* chunk_p;        // [R_main/32 + 1] the probe of each 32-ray chunk's first ray (allocation)
};

// One volume of a tick: what the update's ordinary kernels take as
// parameters, kept in device memory for the persistent kernel.
struct TickVol {
    TickWave w;
    const uint16_t* lut_c;
    uint8_t* cls;             // [P] clip classes (written by the first phase)
    float4* pil_rec;
    float* pil_lum;
    float4* m_rec;
    uint32_t* n;              // [P] rays per probe (the allocation's output)
    uint32_t* off;            // [P+1] adaptive-ray offsets (writable)
    ChangeBufs C;
    BlendBufs B;
    int avg, m0, rmax;        // the allocation's budget, floor and cap
    int chunk0;               // first allocation chunk of this volume
    // the moving part (nd <= kTickRebuildMax triangles), rebuilt inside the
    // tick when its vertices moved: inputs, the build's scratch, and its
    // place in the scene's arrays
    const float* verts;
    const int* idx;
    const int* dlist;         // [nd] the moving triangles
    int nv, nd;
    int node_off, tri_off;    // the moving part's first node and triangle slot
    float eps;
    float4* tri_orig;
    float4* tri_in;
    uint64_t* keys;
    uint32_t* vals;
    int* par_int;
    int* par_leaf;
    int* flags;
    uint64_t* sort_k;         // [kTickRebuildMax] the Morton sort's keys and values (global
    uint32_t* sort_v;         // memory: shared memory stays with the L1 cache the traversals use)
};

constexpr int kTickThreads = 256;  // threads per block of the persistent kernel
constexpr int kTickChunk = 2048;   // probes per allocation chunk (8 per thread)
constexpr int kTickOwn = 8;        // allocation chunks one block owns at most
constexpr int kTickPasses = 64;    // proportional allocation passes at most
constexpr int kTickPhases = 15;    // phases of a tick (grid barriers between them)
constexpr int kTickRebuildMax = 2048;  // moving parts up to this size are rebuilt inside the tick
constexpr int kTickBlendWarps = 4;     // probe tiles a block blends at once (shared memory: 4 x 3.5 KB)
constexpr int kTickScratch = 9;    // 64-bit allocation partial sums per chunk
constexpr int kTickTimedOut = 1;   // TickCtl::status: a barrier wait gave up
constexpr int kTickStamps = 64;    // barrier completion times kept per tick

// Control block of a tick (device memory).  The part up to `limit_ns` is
// cleared before every launch; the wait limit and the test hook stay.
struct TickCtl {
    unsigned bar_count;             // blocks arrived at the current barrier
    unsigned bar_gen;               // barriers completed
    int status;                     // 0, or kTickTimedOut
    unsigned pass_flag[kTickPasses];  // a chunk took part in allocation pass i
    unsigned rem_flag[2];           // a chunk took part in remainder round j (j mod 2)
    unsigned next_item[4];          // the next warp item of the pilot, adaptive, pilot-shadow, adaptive-shadow phases
    unsigned long long t_start;     // %globaltimer at the start of block 0
    unsigned long long t_bar[kTickStamps];  // %globaltimer when barrier i completed (the first kTickStamps)
    unsigned long long limit_ns;    // a barrier wait gives up after this long
    int stall;                      // test hook: barrier that never completes (-1: none)
};

// Per-volume virtual-block counts of each phase (prefix sums, host side):
// pre[ph * (nv + 1) + i] = the first virtual block of volume i in phase ph.
void tick_phase_blocks(const VolConst& V, uint32_t R_main, int nd, uint32_t counts[kTickPhases]);
// dynamic shared memory of the persistent kernel for a volume
size_t tick_smem_bytes(const VolConst& V);
// Raise kernel func's dynamic shared-memory limit on the current device to
// at least `bytes` (never lowers it: the attribute is shared by every launch
// and captured graph in the process).
cudaError_t raise_smem_limit(const void* func, size_t bytes);
// blocks of the persistent grid (all resident at once) for that shared memory, 0 on error
unsigned tick_grid_blocks(size_t smem);
// rebuild: [nv] 1 where the volume's moving part is rebuilt in this tick;
// any_rebuild: some entry is 1 (else the rebuild phases are skipped)
cudaError_t launch_tick(const TickVol* vols, int nv, const uint32_t* pre, const int* cvol, int n_chunks,
                        unsigned long long* scratch, TickCtl* ctl, const int* rebuild, int any_rebuild, unsigned grid,
                        size_t smem, cudaStream_t s);

}  // namespace adgi
