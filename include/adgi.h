/*
 * adgi.h -- C ABI of the GB300 (sm_103a) per-frame probe update of
 * "Adaptive Dynamic Global Illumination" (Datta, Goli, Zhang, arXiv 2301.05125).
 *
 * One volume = a uniform probe grid with an octahedral irradiance atlas and an
 * octahedral depth-moment atlas (Sec. 3.1, Fig. probeStructure), a triangle
 * scene, and the per-probe heuristic state of Sec. 4.1.  Each adgi_update()
 * runs the whole frame on the device, in this order:
 *   1. pilot rays: 8 per probe, one per octant, directions fixed for a pair of
 *      frames (Sec. 4.4 "Improving construction efficiency");
 *   2. heuristics: f_v (Eq. ProbeVis), f_r (Sec. 4.1 "Incoming radiance"),
 *      temporal gradients (Eq. tempGradVis, tempGradIrr), trigger Tr
 *      (Fig. TrCam(a)), 5x5x5 x octant convolution, composition
 *      f_d = f_c f_v (f_dv + mu f_dr) (Eq. priorDynamic, mu = 2), quantised
 *      to integers;
 *   3. allocation of a fixed total ray budget over the probes by f_d
 *      (Sec. 3.4: the sample count is an input, decoupled from the probe count);
 *   4. tracing of every probe's rays against the scene (Alg. ApproxAlgo
 *      "evaluate sample, ray-trace") through a software BVH;
 *   5. shading: direct light with shadow rays plus a multi-bounce term
 *      albedo * Q_{t-1}(x, n) read from the atlases of the previous frame;
 *   6. blending: every sample updates its nearest texel with the moving
 *      average of Alg. MovingAvgUpdate (batched per texel, hysteresis h),
 *      followed by the octahedral border copy.
 * adgi_query_irradiance() is the 8-probe trilinear lookup with Chebyshev
 * visibility weights (Sec. 3.1; g_c of Table "List of symbols").
 *
 * Conventions for every call:
 *   - return ADGI_OK (0) or a negative ADGI_ERR_* code; adgi_last_error()
 *     returns a message for the calling thread's last failure;
 *   - every array argument is row-major, tightly packed; "host" pointers are
 *     plain host memory (pageable or pinned), "device" pointers are CUDA
 *     device memory of the volume's device;
 *   - the caller owns every array it passes; the library copies what it keeps
 *     and never frees caller memory;
 *   - all device work of a volume is ordered on the stream given at creation
 *     (adgi_set_stream() changes it); calls return once the work is enqueued
 *     unless they read results back into host memory;
 *   - a handle must not be used from two threads at once; different handles
 *     are independent.
 * Device memory is owned by the library and released by adgi_destroy().
 */
#ifndef ADGI_H
#define ADGI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADGI_OK 0
#define ADGI_ERR_INVALID_ARG (-1) /* an argument is out of range or NULL */
#define ADGI_ERR_OOM (-2)         /* a device or host allocation failed */
#define ADGI_ERR_OVER_BUDGET (-3) /* the volume does not fit the memory budget */
#define ADGI_ERR_NO_SCENE (-4)    /* adgi_update() before adgi_set_scene() */
#define ADGI_ERR_CUDA (-5)        /* a CUDA call failed (message in adgi_last_error) */
#define ADGI_ERR_TIMEOUT (-6)     /* a bounded wait gave up (adgi_server_drain, adgi_tick_sync) */

typedef struct adgi_volume_s* adgi_volume;

/* Probe grid and update parameters.  Probe (i,j,k) sits at
 * origin + spacing * (i,j,k) (FP32), with probe index i + dims[0]*(j + dims[1]*k). */
typedef struct {
    float origin[3];
    float spacing[3];
    int32_t dims[3];        /* >= 2 each */
    int32_t irr_interior;   /* irradiance tile interior n (tile n+2 with border); 8x8 tiles: 6 (Sec. 3.1) */
    int32_t depth_interior; /* depth tile interior n; 16x16 tiles: 14 */
    int32_t rays_avg;       /* fixed budget: rays_avg * probes rays per update, pilots included */
    int32_t rays_min;       /* per-probe floor; the effective floor is max(rays_min, 8) (the pilots) */
    int32_t rays_max;       /* per-probe cap, <= 4096 */
    float hysteresis;       /* h of the moving average, in [0, 1) (Table cacheDetails: 0.98 / 0.91) */
    float depth_max;        /* depth clamp and miss depth; <= 0 selects 1.5 * voxel diagonal */
    int32_t atlas_fp16;     /* 0: FP32 atlases; 1: half, blended in FP32, stored round-to-nearest;
                               2: half with seeded stochastic rounding (unbiased EMA steps);
                               3: the paper's packed 32-bit texels (Sec. "Probe irradiance cache",
                               "Probe visibility cache", appendix "Probe compression"): irradiance
                               R9 G9 B8 + 6-bit count, visibility two 13-bit moments of the distance
                               over the cage diagonal + count, log-coded and rounded down, updated by
                               one moving-average step per sample (Alg. MovingAvgUpdate, count capped
                               at 63) in sample order; hysteresis is not used */
    int32_t tr_theta;       /* trigger decay length theta in frames (Fig. TrCam(a)), >= 1, <= 255 */
    int32_t sampler;        /* 0: per-probe ray counts from the change weights (Sec. 4.2);
                               1: Metropolis chains draw the (rays_avg - 8) * P adaptive samples
                               over (probe, direction) from the static guide
                               h = exp(min(alpha g / f_s, 1)) f_s, f_s = q_c q_v / 1023^2, g the
                               cached irradiance luminance (Sec. "Adaptive sampling - static",
                               Alg. MetropolisStep); each sample also traces -w for the visibility
                               texel at -w.  Not with atlas_fp16 = 3 or adgi_autotune */
    float alpha;            /* sampler = 1: confidence alpha of the cached irradiance, >= 0 */
    int32_t dyn_ratio;      /* sampler = 1: > 0 adds the dynamic chains (Sec. "Adaptive sampling -
                               dynamic"): proxies of 3x3x3 probes, target max over the proxy of the
                               per-octant dynamic weight q_d (alpha = 0), steps 3x and 6x the static
                               ones; a sample marks its (proxy, octant) cell once per frame, and marked
                               cells in first-sample order send, within the dynamic ray budget, one ray
                               from each probe of the proxy through the centre of every irradiance
                               texel of the octant.  The adaptive budget is split static:dynamic =
                               dyn_ratio:1 (the paper's 4096:1024 chains at 4): floor(B r/(r+1)) static
                               samples, 2 (B - that) dynamic rays, ceil(C_s / r) dynamic chains; static
                               samples at probes and octants with q_d > 0 trace through texel centres.
                               0: off.  <= 1024 */
    float hysteresis_dyn;   /* dyn_ratio > 0: hysteresis of the dynamic rays' batch step, applied after
                               the static samples' (Table cacheDetails: 0.91), in [0, 1) */
    int32_t blend_mode;     /* 0: nearest texel (Alg. ApproxAlgo).  1: DDGI's cosine gather (Sec. 3.1):
                               every ray feeds every texel of its hemisphere, the irradiance texel at
                               centre direction n taking the (n . w)-weighted mean radiance over
                               n . w > 0 (tested in FP32), the visibility texel the (n . w)^50-weighted
                               mean of {d, d^2}; the number of rays with n . w > 0 is the batch count
                               of the moving average.  Only with sampler = 0 and atlas_fp16 < 3 */
    float cheb_var_floor_rel; /* the query's Chebyshev visibility weight var / (var + (d - mu)^2)
                               (one-sided bound on the filtered depth moments, as in variance shadow
                               maps, which the paper cites for g_c) takes var = mu2 - mu^2 raised to at
                               least 1e-6 s^2 (s the voxel diagonal).  A value r > 0 raises it further
                               to r * mu2: an opt-in for reduced-precision (half) atlases, whose stored
                               moments carry an error of about 1e-3 mu2.  0 (the default): the absolute
                               floor alone.  In [0, 1) */
} adgi_volume_desc;

/* kind 0: point light at pos_or_dir with intensity rgb (irradiance rgb/d^2);
 * kind 1: directional light travelling along pos_or_dir with irradiance rgb. */
typedef struct {
    int32_t kind;
    float pos_or_dir[3];
    float rgb[3];
} adgi_light;

/* Per-frame input.  frame numbers pair up as (2k, 2k+1): both frames of a pair
 * trace the same pilot rays; the change is measured on the second (Sec. 4.4). */
typedef struct {
    uint64_t frame;
    uint64_t seed;
    const adgi_light* lights; /* host array of n_lights, copied at the call */
    int32_t n_lights;         /* 0..64 */
    float sky_rgb[3];         /* radiance of rays that escape the scene */
    int32_t has_camera;       /* 1: apply the camera-distance heuristic f_c (Eq. cameraD) */
    float cam_pos[3];
    float cam_k;              /* f_c = 1 within cam_k of the camera */
    int32_t has_clip;         /* 1 (with has_camera): clip volumes (Fig. TrCam(b)) from view_proj: a
                                 probe is in V_in when |c_x|, |c_y| <= 1.2 w (w > 0, (c_x, c_y, -, w)
                                 = view_proj (p, 1) in FP32, row order) and f_c >= 0.75 (q_c >= 768),
                                 in V_out when <= 1.4 w and f_c >= 0.5 (q_c >= 512).  Outside V_out:
                                 no pilot rays, heuristic state and atlases left as they are; a pair
                                 gradient needs both frames inside V_out; only V_in probes take adaptive
                                 rays or samples (the (rays_avg - 8) * probes adaptive budget spread
                                 over V_in, capped at rays_max; culled pilots are not reassigned);
                                 V_out - V_in probes have their texel counts set down to 16
                                 (Sec. "Adaptive sampling - static", last paragraph).  0: every probe
                                 in V_in */
    float view_proj[16];      /* row-major 4x4 camera view-projection matrix */
} adgi_frame;

typedef struct {
    uint64_t frames;          /* updates run so far */
    uint64_t rays_per_update; /* rays_avg * probes: pilot + adaptive rays (Metropolis volumes:
                                 8 * probes + 2 * samples, the -w visibility rays included, plus
                                 the last update's dynamic rays) */
    uint64_t pilot_rays;      /* 8 * probes */
    uint64_t shadow_rays;     /* shadow rays of the last update (counted on the device) */
    uint32_t bvh_nodes;       /* internal nodes of the current BVH */
    uint32_t n_tris;
    uint64_t device_bytes;    /* device memory held by the volume */
    float ms_last_update;     /* device time of the last update (0 unless timing was enabled) */
    float ms_phase[8];        /* device time per phase of the last update (timing enabled):
                                 0 BVH rebuild, 1 pilot trace, 2 pilot shade, 3 heuristics,
                                 4 allocation (Metropolis: chain steps and grouping),
                                 5 adaptive trace, 6 adaptive shade, 7 blend */
    uint64_t kernels_launched; /* kernels this library has launched in the process so far */
    float ms_shadow[2];        /* device time of the shadow-ray kernel inside phases 2 and 6 (timing enabled) */
    float ms_blend_plan;       /* device time of the per-frame blend plan, which runs on a side stream
                                  beside phases 1-6 (timing enabled) */
} adgi_stats;

/* Create a volume on the current CUDA device.  desc: host pointer, copied.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  *out receives
 * the handle.  Allocates the atlases (zeroed), the heuristic state and the
 * ray buffers for rays_avg * probes rays.  Errors: INVALID_ARG (NULL
 * pointers, dims < 2, tile sizes < 1, rays_avg outside
 * [max(rays_min, 8), rays_max], hysteresis outside [0,1), theta outside
 * [1,255]), OOM, CUDA. */
int adgi_create_volume(const adgi_volume_desc* desc, void* cuda_stream, adgi_volume* out);

/* Replace the scene: n_verts xyz vertices (float[3*n_verts]), n_tris
 * triangles of vertex indices (int32[3*n_tris], counter-clockwise = front,
 * normal (B-A)x(C-A)), per-triangle albedo (float[3*n_tris]).  Pointers are
 * host memory, or device memory when ptrs_on_device = 1; they are copied.
 * The BVH is rebuilt on the volume's stream.  Errors: INVALID_ARG (an index
 * outside [0, n_verts), negative counts), OOM, CUDA. */
int adgi_set_scene(adgi_volume vol, const float* verts_xyz, int32_t n_verts, const int32_t* tri_idx,
                   int32_t n_tris, const float* tri_albedo_rgb, int32_t ptrs_on_device);

/* Overwrite vertices [first, first+count) with verts_xyz (host, or device
 * when ptrs_on_device = 1) -- moving geometry (the paper's dynamic gate,
 * Sec. 5).  The BVH is rebuilt at the next adgi_update().  Errors:
 * INVALID_ARG (range outside the scene), NO_SCENE, CUDA. */
int adgi_move_vertices(adgi_volume vol, int32_t first, int32_t count, const float* verts_xyz,
                       int32_t ptrs_on_device);

/* Run one per-frame update (steps 1-6 above) on the volume's stream.  Host
 * data of *frame is copied before return; the call does not wait for the
 * device.  Errors: INVALID_ARG, NO_SCENE, CUDA. */
int adgi_update(adgi_volume vol, const adgi_frame* frame);

/* Irradiance query at n points with normals (float[3*n] each): 8-probe
 * trilinear interpolation weighted by the one-sided Chebyshev bound of the
 * depth moments; out_rgb (float[3*n]).  Pointers are host memory (the call
 * copies in, runs, copies out and synchronises the stream) or device memory
 * when ptrs_on_device = 1 (enqueued only).  Errors: INVALID_ARG, OOM, CUDA. */
int adgi_query_irradiance(adgi_volume vol, const float* pos, const float* nrm, int32_t n, float* out_rgb,
                          int32_t ptrs_on_device);

/* Counters of the volume; synchronises the stream.  Errors: INVALID_ARG, CUDA. */
int adgi_get_stats(adgi_volume vol, adgi_stats* out);

/* Destroy the volume: waits for its stream, frees its device memory.
 * NULL is accepted. */
int adgi_destroy(adgi_volume vol);

/* ---------------------------------------------------------------------------
 * Additional entry points.
 * ------------------------------------------------------------------------- */

/* adgi_update with the device work as a CUDA graph: the first call (and any
 * call after the scene, the moving set, the shadow-job capacity or the tuning
 * changed) captures the update on the volume's stream and instantiates it;
 * later calls only rewrite the frame-descriptor node's parameters and launch
 * the graph.  Results are those of adgi_update.  No phase timing. */
int adgi_update_graph(adgi_volume vol, const adgi_frame* frame);

/* Batched update of several volumes (the batched form of the update): one
 * CUDA graph launch per tick covers every volume of the batch, each volume on
 * its own branch of the graph so that their kernels overlap on the device.
 * The graph is captured on the first tick (and again when a volume's scene,
 * moving set, shadow-job capacity or tuning changed); later ticks rewrite each
 * volume's frame-descriptor node and launch the graph once on cuda_stream.
 * A volume may belong to one live batch at a time; while a batch tick may be
 * running, order other calls on its volumes after cuda_stream (e.g. by
 * synchronising it).  Errors: INVALID_ARG (NULL, duplicates), CUDA. */
typedef struct adgi_batch_s* adgi_batch;
int adgi_batch_create(const adgi_volume* vols, int32_t n, void* cuda_stream, adgi_batch* out);
/* frames: host array of n frames, frames[i] for vols[i]. */
int adgi_batch_update(adgi_batch batch, const adgi_frame* frames);
int adgi_batch_destroy(adgi_batch batch);

/* The batched update as ONE persistent kernel launch per tick (the batched
 * form of Sec. 3.4's update with grid-wide phases): a cooperative grid of as
 * many blocks as the GPU holds at once runs the update's phases (clip classes
 * and blend plan, pilot rays and their shading, change measure, allocation,
 * adaptive rays and their shading, blend) for every volume, with a grid-wide
 * barrier between phases.  Results equal those of adgi_update on each volume
 * (same integers, same floating-point operations in the same order).  Each
 * tick copies the frame descriptors from pinned host memory, clears the
 * tick's control block and launches the kernel on cuda_stream; a volume's
 * moving part, when its vertices moved, is rebuilt inside the launch (up to
 * 2,048 triangles; a larger one before it).
 *
 * Every barrier wait gives up after a time limit (2 s unless set by
 * adgi_tick_set_wait); the blocks then return and the tick's status records
 * it: adgi_tick_sync waits for the stream and returns ADGI_ERR_TIMEOUT (the
 * volumes' state of that tick is then undefined; the next tick runs normally).
 *
 * Volumes: deterministic allocation (sampler 0) and the texel blend
 * (blend_mode 0), on the current device; their probes at most 8 x 2,048 per
 * resident block in total.  Errors: INVALID_ARG (NULL, duplicates, another
 * mode, too many probes), OOM, CUDA (no resident grid). */
typedef struct adgi_tick_s* adgi_tick;
int adgi_tick_create(const adgi_volume* vols, int32_t n, void* cuda_stream, adgi_tick* out);
/* frames: host array of n frames, frames[i] for vols[i]; enqueues one tick. */
int adgi_tick_update(adgi_tick tick, const adgi_frame* frames);
/* Wait for cuda_stream; ADGI_ERR_TIMEOUT when a wait of the last tick gave up. */
int adgi_tick_sync(adgi_tick tick);
/* Barrier wait limit in ns (1 ns .. 60 s) and a test hook: stall_barrier >= 0
 * names a barrier of the next ticks that no block arrives at, so its wait
 * runs out (-1: none).  Synchronises cuda_stream. */
int adgi_tick_set_wait(adgi_tick tick, uint64_t limit_ns, int32_t stall_barrier);
/* The persistent grid (blocks), its dynamic shared memory per block and the
 * allocation chunks of the last tick (0 before the first). */
int adgi_tick_info(adgi_tick tick, uint32_t* grid_blocks, uint32_t* smem_bytes, uint32_t* chunks);
/* Timeline of the last tick: out[i] = ns from the start of block 0 to the
 * completion of grid barrier i (0 for barriers not reached or beyond 64).
 * In order: one barrier after each phase before the allocation (clip
 * classes and blend plan; when a moving part is rebuilt in the tick, its
 * tree and its boxes; pilot trace; shadow jobs; shadow rays; pilot records;
 * change state; change weights), the allocation's own barriers, then one
 * after each later phase but the last.  Synchronises cuda_stream. */
int adgi_tick_phase_ns(adgi_tick tick, uint64_t* out, int32_t n);
int adgi_tick_destroy(adgi_tick tick);

/* Block shapes of a volume's kernels.  adgi_autotune times candidate shapes
 * of the nearest-hit traversal (64/128/256 threads), the shading wavefront
 * (prep/finish blocks 64/128/256 x shadow grid of 0 = occupancy, 2, 4, 8
 * blocks per SM) and the blend (32/64/128 threads per CTA: one warp per probe
 * tile, so 1, 2 or 4 tiles per CTA) on the
 * volume's own data and keeps the fastest; results do not depend on the
 * shapes.  It needs one update first, uses that update's rays (reps timed
 * repetitions per candidate), leaves the atlases and the heuristic state as
 * they were (blend trials run on the live atlases, restored afterwards) and
 * recomputes the last update's ray records.  Synchronises the stream. */
typedef struct {
    int32_t trace_block;
    int32_t shade_block;
    int32_t shadow_blocks_per_sm; /* 0: occupancy limit */
    int32_t blend_block;
    float ms_trace, ms_shade, ms_blend; /* best times found by adgi_autotune */
} adgi_tuning;
int adgi_autotune(adgi_volume vol, const adgi_frame* frame, int32_t reps, adgi_tuning* out);
int adgi_set_tuning(adgi_volume vol, const adgi_tuning* tuning);
int adgi_get_tuning(adgi_volume vol, adgi_tuning* tuning);

/* Use another stream for all later work of the volume (cudaStream_t). */
int adgi_set_stream(adgi_volume vol, void* cuda_stream);

/* 1: time each adgi_update() with CUDA events (adgi_stats.ms_last_update). */
int adgi_enable_timing(adgi_volume vol, int32_t enable);

/* Debug readers: copy a piece of the volume's device state into host memory
 * dst (bytes must equal adgi_state_bytes()); synchronises the stream.
 * Layouts (P probes, Ti = irr_interior+2, Td = depth_interior+2, R = main rays
 * = (rays_avg - 8) * P):
 *   ADGI_STATE_W        uint32[P]        change weight W_p of the last update
 *   ADGI_STATE_N        uint32[P]        rays of probe p (pilots included)
 *   ADGI_STATE_OFF      uint32[P+1]      exclusive prefix of n_p - 8 (main rays)
 *   ADGI_STATE_QV/QR    uint16[P][8]     quantised f_v / f_r of the last update
 *   ADGI_STATE_TRV/TRR  uint16[P][8]     trigger outputs
 *   ADGI_STATE_PILOT_HIT int32[P][8][2]  {tri (-1 miss; bit 31 = back face), t bits}
 *   ADGI_STATE_PILOT_REC float[P][8][4]  {r, g, b, depth sample}
 *   ADGI_STATE_PILOT_LUM float[P][8]     FP32 luminance of the direct light (f_r input)
 *   ADGI_STATE_MAIN_HIT int32[R][2]      as PILOT_HIT, rays in probe order
 *   ADGI_STATE_MAIN_REC float[R][4]
 *   ADGI_STATE_IRR      float[P][Ti][Ti][4] {r,g,b,count} (half[...][4] when atlas_fp16 is
 *                       1 or 2; uint32[P][Ti][Ti] packed texels when it is 3)
 *   ADGI_STATE_DEP      float[P][Td][Td][2] {mean, variance} of the depth samples (the
 *                       second moment is variance + mean^2); half[...][2] when atlas_fp16
 *                       is 1 or 2; uint32[P][Td][Td] packed texels when it is 3
 *   ADGI_STATE_DEP_MOMENTS double[P][Td][Td][2] the depth atlas as the moments {mean, mean^2}
 *                       (mean^2 = variance + mean^2 of the stored texel, formed in FP64);
 *                       FP32 and half atlases only (INVALID_ARG when atlas_fp16 is 3)
 *   ADGI_STATE_G        uint32[P][8]      per probe and octant: the sum over the octant and its
 *                       three edge neighbours of Tr_v + 2 Tr_r, which W_p sums over the
 *                       5x5x5 probes around p (step 2)
 *   ADGI_STATE_DEP_N    uint8[P][Td][Td]  depth sample counts (unused with packed texels,
 *                       which carry their own count)
 *   ADGI_STATE_ROT      float[9]          main-ray rotation of the last update
 *   ADGI_STATE_BVH_NODES bytes[max(T-1,1)][64]  nodes of the static part's BVH (T static
 *                       triangles; layout of adgi_build_bvh; zeros when T < 2)
 *   ADGI_STATE_BVH_TRIS  float[T][3][4]    static triangles in BVH order (layout of adgi_build_bvh)
 *   ADGI_STATE_MOVING_BVH_NODES / _TRIS    the same for the moving part (triangles that touch a
 *                       vertex passed to adgi_move_vertices), a linear BVH rebuilt after moves
 * Metropolis volumes (sampler = 1; B = (rays_avg - 8) * P samples, C = ceil(B / 5) chains):
 *   ADGI_STATE_MH_CHAINS  float[2][C][4]   chain states after the last update: {g.xyz, u.x},
 *                       then {u.y, 0, 0, 0} (g grid coordinates, u octahedral coordinates)
 *   ADGI_STATE_MH_SAMPLES float[B][4]      the last update's samples in chain order (sample
 *                       5c + j is the state after step K+1+j of chain c): {w.xyz, probe (int32 bits)}
 *   ADGI_STATE_MH_ORDER uint32[B]         the sample at each grouped position: by probe, then by
 *                       the Morton index of the direction's cell in a 16 x 16 octahedral grid,
 *                       then by sample index
 *   ADGI_STATE_MH_OFF   uint32[P+1]       first grouped position of each probe
 *   ADGI_STATE_MH_HIT_NEG int32[B][2]     -w hits in grouped order (as PILOT_HIT); MAIN_HIT and
 *                       MAIN_REC then hold the +w hits and records in grouped order, and N and
 *                       OFF are not computed (the chains replace the per-probe counts)
 *   ADGI_STATE_QD       uint32[P][8]      dynamic weight q_d per probe and octant (W_p is their sum)
 *   ADGI_STATE_CLS      uint8[P]          clip volume of the last update: 2 V_in, 1 V_out - V_in, 0 outside
 * Dynamic chains (dyn_ratio > 0; Cd chains, Bd = 5 Cd samples, Pp proxies, Rd = ray budget):
 *   ADGI_STATE_DYN_CHAINS  float[2][Cd][4] chain states (as MH_CHAINS, in proxy-grid units)
 *   ADGI_STATE_DYN_SAMPLES float[Bd][4]    {w.xyz, proxy (int32 bits)}, chain order
 *   ADGI_STATE_DYN_CELLS   int32[Bd]       proxy*8 + octant of each sample, -1 where the target is 0
 *   ADGI_STATE_DYN_FIRST   uint32[Pp*8]    first sample marking each cell (0xFFFFFFFF: unmarked)
 *   ADGI_STATE_DYN_INCL    uint8[Pp*8]     1: the cell's rays were traced
 *   ADGI_STATE_DYN_OFF     uint32[P+1]     first dynamic ray of each probe (off[P] = rays)
 *   ADGI_STATE_DYN_HIT     int32[Rd][2]    dynamic ray hits (as PILOT_HIT), grouped by probe:
 *                       octants in order, texels in texel order within the octant
 *   ADGI_STATE_DYN_REC     float[Rd][4]    dynamic ray records {r, g, b, depth}
 * The scene is traced as two parts: triangles that touch any vertex ever passed
 * to adgi_move_vertices form the moving part (linear BVH, rebuilt at the next
 * update after each move); the others form the static part (agglomerative
 * PLOC BVH, rebuilt only when the moving set grows).
 */
enum {
    ADGI_STATE_W = 0,
    ADGI_STATE_N = 1,
    ADGI_STATE_OFF = 2,
    ADGI_STATE_QV = 3,
    ADGI_STATE_QR = 4,
    ADGI_STATE_TRV = 5,
    ADGI_STATE_TRR = 6,
    ADGI_STATE_PILOT_HIT = 7,
    ADGI_STATE_PILOT_REC = 8,
    ADGI_STATE_PILOT_LUM = 9,
    ADGI_STATE_MAIN_HIT = 10,
    ADGI_STATE_MAIN_REC = 11,
    ADGI_STATE_IRR = 12,
    ADGI_STATE_DEP = 13,
    ADGI_STATE_DEP_N = 14,
    ADGI_STATE_ROT = 15,
    ADGI_STATE_BVH_NODES = 16,
    ADGI_STATE_BVH_TRIS = 17,
    ADGI_STATE_MOVING_BVH_NODES = 18,
    ADGI_STATE_MOVING_BVH_TRIS = 19,
    ADGI_STATE_MH_CHAINS = 20,
    ADGI_STATE_MH_SAMPLES = 21,
    ADGI_STATE_MH_ORDER = 22,
    ADGI_STATE_MH_OFF = 23,
    ADGI_STATE_MH_HIT_NEG = 24,
    ADGI_STATE_QD = 25,
    ADGI_STATE_DYN_CHAINS = 26,
    ADGI_STATE_DYN_SAMPLES = 27,
    ADGI_STATE_DYN_CELLS = 28,
    ADGI_STATE_DYN_FIRST = 29,
    ADGI_STATE_DYN_INCL = 30,
    ADGI_STATE_DYN_OFF = 31,
    ADGI_STATE_DYN_HIT = 32,
    ADGI_STATE_DYN_REC = 33,
    ADGI_STATE_CLS = 34,
    ADGI_STATE_DEP_MOMENTS = 35,
    ADGI_STATE_G = 36
};
int adgi_state_bytes(adgi_volume vol, int32_t which, uint64_t* bytes);
int adgi_read_state(adgi_volume vol, int32_t which, void* dst_host, uint64_t bytes);

/* Probe-slab split of one volume's update over several GPUs (one process and
 * one volume per GPU, each holding the whole grid's arrays; the paper runs one
 * GPU, so this has no counterpart there and only restates the update's own
 * data flow).  Rank r owns probes [p0, p1) -- whole z-planes of the grid --
 * and calls, per frame, on its volume:
 *   step 0: the frame set-up (moving-part BVH, rotation, clip classes of every
 *           probe), the pilot rays of its probes and their change state up to
 *           ADGI_STATE_G (Sec. 4.1, Sec. 4.4);
 *   --- the ranks exchange G of the two z-planes beside each slab border ---
 *   step 1: W_p of its probes (the 5x5x5 sum of G, Sec. 4.1-4.2);
 *   --- the ranks all-gather W ---
 *   step 2: the allocation of the whole budget over every W_p (identical on
 *           every rank: the integers need no collective beyond the gather),
 *           the adaptive rays of its probes (their shading reads the previous
 *           atlases wherever a ray hits) and the blend of its tiles;
 *   --- the ranks all-gather the irradiance / depth tiles (ADGI_STATE_IRR,
 *       _DEP, _DEP_N), which the next frame's shading reads anywhere ---
 * With every exchange done, each rank's probes end exactly as adgi_update
 * leaves them.  The steps run in the order 0, 1, 2 with one frame and one
 * probe range (INVALID_ARG otherwise); sampler 0 with FP32 or half atlases
 * only.  Enqueued on the volume's stream; the caller moves the data between
 * ranks (for example with NCCL on the same stream) using adgi_slab_copy. */
int adgi_update_slab(adgi_volume vol, const adgi_frame* frame, int32_t step, int32_t p0, int32_t p1);

/* Copy the part of a per-probe state array (ADGI_STATE_W, _TRV, _TRR, _G,
 * _IRR, _DEP, _DEP_N; layouts as adgi_read_state) that belongs to probes
 * [p0, p1) out to the device buffer dev_buf (into = 0) or in from it (into =
 * 1); adgi_slab_bytes gives the size.  Enqueued on the volume's stream.
 * Errors: INVALID_ARG, CUDA. */
int adgi_slab_copy(adgi_volume vol, int32_t which, int32_t p0, int32_t p1, void* dev_buf, int32_t into);
int adgi_slab_bytes(adgi_volume vol, int32_t which, int32_t p0, int32_t p1, uint64_t* bytes);

/* Fault injection for testing the failure paths (no counterpart in the
 * paper): with n > 0, the n-th device allocation a volume makes from now on
 * (adgi_create_volume's buffers, the shadow-job list, the 4-wide tree) fails
 * as cudaMalloc would when the device is full -- without allocating -- and
 * the call that made it returns ADGI_ERR_OOM after releasing what it had
 * allocated.  One failure per arming; n = 0 disarms.  Process-wide.
 * Errors: INVALID_ARG (n < 0). */
int adgi_inject_alloc_failure(int32_t n);

/* Overwrite the atlases from host memory (same layouts as ADGI_STATE_IRR /
 * _DEP / _DEP_N; any pointer may be NULL to keep that part).  For tests and
 * for restoring a saved state. */
int adgi_write_atlas(adgi_volume vol, const void* irr, const void* dep, const uint8_t* dep_n);

/* Trace n rays (origins o, directions d: float[3*n], device memory) against
 * the volume's current scene: nearest hit with t in (tmin, tmax], ties broken
 * by the smaller triangle index; writes t_out (float[n], tmax on a miss) and
 * tri_out (int32[n], -1 on a miss, bit 31 set for a back-face hit).  The same
 * watertight test and BVH as the update.  Enqueued on the volume's stream. */
int adgi_trace_closest(adgi_volume vol, const float* o, const float* d, int32_t n, float tmin, float tmax,
                       float* t_out, int32_t* tri_out);

/* Traversal work of the last update, for roofline accounting: re-traces the
 * last update's pilot and adaptive rays (and their shadow rays for the lights
 * of *frame, which must be the last update's frame) with counters, without
 * changing any state.  counts (host uint64[12]) receives, for the pilot rays
 * then for the adaptive rays: nearest-hit box tests, nearest-hit triangle
 * tests, shadow-ray box tests, shadow-ray triangle tests (a BVH node visit
 * tests the boxes of both children: 2 box tests); then for the adaptive
 * rays: [8] the sum over warps of 32 x the largest box-test count of the
 * warp's rays (a warp traverses as long as its longest ray, so
 * counts[4] / counts[8] is the lane efficiency the ray lengths allow),
 * [9] the rays traced, [10] shadow rays that found a blocker, [11] shadow
 * rays traced.  Metropolis volumes: the adaptive part counts the samples' +w
 * and -w rays and the +w rays' shadow rays.  Synchronises the stream.
 * Errors: INVALID_ARG, NO_SCENE, CUDA. */
int adgi_count_traversal(adgi_volume vol, const adgi_frame* frame, uint64_t* counts);

/* Build the linear BVH (Morton codes, stable radix sort, radix tree,
 * bottom-up child boxes enlarged by eps) for caller triangles into caller
 * buffers -- the structure adgi_update() uses for the moving part of a scene.
 *   verts:     device float[3*n_verts];  tri_idx: device int32[3*n_tris]
 *   eps:       absolute box enlargement (adgi_set_scene uses 1e-5 x the
 *              larger of the scene extent and the largest |coordinate|); a
 *              triangle's box is enlarged by at least 1e-5 x its own largest
 *              |coordinate|
 *   nodes_out: device buffer of max(n_tris-1, 1) * 64 bytes; node i holds
 *              float[12] child boxes {lo0.xyz, hi0.xyz, lo1.xyz, hi1.xyz} then
 *              int32[4] {left, right, 0, 0}: a child c >= 0 is node c, c < 0 is
 *              triangle slot ~c; node 0 is the root (n_tris >= 2)
 *   tris_out:  device float[n_tris][3][4]: the triangles in BVH order, vertex
 *              xyz + w, where w of vertex 0 holds the original triangle index
 *              as int32 bits
 * Scratch (sort keys and values, parents, flags: about 84 bytes a triangle)
 * is allocated on the stream with cudaMallocAsync and released with
 * cudaFreeAsync.  Synchronises the stream before return.  Errors:
 * INVALID_ARG (NULL pointers, negative counts, n_tris > 0 with n_verts <= 0,
 * a vertex index outside [0, n_verts): detected on the device, the build
 * then used vertex 0 for it), OOM, CUDA. */
int adgi_build_bvh(const float* verts, int32_t n_verts, const int32_t* tri_idx, int32_t n_tris, float eps,
                   void* nodes_out, void* tris_out, void* cuda_stream);

/* adgi_build_bvh without any allocation.  The paper has no counterpart: this
 * is a service for callers that may not allocate device memory while they
 * run -- a frame loop that must not stall on cudaMalloc/cudaFree (both can
 * synchronise the device), or a plugin whose host application's allocator
 * already holds all the device memory it may use.  Same arguments, outputs
 * and errors as adgi_build_bvh, with these differences:
 *   - n_tris must be <= ADGI_BVH_NOALLOC_MAX_TRIS; larger builds are rejected
 *     with ADGI_ERR_INVALID_ARG and a message naming the limit;
 *   - the scratch is one fixed device array inside the library (about
 *     2.6 MiB), held on every GPU that loads the library until exit; the call
 *     performs no cudaMalloc, cudaFree or other allocating routine;
 *   - each call looks up that array's device address in the calling thread's
 *     current CUDA context (cudaGetSymbolAddress; nothing is allocated once
 *     the library's device code is loaded there, which the first call in a
 *     context may do), so any context works, also after a device reset;
 *   - every call shares the array, which keeps the last call's contents (each
 *     call clears what must start at zero); calls whose GPU work overlaps
 *     (other streams, other host threads) race on it: order them on one
 *     stream or serialise them;
 *   - the call reads the build's error word back and synchronises the stream,
 *     so it must not be called while that stream is being captured. */
#define ADGI_BVH_NOALLOC_MAX_TRIS 32768
int adgi_build_bvh_noalloc(const float* verts, int32_t n_verts, const int32_t* tri_idx, int32_t n_tris, float eps,
                           void* nodes_out, void* tris_out, void* cuda_stream);

/* Ray allocation of step 3 as a stand-alone call on device arrays:
 * W (uint32[P]) -> n_out (uint32[P], pilots included, sum = rays_avg * P),
 * off_out (uint32[P+1], exclusive prefix of n_p - 8).  Enqueued on
 * cuda_stream.  Errors: INVALID_ARG when the budget cannot be met. */
int adgi_allocate_rays(const uint32_t* W, int32_t P, int32_t rays_avg, int32_t rays_min, int32_t rays_max,
                       uint32_t* n_out, uint32_t* off_out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over many resident volumes.
 * The paper updates one volume per frame inside one renderer; this loop is
 * the server form of that update for many clients, with no counterpart in
 * the paper.
 *
 * adgi_server_create starts a worker thread on the current device with
 * `streams` CUDA streams ("slots", 1..64) and a device-memory budget in bytes.
 * Volumes are registered with adgi_server_add_volume (desc, scene: host
 * arrays as for adgi_create_volume / adgi_set_scene, copied); the worker
 * creates and uploads them -- "admits" them -- in registration order while
 * the sum of their device footprints (estimated before creation, the true
 * figure of adgi_stats.device_bytes after) stays within the budget; a
 * volume that does not fit waits until adgi_server_remove_volume releases
 * enough memory.  adgi_server_submit queues one frame update for a volume
 * (host data copied; optional vertex move as adgi_move_vertices, applied
 * before the update).  Whenever a slot is free the worker starts the oldest
 * queued request of an idle admitted volume on it -- requests of one volume
 * run in submission order, those of different volumes overlap on the
 * device, and a request never waits for a batch boundary.  Each update is a
 * replay of the volume's captured update graph (adgi_update_graph), or a
 * plain adgi_update with ADGI_SERVER_NO_GRAPH.  With ADGI_SERVER_COALESCE a
 * request that is still queued when a newer one of the same volume is
 * dispatched is dropped and reported with status 1 (superseded): a renderer
 * wants its latest frame, not a backlog.  Results are identical to those of
 * the same requests run on a lone volume with adgi_update.
 *
 * adgi_server_poll moves up to `max` finished results into out (host
 * array), *n = count; times are seconds of a monotonic host clock (submit,
 * start on a slot, completion seen by the worker).  It returns CUDA with the
 * message of the worker's last failure once one happened.
 * adgi_server_drain waits until no request is queued or running (TIMEOUT
 * after timeout_s seconds).  adgi_server_volume hands out the handle of an
 * admitted, idle volume for queries and state reads (INVALID_ARG if it is
 * busy or not admitted); the caller must submit nothing to that volume while
 * it uses the handle.  adgi_server_destroy stops the worker, waits for the
 * streams and destroys every volume.  Errors: INVALID_ARG (NULL, unknown
 * volume, streams outside 1..64, unknown flags), OVER_BUDGET (a volume larger
 * than the whole budget), CUDA.
 * ------------------------------------------------------------------------- */
typedef struct adgi_server_s* adgi_server;
#define ADGI_SERVER_COALESCE 1
#define ADGI_SERVER_NO_GRAPH 2
typedef struct {
    uint64_t request_id; /* as returned by adgi_server_submit (from 1) */
    int32_t volume;      /* volume id */
    int32_t status;      /* ADGI_OK, 1 = superseded, or a negative ADGI_ERR_* */
    double t_submit_s, t_start_s, t_done_s;
    uint64_t rays;       /* rays of the update: rays_avg * probes (0 if superseded) */
} adgi_result;
int adgi_server_create(int32_t streams, uint64_t hbm_budget_bytes, int32_t flags, adgi_server* out);
int adgi_server_add_volume(adgi_server s, const adgi_volume_desc* desc, const float* verts_xyz, int32_t n_verts,
                           const int32_t* tri_idx, int32_t n_tris, const float* tri_albedo_rgb, int32_t* id_out);
int adgi_server_submit(adgi_server s, int32_t volume, const adgi_frame* frame, int32_t move_first,
                       int32_t move_count, const float* move_verts_xyz, uint64_t* request_id);
int adgi_server_poll(adgi_server s, adgi_result* out, int32_t max, int32_t* n);
int adgi_server_drain(adgi_server s, double timeout_s);
int adgi_server_volume(adgi_server s, int32_t volume, adgi_volume* out);
int adgi_server_remove_volume(adgi_server s, int32_t volume);
/* used: bytes charged to admitted volumes; superseded: requests dropped so
 * far; resident / waiting: admitted volumes and volumes waiting for memory. */
int adgi_server_info(adgi_server s, uint64_t* used_bytes, uint64_t* superseded, int32_t* resident,
                     int32_t* waiting);
int adgi_server_destroy(adgi_server s);

/* Message of the calling thread's last error ("" if none). */
const char* adgi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADGI_H */
