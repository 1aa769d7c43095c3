// capi.cu -- host runtime behind include/adgi.h: volume objects, device memory,
// per-frame constants, and the ordered launch sequence of one update.
//
// Host-side tables (built once per volume, in FP64 with only IEEE basic
// operations plus exp for the two heuristic LUTs; compiled with
// -ffp-contract=off so the rounding is that of the written order):
//   * spherical Fibonacci sets SF_m, m = 1..rays_max-8 (Keinert et al. 2015),
//     cos/sin of i * golden angle by the exact complex recurrence;
//   * LUT_v[i] = floor(1023 exp(-2 (i+0.5)/256))   (Eq. ProbeVis, bin s/256)
//   * LUT_c[i] = floor(1023 exp(-(i+0.5) s/64))    (Eq. cameraD, bin s/64)
// Per frame: the pilot hash key of the frame pair and the main-ray rotation (a
// uniform unit quaternion by rejection from the 4-ball, FP64 -> FP32).
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "adgi_internal.cuh"
#include "bvh.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <atomic>
#include <tuple>

namespace adgi {
size_t blend_smem_bytes(const VolConst& V);

static std::atomic<unsigned long long> g_launches{0};
const char* noalloc_fail(const std::string& msg);
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long kernels_launched() { return g_launches.load(std::memory_order_relaxed); }
}

using namespace adgi;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return fail(ADGI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

const double kGaCos = -0.7373688780783197;  // cos(pi (3 - sqrt 5))
const double kGaSin = 0.6754902942615238;   // sin(pi (3 - sqrt 5))

// Spherical Fibonacci sets SF_m, m = 1..M, one row of m points per m.  Row m
// lists its points in the order of a Morton curve over their octahedral
// coordinates, and .w holds each point's SF index i (int bits): a warp that
// takes 32 consecutive positions traces a compact cone of directions, while
// every result is still stored under its SF index.
void build_sf(int M, std::vector<float4>& out)
{
    out.resize((size_t)M * (M + 1) / 2 + 1);
    std::vector<float4> pts;
    std::vector<std::pair<uint32_t, int>> order;
    auto spread = [](uint32_t x) {  // 10 bits -> every second bit
        x &= 0x3FFu;
        x = (x | (x << 8)) & 0x00FF00FFu;
        x = (x | (x << 4)) & 0x0F0F0F0Fu;
        x = (x | (x << 2)) & 0x33333333u;
        x = (x | (x << 1)) & 0x55555555u;
        return x;
    };
    for (int m = 1; m <= M; ++m) {
        float4* dst = out.data() + (size_t)m * (m - 1) / 2;
        pts.resize((size_t)m);
        order.resize((size_t)m);
        double c = 1.0, s = 0.0;
        for (int i = 0; i < m; ++i) {
            double z = 1.0 - (2.0 * (double)i + 1.0) / (double)m;
            double r2 = 1.0 - z * z;
            double r = r2 > 0.0 ? std::sqrt(r2) : 0.0;
            double x = r * c, y = r * s;
            pts[(size_t)i] = make_float4((float)x, (float)y, (float)z, 0.0f);
            // octahedral coordinates in [-1,1]^2 (any order would do: this one
            // only groups nearby directions)
            double l1 = std::fabs(x) + std::fabs(y) + std::fabs(z);
            double u = x / l1, v = y / l1;
            if (z < 0.0) {
                double uu = (1.0 - std::fabs(v)) * (u >= 0.0 ? 1.0 : -1.0);
                double vv = (1.0 - std::fabs(u)) * (v >= 0.0 ? 1.0 : -1.0);
                u = uu;
                v = vv;
            }
            uint32_t qu = (uint32_t)std::min(1023.0, std::max(0.0, (u + 1.0) * 512.0));
            uint32_t qv = (uint32_t)std::min(1023.0, std::max(0.0, (v + 1.0) * 512.0));
            order[(size_t)i] = {spread(qu) | (spread(qv) << 1), i};
            double cn = c * kGaCos - s * kGaSin;
            double sn = s * kGaCos + c * kGaSin;
            c = cn;
            s = sn;
        }
        std::sort(order.begin(), order.end());
        for (int k = 0; k < m; ++k) {
            const int i = order[(size_t)k].second;
            float4 q = pts[(size_t)i];
            std::memcpy(&q.w, &i, sizeof(int));
            dst[k] = q;
        }
    }
}

const uint64_t kMhSalt = 0x4D4554524Full;      // 'METRO': Metropolis counters
const uint64_t kMhInitSalt = 0x494E4954ull;    // 'INIT': first chain states
const uint64_t kDynSalt = 0x44594E414Dull;     // 'DYNAM': the dynamic chains

// Host tables of the Metropolis sampler.  nq[i] = Phi^-1((i + 0.5) / 4096) by
// Newton's method on Phi(x) = erfc(-x / sqrt 2) / 2 from x = 0 (monotone:
// Phi is convex left of 0 and concave right of it), FP64, rounded to FP32;
// ex[k] = exp(k / 1023) rounded to FP32.
void mh_tables(std::vector<float>& out)
{
    out.assign(kMhNq + kMhEx, 0.0f);
    const double rs2 = 0.70710678118654752440, rs2pi = 0.39894228040143267794;
    for (int i = 0; i < kMhNq; ++i) {
        const double p = ((double)i + 0.5) / (double)kMhNq;
        double x = 0.0;
        for (int it = 0; it < 200; ++it) {
            const double dx = (0.5 * std::erfc(-x * rs2) - p) / (rs2pi * std::exp(-0.5 * x * x));
            x -= dx;
            if (std::fabs(dx) <= 2e-16 * std::max(1.0, std::fabs(x))) break;
        }
        out[(size_t)i] = (float)x;
    }
    for (int k = 0; k < kMhEx; ++k) out[(size_t)kMhNq + k] = (float)std::exp((double)k / 1023.0);
}

uint64_t h3(uint64_t a, uint64_t b, uint64_t c) { return splitmix(splitmix(splitmix(a) ^ b) ^ c); }

void frame_rotation(uint64_t seed, uint64_t frame, float R[9])
{
    const double k53 = 1.1102230246251565e-16;
    double q[4] = {1.0, 0.0, 0.0, 0.0};
    for (uint64_t att = 0; att < 1000; ++att) {
        double c[4];
        for (int k = 0; k < 4; ++k) c[k] = ((double)(h3(seed ^ 0x524F54ull, frame, att * 4u + k) >> 11) * k53) * 2.0 - 1.0;
        double n2 = ((c[0] * c[0] + c[1] * c[1]) + c[2] * c[2]) + c[3] * c[3];
        if (n2 > 1e-6 && n2 <= 1.0) {
            double nn = std::sqrt(n2);
            for (int k = 0; k < 4; ++k) q[k] = c[k] / nn;
            break;
        }
    }
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double m[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z),       2.0 * (x * z + w * y),
                   2.0 * (x * y + w * z),       1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
                   2.0 * (x * z - w * y),       2.0 * (y * z + w * x),       1.0 - 2.0 * (x * x + y * y)};
    for (int k = 0; k < 9; ++k) R[k] = (float)m[k];
}

// Fault injection for the failure paths (adgi_inject_alloc_failure): when
// armed with n > 0, the n-th volume allocation from now on reports
// cudaErrorMemoryAllocation without calling cudaMalloc, once.
std::atomic<long> g_fail_alloc_in{0};

template <typename T>
cudaError_t dalloc(T** p, size_t count, size_t* total)
{
    if (g_fail_alloc_in.load() > 0 && g_fail_alloc_in.fetch_sub(1) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    size_t sz = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = cudaMalloc((void**)p, sz);
    if (e == cudaSuccess) *total += sz;
    return e;
}

}  // namespace

// error reporting for the allocation-free entry point (noalloc.cu)
const char* adgi::noalloc_fail(const std::string& msg)
{
    g_err = msg;
    return g_err.c_str();
}

struct adgi_volume_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    adgi_volume_desc desc{};
    VolConst V{};
    double s = 0.0;
    size_t bytes = 0;
    // tables
    float4* sf = nullptr;
    void* plan = nullptr;  // per-frame blend plan (BlendPlan)
    uint16_t* tex_src = nullptr;  // per texel: itself, or a border texel's octahedral fold partner
    float* ctab = nullptr;        // values of the packed atlas codes
    uint16_t* lut_v = nullptr;
    uint16_t* lut_c = nullptr;
    // atlases
    void* irr = nullptr;
    void* dep = nullptr;
    uint8_t* dep_n = nullptr;
    // heuristic state
    uint16_t *qv = nullptr, *qr = nullptr, *qv_even = nullptr, *qr_even = nullptr;
    uint16_t *amp_v = nullptr, *amp_r = nullptr, *trv = nullptr, *trr = nullptr;
    uint8_t *age_v = nullptr, *age_r = nullptr;
    uint32_t* G = nullptr;
    uint32_t *W = nullptr, *n = nullptr, *off = nullptr;
    // rays
    int2* pil_hit = nullptr;
    float4* pil_rec = nullptr;
    float* pil_lum = nullptr;
    uint32_t R_main = 0;
    int2* m_hit = nullptr;
    float4* m_rec = nullptr;
    unsigned long long* shadow_ctr = nullptr;
    int* err = nullptr;  // device anomaly flags
    FrameDev* fdev = nullptr;  // per-frame descriptor read by the kernels
    Tuning tune;               // block shapes (autotuner)
    // captured graph of the update (adgi_update_graph)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t gset = nullptr;
    bool graph_ok = false;
    cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
    // shading wavefront
    unsigned long long* vis = nullptr;
    uint4* jobs = nullptr;
    uint8_t* job_light = nullptr;
    unsigned* job_count = nullptr;
    size_t job_cap = 0;
    unsigned shadow_blocks = 0;
    // scene
    float* verts = nullptr;
    int* idx = nullptr;
    float* albedo = nullptr;
    int nv = 0, nt = 0;
    bool has_scene = false;
    float eps = 0.f;
    // two-part scene: triangles that touch a moved vertex form the moving part
    Bvh sbvh, dbvh;               // static part (PLOC, built once) and moving part (linear, per move)
    float4* w4 = nullptr;         // the static part's 4-wide tree (7 float4 a node), null: binary traversal
    int w4_nodes = 0, w4_depth = 0;
    size_t w4_bytes = 0;
    float4* tri_orig = nullptr;   // [3*nt] vertices in original order (shading normals)
    uint8_t* vmoved = nullptr;    // [nv] 1: vertex has been moved
    int* slist = nullptr;         // static triangles
    int* dlist = nullptr;         // moving triangles
    int ns = 0, nd = 0;
    size_t scene_cap_v = 0, scene_cap_t = 0;
    std::vector<std::pair<int, int>> moved;  // union of moved vertex ranges [a, b)
    bool split_dirty = false;     // the moved set grew: split and rebuild the static part
    bool dyn_dirty = false;       // moving vertices changed: rebuild the moving part
    // frame bookkeeping
    int64_t last_even = -2;
    uint64_t frames = 0;
    // a split update in progress (adgi_update_slab): its frame, step and probes
    FrameDev slab_fd;
    uint64_t slab_frame = 0;
    int slab_step = -1, slab_p0 = 0, slab_p1 = 0;
    float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ph[9] = {};  // phase boundaries of the last timed update
    cudaEvent_t shq[4] = {};  // around the shadow-ray kernel: pilot, adaptive
    cudaStream_t side = nullptr;  // the blend plan runs here, beside the traces
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t plq[2] = {};  // around the blend plan (timing)
    bool timed_pending = false;
    // query scratch for host pointers
    float* q_buf = nullptr;
    int q_cap = 0;
    // Metropolis sampler (desc.sampler = 1)
    uint32_t mh_B = 0, mh_C = 0;       // samples and chains per update
    float* mh_tab = nullptr;           // [4096] normal quantiles, then [1024] exp values
    float4* mh_chain = nullptr;        // [2C] chain states
    float4* mh_smp = nullptr;          // [B] samples, chain order
    float4* mh_smp_g = nullptr;        // [B] samples, grouped order
    uint64_t* mh_keys = nullptr;       // [2B] radix sort by probe
    uint32_t* mh_vals = nullptr;       // [2B]
    uint32_t* mh_hist = nullptr;       // radix histograms, then [1024] partial sums
    uint32_t* mh_off = nullptr;        // [P+1]
    int2* mh_hitn = nullptr;           // [B] -w hits, grouped order
    const uint32_t* mh_ord = nullptr;  // grouped order of the last update
    bool mh_live = false;              // chain states initialised
    uint32_t* qd = nullptr;            // [P][8] q_d of the last update
    uint8_t* cls = nullptr;            // [P] clip volume of the last update
    uint8_t* vout_even = nullptr;      // [P] in V_out on the last first-of-pair frame
    uint32_t* dyn_npin = nullptr;      // [Pp] probes of each proxy inside V_in
    // dynamic chains over virtual proxies (desc.dyn_ratio > 0)
    uint32_t dyn_Cd = 0, dyn_Bd = 0, dyn_Rd = 0;
    int dyn_dp[3] = {0, 0, 0}, dyn_pp = 0;
    float4* mh_smp_gn = nullptr;       // [B] -w ray directions, grouped order
    float4* dyn_chain = nullptr;       // [2Cd]
    float4* dyn_smp = nullptr;         // [Bd]
    int* dyn_cell = nullptr;           // [Bd]
    uint32_t* dyn_val = nullptr;       // [Pp*8]
    uint32_t* dyn_first = nullptr;     // [Pp*8]
    uint64_t* dyn_keys = nullptr;      // [2][Pp*8]
    uint32_t* dyn_vals = nullptr;      // [2][Pp*8]
    uint32_t* dyn_hist = nullptr;
    uint8_t* dyn_incl = nullptr;       // [Pp*8]
    uint32_t* dyn_off = nullptr;       // [P+1]
    uint32_t* dyn_part = nullptr;      // [1024]
    uint32_t* dyn_info = nullptr;      // [2]
    int* dyn_tab = nullptr;            // [8] texels per octant, then [8][n_irr^2] their tile indices
    float4* dyn_tex_dir = nullptr;     // [8][n_irr^2]
    int2* dyn_hit = nullptr;           // [Rd]
    float4* dyn_rec = nullptr;         // [Rd]
    bool dyn_live = false;
};

namespace {

void free_volume(adgi_volume v)
{
    if (!v) return;
    void* ptrs[] = {v->sf,      v->plan,    v->tex_src, v->ctab,    v->lut_v,   v->lut_c,  v->irr,   v->dep,     v->dep_n,   v->qv,     v->qr,
                    v->qv_even, v->qr_even, v->amp_v,  v->amp_r, v->trv,     v->trr,     v->age_v,  v->age_r,
                    v->G,       v->W,       v->n,      v->off,   v->pil_hit, v->pil_rec, v->pil_lum, v->m_hit,
                    v->m_rec,   v->shadow_ctr, v->verts, v->idx, v->albedo,  v->q_buf, v->err,
                    v->vis,     v->jobs,    v->job_light, v->job_count, v->fdev,
                    v->qd, v->cls, v->vout_even, v->dyn_npin, v->mh_smp_gn, v->dyn_chain, v->dyn_smp, v->dyn_cell, v->dyn_val, v->dyn_first, v->dyn_keys,
                    v->dyn_vals, v->dyn_hist, v->dyn_incl, v->dyn_off, v->dyn_part, v->dyn_info, v->dyn_tab,
                    v->dyn_tex_dir, v->dyn_hit, v->dyn_rec,
                    v->mh_tab,  v->mh_chain, v->mh_smp, v->mh_smp_g, v->mh_keys, v->mh_vals, v->mh_hist, v->mh_off, v->mh_hitn};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    v->sbvh.release();
    v->dbvh.release();
    cudaFree(v->w4);
    cudaFree(v->tri_orig);
    cudaFree(v->vmoved);
    cudaFree(v->slist);
    cudaFree(v->dlist);
    if (v->ev0) cudaEventDestroy(v->ev0);
    if (v->ev1) cudaEventDestroy(v->ev1);
    for (cudaEvent_t e : v->ph)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : v->shq)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : v->plq)
        if (e) cudaEventDestroy(e);

    if (v->fork) cudaEventDestroy(v->fork);
    if (v->join) cudaEventDestroy(v->join);
    if (v->side) cudaStreamDestroy(v->side);
    if (v->gexec) cudaGraphExecDestroy(v->gexec);
    if (v->graph) cudaGraphDestroy(v->graph);
    if (v->cap_stream) cudaStreamDestroy(v->cap_stream);
    delete v;
}

int validate_desc(const adgi_volume_desc* d)
{
    if (!d) return fail(ADGI_ERR_INVALID_ARG, "desc is NULL");
    for (int k = 0; k < 3; ++k) {
        if (d->dims[k] < 2) return fail(ADGI_ERR_INVALID_ARG, "dims must be >= 2");
        if (!(d->spacing[k] > 0.0f) || !std::isfinite(d->spacing[k]))
            return fail(ADGI_ERR_INVALID_ARG, "spacing must be positive");
        if (!std::isfinite(d->origin[k])) return fail(ADGI_ERR_INVALID_ARG, "origin must be finite");
    }
    if ((int64_t)d->dims[0] * d->dims[1] * d->dims[2] > (1 << 26))
        return fail(ADGI_ERR_INVALID_ARG, "too many probes");
    if (d->irr_interior < 1 || d->irr_interior > 30 || d->depth_interior < 1 || d->depth_interior > 30)
        return fail(ADGI_ERR_INVALID_ARG, "tile interior must be in [1, 30]");
    int m0 = d->rays_min > 8 ? d->rays_min : 8;
    if (d->rays_max > 4096 || d->rays_avg < m0 || d->rays_avg > d->rays_max)
        return fail(ADGI_ERR_INVALID_ARG, "need max(rays_min, 8) <= rays_avg <= rays_max <= 4096");
    if (!(d->hysteresis >= 0.0f && d->hysteresis < 1.0f)) return fail(ADGI_ERR_INVALID_ARG, "hysteresis in [0,1)");
    if (d->tr_theta < 1 || d->tr_theta > 255) return fail(ADGI_ERR_INVALID_ARG, "tr_theta in [1,255]");
    if (d->atlas_fp16 < 0 || d->atlas_fp16 > 3) return fail(ADGI_ERR_INVALID_ARG, "atlas_fp16 in {0,1,2,3}");
    if (d->sampler < 0 || d->sampler > 1) return fail(ADGI_ERR_INVALID_ARG, "sampler in {0,1}");
    if (d->sampler == 1 && d->atlas_fp16 == 3)
        return fail(ADGI_ERR_INVALID_ARG, "the Metropolis sampler blends batched moving averages: not with packed atlases");
    if (d->sampler == 1 && !(d->alpha >= 0.0f && std::isfinite(d->alpha)))
        return fail(ADGI_ERR_INVALID_ARG, "alpha must be finite and >= 0");
    if (d->dyn_ratio < 0 || d->dyn_ratio > 1024 || (d->dyn_ratio > 0 && d->sampler != 1))
        return fail(ADGI_ERR_INVALID_ARG, "dyn_ratio in [0, 1024], and > 0 only with sampler = 1");
    if (d->dyn_ratio > 0 && !(d->hysteresis_dyn >= 0.0f && d->hysteresis_dyn < 1.0f))
        return fail(ADGI_ERR_INVALID_ARG, "hysteresis_dyn in [0,1)");
    if (d->blend_mode < 0 || d->blend_mode > 1 || (d->blend_mode == 1 && (d->sampler != 0 || d->atlas_fp16 == 3)))
        return fail(ADGI_ERR_INVALID_ARG, "blend_mode in {0,1}; the cosine gather needs sampler 0 and atlas_fp16 < 3");
    if (!(d->cheb_var_floor_rel >= 0.0f && d->cheb_var_floor_rel < 1.0f))
        return fail(ADGI_ERR_INVALID_ARG, "cheb_var_floor_rel in [0,1)");
    int64_t P = (int64_t)d->dims[0] * d->dims[1] * d->dims[2];
    if (P * (int64_t)d->rays_avg >= (int64_t)1 << 31) return fail(ADGI_ERR_INVALID_ARG, "ray budget too large");
    return ADGI_OK;
}

FrameConst frame_const(adgi_volume v, const adgi_frame* f)
{
    FrameConst F{};
    F.pilot_key = splitmix(splitmix(f->seed) ^ (f->frame >> 1));
    frame_rotation(f->seed, f->frame, v->R);
    for (int k = 0; k < 9; ++k) F.R[k] = v->R[k];
    for (int k = 0; k < 3; ++k) F.sky[k] = f->sky_rgb[k];
    F.n_lights = f->n_lights;
    F.even = (f->frame & 1u) == 0;
    F.pair_valid = !F.even && v->last_even == (int64_t)f->frame - 1;
    F.has_camera = f->has_camera ? 1 : 0;
    for (int k = 0; k < 3; ++k) F.cam[k] = f->cam_pos[k];
    F.cam_k = f->cam_k;
    F.mh_key = splitmix(splitmix(f->seed ^ kMhSalt) ^ f->frame);
    F.dyn_key = splitmix(splitmix(f->seed ^ kDynSalt) ^ f->frame);
    F.has_clip = f->has_clip && f->has_camera ? 1 : 0;
    for (int k = 0; k < 16; ++k) F.clip[k] = f->view_proj[k];
    return F;
}

}  // namespace

extern "C" {

namespace {
DynBufs dyn_bufs(adgi_volume v);
}

const char* adgi_last_error(void) { return g_err.c_str(); }

int adgi_inject_alloc_failure(int32_t n)
{
    if (n < 0) return fail(ADGI_ERR_INVALID_ARG, "adgi_inject_alloc_failure: n < 0");
    g_fail_alloc_in.store(n);
    return ADGI_OK;
}

int adgi_create_volume(const adgi_volume_desc* desc, void* cuda_stream, adgi_volume* out)
{
    if (!out) return fail(ADGI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate_desc(desc);
    if (rc) return rc;
    adgi_volume v = new adgi_volume_s();
    v->desc = *desc;
    v->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&v->device);
    const adgi_volume_desc& d = *desc;
    VolConst& V = v->V;
    for (int k = 0; k < 3; ++k) {
        V.origin[k] = d.origin[k];
        V.spacing[k] = d.spacing[k];
        V.dims[k] = d.dims[k];
    }
    V.P = d.dims[0] * d.dims[1] * d.dims[2];
    V.n_irr = d.irr_interior;
    V.n_dep = d.depth_interior;
    V.Ti = d.irr_interior + 2;
    V.Td = d.depth_interior + 2;
    double sx = d.spacing[0], sy = d.spacing[1], sz = d.spacing[2];
    v->s = std::sqrt((sx * sx + sy * sy) + sz * sz);
    V.tmin = (float)(1e-4 * v->s);
    V.depth_max = d.depth_max > 0.0f ? d.depth_max : (float)(1.5 * v->s);
    V.qv_scale = (float)(256.0 / v->s);
    V.qc_scale = (float)(64.0 / v->s);
    V.var_min = (float)(1e-6 * v->s * v->s);
    V.var_rel = d.cheb_var_floor_rel;
    V.hyst = d.hysteresis;
    V.theta = d.tr_theta;
    V.m0 = d.rays_min > 8 ? d.rays_min : 8;
    V.rays_max = d.rays_max;
    V.rays_avg = d.rays_avg;
    V.fp16 = d.atlas_fp16;
    const size_t P = (size_t)V.P;
    v->R_main = (uint32_t)((size_t)(d.rays_avg - 8) * P);
    size_t& B = v->bytes;
    cudaError_t e = cudaSuccess;
#define DA(ptr, count)                                      \
    do {                                                    \
        e = dalloc(&(ptr), (count), &B);                    \
        if (e != cudaSuccess) {                             \
            free_volume(v);                                 \
            return fail(ADGI_ERR_OOM, "device allocation"); \
        }                                                   \
    } while (0)
    // tables
    int M = d.rays_max - 8;
    std::vector<float4> sf;
    build_sf(M > 0 ? M : 0, sf);
    DA(v->sf, sf.size());
    {
        uint8_t* pb;
        DA(pb, blend_plan_bytes(M > 0 ? M : 0, V.Ti, V.Td));
        v->plan = pb;
    }
    DA(v->tex_src, (size_t)V.Ti * V.Ti + (size_t)V.Td * V.Td);
    // packed atlas codes (the paper's codecs): code k of a b-bit channel with
    // parameters (beta, gamma) stands for (exp(beta k / (2^b - 1)) - 1) / gamma,
    // computed in FP64 and rounded to FP32: 9-bit and 8-bit irradiance (5, 15),
    // 13-bit mean distance (5, 15) and mean squared distance (8, 20)
    std::vector<float> ctab;
    for (auto cf : {std::make_tuple(9, 5.0, 15.0), std::make_tuple(8, 5.0, 15.0), std::make_tuple(13, 5.0, 15.0),
                    std::make_tuple(13, 8.0, 20.0)}) {
        const int bits = std::get<0>(cf);
        const double beta = std::get<1>(cf), gamma = std::get<2>(cf), kmax = (double)((1 << bits) - 1);
        for (int k = 0; k < (1 << bits); ++k) ctab.push_back((float)((std::exp(beta * (double)k / kmax) - 1.0) / gamma));
    }
    DA(v->ctab, ctab.size());
    V.ctab = v->ctab;
    V.s_f = (float)v->s;
    std::vector<uint16_t> tsrc;
    for (int n : {V.n_irr, V.n_dep}) {  // octahedral border fold of a tile with n x n interior
        const int T = n + 2;
        for (int i = 0; i < T; ++i)
            for (int j = 0; j < T; ++j) {
                int si = i, sj = j;
                const bool top = i == 0, bot = i == n + 1, lef = j == 0, rig = j == n + 1;
                if ((top || bot) && (lef || rig)) {  // corners: the diagonally opposite interior corner
                    si = top ? n : 1;
                    sj = lef ? n : 1;
                } else if (top || bot) {
                    si = top ? 1 : n;
                    sj = n + 1 - j;
                } else if (lef || rig) {
                    si = n + 1 - i;
                    sj = lef ? 1 : n;
                }
                tsrc.push_back((uint16_t)(si * T + sj));
            }
    }
    DA(v->lut_v, 4096);
    DA(v->lut_c, 4096);
    std::vector<uint16_t> lv(4096), lc(4096);
    for (int i = 0; i < 4096; ++i) {
        lv[i] = (uint16_t)std::floor(1023.0 * std::exp(-2.0 * ((double)i + 0.5) / 256.0));
        lc[i] = (uint16_t)std::floor(1023.0 * std::exp(-((double)i + 0.5) * v->s / 64.0));
    }
    // atlases
    size_t ti2 = (size_t)V.Ti * V.Ti, td2 = (size_t)V.Td * V.Td;
    size_t irr_bytes = P * ti2 * (V.fp16 == 3 ? 4 : V.fp16 ? 8 : 16), dep_bytes = P * td2 * (V.fp16 ? 4 : 8);
    {
        uint8_t* a;
        DA(a, irr_bytes);
        v->irr = a;
        DA(a, dep_bytes);
        v->dep = a;
    }
    DA(v->dep_n, P * td2);
    DA(v->qv, P * 8);
    DA(v->qr, P * 8);
    DA(v->qv_even, P * 8);
    DA(v->qr_even, P * 8);
    DA(v->amp_v, P * 8);
    DA(v->amp_r, P * 8);
    DA(v->trv, P * 8);
    DA(v->trr, P * 8);
    DA(v->age_v, P * 8);
    DA(v->age_r, P * 8);
    DA(v->G, P * 8);
    DA(v->W, P);
    DA(v->n, P);
    DA(v->off, P + 1);
    DA(v->pil_hit, P * 8);
    DA(v->pil_rec, P * 8);
    DA(v->pil_lum, P * 8);
    DA(v->m_hit, (size_t)v->R_main);
    DA(v->m_rec, (size_t)v->R_main);
    DA(v->shadow_ctr, 1);
    DA(v->err, 1);
    DA(v->fdev, 1);
    DA(v->vis, std::max<size_t>(P * 8, (size_t)v->R_main));
    DA(v->job_count, 4);  // the shadow-job count and the work counters of the shadow and trace kernels
    DA(v->qd, P * 8);
    DA(v->cls, P);
    DA(v->vout_even, P);
    if (d.sampler == 1) {
        v->mh_B = v->R_main;
        if (d.dyn_ratio > 0) {  // budget split static:dynamic = r:1; a static sample traces two rays
            const uint64_t Bt = v->R_main, r = (uint64_t)d.dyn_ratio;
            v->mh_B = (uint32_t)(Bt * r / (r + 1));
            v->dyn_Rd = (uint32_t)(2 * (Bt - v->mh_B));
        }
        v->mh_C = (v->mh_B + kMhPer - 1) / kMhPer;
        const size_t nB = v->mh_B;
        DA(v->mh_tab, (size_t)(kMhNq + kMhEx));
        DA(v->mh_chain, 2 * (size_t)v->mh_C);
        DA(v->mh_smp, nB);
        DA(v->mh_smp_g, nB);
        DA(v->mh_keys, 2 * nB);
        DA(v->mh_vals, 2 * nB);
        DA(v->mh_hist, radix_hist_entries((int)nB) + 1024);
        DA(v->mh_off, P + 1);
        DA(v->mh_hitn, nB);
        if (d.dyn_ratio > 0) {
            const uint32_t r = (uint32_t)d.dyn_ratio;
            v->dyn_Cd = v->mh_C ? (v->mh_C + r - 1) / r : 0;
            v->dyn_Bd = v->dyn_Cd * kMhPer;
            for (int k = 0; k < 3; ++k) v->dyn_dp[k] = (d.dims[k] + 2) / 3;
            v->dyn_pp = v->dyn_dp[0] * v->dyn_dp[1] * v->dyn_dp[2];
            const size_t cells = (size_t)v->dyn_pp * 8, nn = (size_t)V.n_irr * V.n_irr;
            DA(v->mh_smp_gn, nB);
            DA(v->dyn_chain, 2 * (size_t)v->dyn_Cd);
            DA(v->dyn_smp, (size_t)v->dyn_Bd);
            DA(v->dyn_cell, (size_t)v->dyn_Bd);
            DA(v->dyn_val, cells);
            DA(v->dyn_npin, (size_t)v->dyn_pp);
            DA(v->dyn_first, cells);
            DA(v->dyn_keys, 2 * cells);
            DA(v->dyn_vals, 2 * cells);
            DA(v->dyn_hist, radix_hist_entries((int)cells));
            DA(v->dyn_incl, cells);
            DA(v->dyn_off, P + 1);
            DA(v->dyn_part, 1024);
            DA(v->dyn_info, 2);
            DA(v->dyn_tab, 8 + 8 * nn);
            DA(v->dyn_tex_dir, 8 * nn);
            DA(v->dyn_hit, (size_t)v->dyn_Rd);
            DA(v->dyn_rec, (size_t)v->dyn_Rd);
        }
    }
#undef DA
    V.R_main = v->R_main;
    V.err = v->err;
    V.dyn = d.dyn_ratio > 0 ? 1 : 0;
    V.hyst_dyn = d.hysteresis_dyn;
    V.cls = v->cls;
    V.p_lo = 0;
    V.p_hi = V.P;
    cudaStream_t s = v->stream;
#define CKV(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e__ = (call);                                                                        \
        if (e__ != cudaSuccess) {                                                                        \
            free_volume(v);                                                                              \
            return fail(ADGI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__));             \
        }                                                                                                \
    } while (0)
    CKV(cudaMemcpyAsync(v->sf, sf.data(), sizeof(float4) * sf.size(), cudaMemcpyHostToDevice, s));
    CKV(cudaMemcpyAsync(v->tex_src, tsrc.data(), sizeof(uint16_t) * tsrc.size(), cudaMemcpyHostToDevice, s));
    CKV(cudaMemcpyAsync(v->ctab, ctab.data(), sizeof(float) * ctab.size(), cudaMemcpyHostToDevice, s));
    CKV(cudaMemcpyAsync(v->lut_v, lv.data(), 2 * 4096, cudaMemcpyHostToDevice, s));
    CKV(cudaMemcpyAsync(v->lut_c, lc.data(), 2 * 4096, cudaMemcpyHostToDevice, s));
    CKV(cudaMemsetAsync(v->irr, 0, irr_bytes, s));
    CKV(cudaMemsetAsync(v->dep, 0, dep_bytes, s));
    CKV(cudaMemsetAsync(v->dep_n, 0, P * td2, s));
    for (uint16_t* p : {v->qv, v->qr, v->qv_even, v->qr_even, v->amp_v, v->amp_r, v->trv, v->trr})
        CKV(cudaMemsetAsync(p, 0, P * 8 * 2, s));
    CKV(cudaMemsetAsync(v->age_v, 0xFF, P * 8, s));
    CKV(cudaMemsetAsync(v->age_r, 0xFF, P * 8, s));
    CKV(cudaMemsetAsync(v->W, 0, P * 4, s));
    CKV(cudaMemsetAsync(v->shadow_ctr, 0, 8, s));
    CKV(cudaMemsetAsync(v->err, 0, 4, s));
    std::vector<float> mh_tab;
    if (d.sampler == 1) {
        mh_tables(mh_tab);
        CKV(cudaMemcpyAsync(v->mh_tab, mh_tab.data(), sizeof(float) * mh_tab.size(), cudaMemcpyHostToDevice, s));
        CKV(cudaMemsetAsync(v->mh_off, 0, 4 * (P + 1), s));
        v->mh_ord = v->mh_vals;
        if (V.dyn) {
            CKV(cudaMemsetAsync(v->dyn_off, 0, 4 * (P + 1), s));
            CKV(cudaMemsetAsync(v->dyn_incl, 0, (size_t)v->dyn_pp * 8, s));
            CKV(cudaMemsetAsync(v->dyn_info, 0, 8, s));
            CKV(launch_dyn_tables(V, dyn_bufs(v), s));
        }
    }
    CKV(cudaMemsetAsync(v->qd, 0, P * 8 * 4, s));
    CKV(cudaMemsetAsync(v->cls, 2, P, s));
    CKV(cudaMemsetAsync(v->vout_even, 0, P, s));
    v->shadow_blocks = shadow_grid_blocks(0);
    CKV(cudaEventCreate(&v->ev0));
    CKV(cudaEventCreate(&v->ev1));
    for (cudaEvent_t& e : v->ph) CKV(cudaEventCreate(&e));
    for (cudaEvent_t& e : v->shq) CKV(cudaEventCreate(&e));
    for (cudaEvent_t& e : v->plq) CKV(cudaEventCreate(&e));
    CKV(cudaEventCreateWithFlags(&v->fork, cudaEventDisableTiming));
    CKV(cudaEventCreateWithFlags(&v->join, cudaEventDisableTiming));
    CKV(cudaStreamCreateWithFlags(&v->side, cudaStreamNonBlocking));
    // the host vectors die at return: wait for the copies
    CKV(cudaStreamSynchronize(s));
#undef CKV
    *out = v;
    return ADGI_OK;
}

int adgi_destroy(adgi_volume v)
{
    if (!v) return ADGI_OK;
    cudaStreamSynchronize(v->stream);
    free_volume(v);
    return ADGI_OK;
}

int adgi_set_stream(adgi_volume v, void* cuda_stream)
{
    if (!v) return fail(ADGI_ERR_INVALID_ARG, "volume is NULL");
    v->stream = (cudaStream_t)cuda_stream;
    return ADGI_OK;
}

int adgi_enable_timing(adgi_volume v, int32_t enable)
{
    if (!v) return fail(ADGI_ERR_INVALID_ARG, "volume is NULL");
    v->timing = enable != 0;
    return ADGI_OK;
}

int adgi_set_scene(adgi_volume v, const float* verts, int32_t nv, const int32_t* idx, int32_t nt, const float* albedo,
                   int32_t on_device)
{
    if (!v) return fail(ADGI_ERR_INVALID_ARG, "volume is NULL");
    if (nv < 0 || nt < 0 || (nv > 0 && !verts) || (nt > 0 && (!idx || !albedo)))
        return fail(ADGI_ERR_INVALID_ARG, "bad scene arrays");
    cudaStream_t s = v->stream;
    std::vector<float> hv;
    std::vector<int> hi;
    std::vector<float> ha;
    const int* idx_host = nullptr;
    if (on_device) {
        hi.resize(3 * (size_t)nt);
        CK(cudaMemcpyAsync(hi.data(), idx, sizeof(int) * 3 * (size_t)nt, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        idx_host = hi.data();
    } else {
        idx_host = idx;
    }
    for (size_t k = 0; k < 3 * (size_t)nt; ++k)
        if (idx_host[k] < 0 || idx_host[k] >= nv) return fail(ADGI_ERR_INVALID_ARG, "triangle index out of range");
    // scene extent -> box enlargement
    if (on_device) {
        hv.resize(3 * (size_t)nv);
        CK(cudaMemcpyAsync(hv.data(), verts, sizeof(float) * 3 * (size_t)nv, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    const float* vh = on_device ? hv.data() : verts;
    double lo[3] = {1e300, 1e300, 1e300}, hi3[3] = {-1e300, -1e300, -1e300};
    for (size_t k = 0; k < (size_t)nv; ++k)
        for (int c = 0; c < 3; ++c) {
            double x = vh[3 * k + c];
            if (!std::isfinite(x)) return fail(ADGI_ERR_INVALID_ARG, "non-finite vertex");
            lo[c] = x < lo[c] ? x : lo[c];
            hi3[c] = x > hi3[c] ? x : hi3[c];
        }
    double ext = 0.0, mag = 0.0;
    for (int c = 0; c < 3 && nv > 0; ++c) {
        ext = std::fmax(ext, hi3[c] - lo[c]);
        mag = std::fmax(mag, std::fmax(std::fabs(lo[c]), std::fabs(hi3[c])));
    }
    v->eps = (float)(1e-5 * std::fmax(ext, mag) + 1e-30);
    if ((size_t)nv > v->scene_cap_v || (size_t)nt > v->scene_cap_t || !v->verts) {
        for (void* p : {(void*)v->verts, (void*)v->idx, (void*)v->albedo, (void*)v->tri_orig, (void*)v->vmoved,
                        (void*)v->slist, (void*)v->dlist})
            cudaFree(p);
        v->verts = nullptr;
        v->idx = nullptr;
        v->albedo = nullptr;
        v->tri_orig = nullptr;
        v->vmoved = nullptr;
        v->slist = nullptr;
        v->dlist = nullptr;
        size_t dummy = 0;
        if (dalloc(&v->verts, 3 * (size_t)nv, &dummy) != cudaSuccess || dalloc(&v->idx, 3 * (size_t)nt, &dummy) != cudaSuccess ||
            dalloc(&v->albedo, 3 * (size_t)nt, &dummy) != cudaSuccess ||
            dalloc(&v->tri_orig, 3 * (size_t)nt, &dummy) != cudaSuccess ||
            dalloc(&v->vmoved, (size_t)nv, &dummy) != cudaSuccess || dalloc(&v->slist, (size_t)nt, &dummy) != cudaSuccess ||
            dalloc(&v->dlist, (size_t)nt, &dummy) != cudaSuccess)
            return fail(ADGI_ERR_OOM, "scene allocation");
        v->scene_cap_v = (size_t)nv;
        v->scene_cap_t = (size_t)nt;
    }
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nv) CK(cudaMemcpyAsync(v->verts, verts, sizeof(float) * 3 * (size_t)nv, k, s));
    if (nt) {
        CK(cudaMemcpyAsync(v->idx, idx, sizeof(int) * 3 * (size_t)nt, k, s));
        CK(cudaMemcpyAsync(v->albedo, albedo, sizeof(float) * 3 * (size_t)nt, k, s));
    }
    if (nv) CK(cudaMemsetAsync(v->vmoved, 0, (size_t)nv, s));
    v->nv = nv;
    v->nt = nt;
    if (!on_device) CK(cudaStreamSynchronize(s));  // pageable sources are read before return anyway
    // every triangle is static until some of its vertices move
    v->moved.clear();
    v->ns = nt;
    v->nd = 0;
    v->dbvh.n_tris = 0;
    CK(fill_tri_orig(v->verts, v->idx, nullptr, nv, nt, v->tri_orig, s));
    CK(v->sbvh.build(v->verts, v->idx, nv, nt, v->eps, v->err, s, nullptr, true));
    v->has_scene = true;
    v->split_dirty = false;
    v->dyn_dirty = false;
    v->graph_ok = false;
    return ADGI_OK;
}

int adgi_move_vertices(adgi_volume v, int32_t first, int32_t count, const float* verts, int32_t on_device)
{
    if (!v) return fail(ADGI_ERR_INVALID_ARG, "volume is NULL");
    if (!v->has_scene) return fail(ADGI_ERR_NO_SCENE, "no scene");
    if (first < 0 || count < 0 || first + count > v->nv || (count > 0 && !verts))
        return fail(ADGI_ERR_INVALID_ARG, "vertex range outside the scene");
    if (count == 0) return ADGI_OK;
    CK(cudaMemcpyAsync(v->verts + 3 * (size_t)first, verts, sizeof(float) * 3 * (size_t)count,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, v->stream));
    // a range not yet known to move makes its triangles part of the moving set
    bool covered = false;
    for (auto& r : v->moved)
        if (r.first <= first && first + count <= r.second) covered = true;
    if (!covered) {
        v->moved.push_back({first, first + count});
        std::sort(v->moved.begin(), v->moved.end());
        std::vector<std::pair<int, int>> merged;
        for (auto& r : v->moved) {
            if (!merged.empty() && r.first <= merged.back().second)
                merged.back().second = std::max(merged.back().second, r.second);
            else
                merged.push_back(r);
        }
        v->moved.swap(merged);
        CK(cudaMemsetAsync(v->vmoved + first, 1, (size_t)count, v->stream));
        v->split_dirty = true;
    }
    v->dyn_dirty = true;
    return ADGI_OK;
}

namespace {
// Where the moving part lives in the static part's arrays (which hold room
// for every triangle): its nodes from node max(ns-1, 0), its triangles from
// slot ns.
int moving_node_off(adgi_volume v) { return v->ns > 1 ? v->ns - 1 : 0; }
int moving_tri_off(adgi_volume v) { return v->ns; }

// Rebuild the moving part's linear BVH after the static part's nodes and
// triangles, and relocate its references to those global indices.
int build_moving(adgi_volume v, cudaStream_t s)
{
    const int no = moving_node_off(v), to = moving_tri_off(v);
    CK(v->dbvh.build(v->verts, v->idx, v->nv, v->nd, v->eps, v->err, s, v->dlist, false,
                     v->sbvh.tri_v + 3 * (size_t)to, v->sbvh.nodes + no));
    if (v->nd > 1) CK(relocate_nodes(v->sbvh.nodes + no, v->nd - 1, no, to, s));
    return ADGI_OK;
}

// The static part's 4-wide tree, collapsed on the host from its binary tree
// (once per static build; collapse_wide4).  Left out, so that the binary
// tree is traversed, when the static part has fewer than two triangles or the
// tree is deeper than the traversal stack allows (3 entries a level).
int build_wide(adgi_volume v, cudaStream_t s)
{
    if (v->w4) {
        cudaFree(v->w4);
        v->bytes -= v->w4_bytes;
    }
    v->w4 = nullptr;
    v->w4_nodes = v->w4_depth = 0;
    v->w4_bytes = 0;
    if (v->ns < 2) return ADGI_OK;
    std::vector<BNode> bn((size_t)v->ns - 1);
    CK(cudaMemcpyAsync(bn.data(), v->sbvh.nodes, sizeof(BNode) * bn.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<float4> w;
    int depth = 0;
    const int nw = collapse_wide4(bn.data(), (int)bn.size(), w, &depth);
    if (nw < 0) return fail(ADGI_ERR_CUDA, "4-wide collapse: malformed binary tree");
    if (3 * depth > kWide4Stack) return ADGI_OK;
    size_t b = 0;
    if (dalloc(&v->w4, w.size(), &b) != cudaSuccess) {
        v->w4 = nullptr;
        return fail(ADGI_ERR_OOM, "4-wide tree");
    }
    CK(cudaMemcpyAsync(v->w4, w.data(), sizeof(float4) * w.size(), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // w is freed on return
    v->bytes += b;
    v->w4_bytes = b;
    v->w4_nodes = nw;
    v->w4_depth = depth;
    return ADGI_OK;
}

// Bring both BVH parts up to date: re-split and rebuild the static part when
// the moving set grew, rebuild the moving part when its vertices moved.
int ensure_bvh(adgi_volume v, cudaStream_t s, bool moving_too = true)
{
    if (v->split_dirty) {
        CK(v->sbvh.reserve(v->nt, true));
        if (!v->sbvh.pscratch) return fail(ADGI_ERR_OOM, "split scratch");
        CK(split_static_moving(v->idx, v->vmoved, v->nt, v->nv, v->sbvh.pbufs, v->slist, v->dlist, &v->ns, &v->nd, s));
        CK(v->sbvh.build(v->verts, v->idx, v->nv, v->ns, v->eps, v->err, s, v->slist, true));
        {
            int rc = build_wide(v, s);
            if (rc) return rc;
        }
        v->split_dirty = false;
        v->dyn_dirty = true;
    }
    if (v->dyn_dirty && moving_too) {
        CK(fill_tri_orig(v->verts, v->idx, v->dlist, v->nv, v->nd, v->tri_orig, s));
        {
            int rc = build_moving(v, s);
            if (rc) return rc;
        }
        v->dyn_dirty = false;
    }
    return ADGI_OK;
}

MhBufs mh_bufs(adgi_volume v)
{
    MhBufs M{};
    M.n_samples = v->mh_B;
    M.n_chains = v->mh_C;
    M.alpha = v->desc.alpha;
    M.inv_q2 = 1.0f / 1046529.0f;
    M.nq = v->mh_tab;
    M.ex = v->mh_tab ? v->mh_tab + kMhNq : nullptr;
    M.chain = v->mh_chain;
    M.smp = v->mh_smp;
    M.smp_g = v->mh_smp_g;
    M.keys[0] = v->mh_keys;
    M.keys[1] = v->mh_keys ? v->mh_keys + v->mh_B : nullptr;
    M.vals[0] = v->mh_vals;
    M.vals[1] = v->mh_vals ? v->mh_vals + v->mh_B : nullptr;
    M.hist = v->mh_hist;
    M.part = v->mh_hist + radix_hist_entries((int)v->mh_B);
    M.off = v->mh_off;
    M.lut_c = v->lut_c;
    M.qv = v->qv;
    M.irr = v->irr;
    M.qd = v->V.dyn ? v->qd : nullptr;
    M.smp_gn = v->V.dyn ? v->mh_smp_gn : nullptr;
    return M;
}

DynBufs dyn_bufs(adgi_volume v)
{
    DynBufs D{};
    D.n_chains = v->dyn_Cd;
    D.n_samples = v->dyn_Bd;
    D.budget = v->dyn_Rd;
    for (int k = 0; k < 3; ++k) D.dp[k] = v->dyn_dp[k];
    D.pp = v->dyn_pp;
    D.nq = v->mh_tab;
    D.qd = v->qd;
    D.chain = v->dyn_chain;
    D.smp = v->dyn_smp;
    D.cell = v->dyn_cell;
    D.val = v->dyn_val;
    D.npin = v->dyn_npin;
    D.first = v->dyn_first;
    const size_t cells = (size_t)v->dyn_pp * 8;
    D.keys[0] = v->dyn_keys;
    D.keys[1] = v->dyn_keys ? v->dyn_keys + cells : nullptr;
    D.vals[0] = v->dyn_vals;
    D.vals[1] = v->dyn_vals ? v->dyn_vals + cells : nullptr;
    D.hist = v->dyn_hist;
    D.incl = v->dyn_incl;
    D.off = v->dyn_off;
    D.part = v->dyn_part;
    D.info = v->dyn_info;
    D.ntex = v->dyn_tab;
    D.tex_t = v->dyn_tab ? v->dyn_tab + 8 : nullptr;
    D.tex_dir = v->dyn_tex_dir;
    return D;
}

SceneDev scene_view(adgi_volume v)
{
    SceneDev S;
    S.w4 = v->w4;
    S.nodes = v->sbvh.nodes;
    S.tri_v = v->sbvh.tri_v;
    S.root[0] = v->ns > 1 ? 0 : -1;
    S.leaf[0] = v->ns == 1 ? 0 : -1;
    S.root[1] = v->nd > 1 ? moving_node_off(v) : -1;
    S.leaf[1] = v->nd == 1 ? moving_tri_off(v) : -1;
    S.max_iter = 2 * (v->ns + v->nd) + 32;
    S.n_tris = v->nt;
    S.n_verts = v->nv;
    S.tri_orig = v->tri_orig;
    S.albedo = v->albedo;
    S.err = v->err;
    return S;
}
}  // namespace

namespace {

// Host side of an update: validate, bring the BVH parts up to date (may
// synchronise: never inside a capture), build the frame descriptor, and make
// room for the shadow jobs.  Sets *graph_stale when a captured graph of this
// volume can no longer be replayed.
int prepare_update(adgi_volume v, const adgi_frame* f, FrameDev& fd, bool* graph_stale)
{
    if (!v || !f) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if (!v->has_scene) return fail(ADGI_ERR_NO_SCENE, "no scene");
    if (f->n_lights < 0 || f->n_lights > kMaxLights || (f->n_lights > 0 && !f->lights))
        return fail(ADGI_ERR_INVALID_ARG, "bad light list");
    cudaStream_t s = v->stream;
    const VolConst& V = v->V;
    bool stale = false;
    if (v->split_dirty) stale = true;
    {
        int rc = ensure_bvh(v, s, false);  // the moving part is rebuilt inside the update itself
        if (rc) return rc;
    }
    if (v->nd > 0) CK(v->dbvh.reserve(v->nd, false));  // no allocation inside a captured update
    const unsigned sb = shadow_grid_blocks(v->tune.shadow_mult);
    if (sb != v->shadow_blocks) {
        v->shadow_blocks = sb;
        stale = true;
    }
    fd.F = frame_const(v, f);
    fd.L.n = f->n_lights;
    for (int i = 0; i < f->n_lights; ++i) {
        fd.L.l[i].kind = f->lights[i].kind;
        for (int k = 0; k < 3; ++k) {
            fd.L.l[i].v[k] = f->lights[i].pos_or_dir[k];
            fd.L.l[i].rgb[k] = f->lights[i].rgb[k];
        }
    }
    // shadow-job capacity: one job per lit light of every ray of the larger set
    size_t need = (size_t)f->n_lights * std::max<size_t>((size_t)V.P * kPilots, (size_t)v->R_main);
    if (need > v->job_cap) {
        cudaFree(v->jobs);
        cudaFree(v->job_light);
        v->jobs = nullptr;
        v->job_light = nullptr;
        v->job_cap = 0;
        size_t dummy = 0;
        if (dalloc(&v->jobs, need, &dummy) != cudaSuccess || dalloc(&v->job_light, need, &dummy) != cudaSuccess)
            return fail(ADGI_ERR_OOM, "shadow job buffer");
        v->job_cap = need;
        stale = true;
    }
    if (v->desc.sampler == 1 && !v->mh_live) {  // first update: the chains' first states, before any capture
        const uint64_t key = splitmix(splitmix((f->seed ^ kMhInitSalt) ^ kMhSalt) ^ 0ull);
        CK(launch_mh_init(V, mh_bufs(v), key, s));
        v->mh_live = true;
        stale = true;
    }
    if (V.dyn && !v->dyn_live) {
        const uint64_t key = splitmix(splitmix(f->seed ^ kDynSalt ^ kMhInitSalt) ^ 0ull);
        CK(launch_dyn_init(V, dyn_bufs(v), key, s));
        v->dyn_live = true;
        stale = true;
    }
    if (graph_stale) *graph_stale = stale;
    return ADGI_OK;
}

// The device work of one update, in order, on stream s (capturable).  The
// frame descriptor fd is written to the device by the first kernel; when
// set_node is given, the captured node of that kernel is returned there.
int enqueue_update(adgi_volume v, const FrameDev& fd, cudaStream_t s, bool phases, cudaGraphNode_t* set_node)
{
    const VolConst& V = v->V;
    const Tuning& T = v->tune;
#define PHASE(i) \
    if (phases) CK(cudaEventRecord(v->ph[i], s))
    if (phases) CK(cudaEventRecord(v->ev0, s));
    CK(launch_set_frame(v->fdev, fd, s));
    if (set_node) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd));
        if (st != cudaStreamCaptureStatusActive || nd != 1) return fail(ADGI_ERR_CUDA, "capture: set-frame node");
        *set_node = deps[0];
    }
    PHASE(0);
    // the moving part of the scene: refresh its vertices and rebuild its BVH
    if (v->nd > 0 && (v->dyn_dirty || set_node)) {
        CK(fill_tri_orig(v->verts, v->idx, v->dlist, v->nv, v->nd, v->tri_orig, s));
        {
            int rc = build_moving(v, s);
            if (rc) return rc;
        }
    }
    if (!set_node) v->dyn_dirty = false;
    // the blend plan needs only the frame descriptor: run it on the side
    // stream, beside the traversals, and join before the blend
    BlendBufs Bb{v->off,  v->sf,  v->pil_rec, v->m_rec,
                 v->irr,  v->dep, v->dep_n,   carve_blend_plan(v->plan, V.rays_max - 8, V.Ti, V.Td), v->tex_src};
    const bool mh = v->desc.sampler == 1, cosg = v->desc.blend_mode == 1;
    if (!mh && !cosg) {
        CK(cudaEventRecord(v->fork, s));
        CK(cudaStreamWaitEvent(v->side, v->fork, 0));
        if (phases) CK(cudaEventRecord(v->plq[0], v->side));
        CK(launch_blend_plan(V, v->fdev, v->sf, Bb.plan, v->side));
        if (phases) CK(cudaEventRecord(v->plq[1], v->side));
        CK(cudaEventRecord(v->join, v->side));
    }
    SceneDev S = scene_view(v);
    const FrameDev* FD = v->fdev;
    CK(cudaMemsetAsync(v->shadow_ctr, 0, 8, s));
    ShadeWork W{v->vis, v->jobs, v->job_light, v->job_count, (unsigned)std::min<size_t>(v->job_cap, 0xFFFFFFFFu),
                v->shadow_blocks, v->shadow_ctr};
    // 1. pilot rays (trace + shade; the shading reads the previous atlases),
    // for the probes inside this frame's clip volume V_out
    PHASE(1);
    CK(launch_classify(V, FD, v->lut_c, v->cls, s));
    CK(launch_pilot_trace(V, FD, S, v->pil_hit, v->job_count + 2, T, s));
    PHASE(2);
    CK(launch_shade(V, FD, S, 0, (uint32_t)V.P * kPilots, nullptr, nullptr, v->irr, v->dep, v->pil_hit, v->pil_rec,
                    v->pil_lum, W, T, s, phases ? v->shq : nullptr));
    // 2. heuristics -> W_p
    PHASE(3);
    ChangeBufs C{v->pil_hit, v->pil_lum, v->lut_v, v->lut_c, v->qv,  v->qr,  v->qv_even, v->qr_even,
                 v->amp_v,   v->amp_r,   v->age_v, v->age_r, v->trv, v->trr, v->G,       v->W, v->qd, v->vout_even};
    CK(launch_change(V, FD, C, s));
    // 3. allocation
    PHASE(4);
    if (!mh) CK(launch_allocate(v->W, V.P, V.rays_avg, V.m0, V.rays_max, v->n, v->off, s, v->cls));
    if (mh) {
        // 3'. Metropolis chains draw the samples; group them by probe
        MhBufs M = mh_bufs(v);
        const uint32_t* ord = nullptr;
        CK(launch_mh_chain(V, FD, M, s));
        CK(launch_mh_group(V, M, s, &ord));
        v->mh_ord = ord;
        DynRays R{};
        if (V.dyn) {  // the dynamic chains, their marks and this frame's dynamic rays
            const DynBufs D = dyn_bufs(v);
            CK(launch_dyn_plan(V, FD, D, s));
            R = dyn_rays_of(D);
        }
        // 4'-5'. the samples' +w and -w rays (and the dynamic rays); shading
        PHASE(5);
        CK(launch_mh_trace(V, S, M, v->m_hit, v->mh_hitn, T, s));
        if (V.dyn) CK(launch_dyn_trace(V, S, R, v->dyn_Rd, v->dyn_hit, T, s));
        PHASE(6);
        CK(launch_shade(V, FD, S, 2, M.n_samples, nullptr, v->mh_smp_g, v->irr, v->dep, v->m_hit, v->m_rec, nullptr, W, T,
                        s, phases ? v->shq + 2 : nullptr));
        if (V.dyn)
            CK(launch_shade(V, FD, S, 3, v->dyn_Rd, nullptr, nullptr, v->irr, v->dep, v->dyn_hit, v->dyn_rec, nullptr, W,
                            T, s, nullptr, &R));
        // 6'. blend of the probes' samples (then their dynamic rays)
        PHASE(7);
        MhBlendBufs MB{M.n_samples, v->mh_off, v->mh_smp_g, v->m_rec,  v->mh_hitn, v->pil_rec, v->irr,
                       v->dep,      v->dep_n,  v->tex_src,  v->mh_smp_gn, R,         v->dyn_rec};
        CK(launch_mh_blend(V, FD, MB, s));
    } else {
        // 4-5. adaptive rays: trace, shade
        PHASE(5);
        CK(launch_main_trace(V, FD, S, v->off, v->sf, v->R_main, v->m_hit, v->job_count + 3, T, s));
        PHASE(6);
        CK(launch_shade(V, FD, S, 1, v->R_main, v->off, v->sf, v->irr, v->dep, v->m_hit, v->m_rec, nullptr, W, T, s,
                        phases ? v->shq + 2 : nullptr));
        // 6. blend (after every read of the previous atlases)
        PHASE(7);
        if (cosg) {
            CK(launch_blend_cos(V, FD, Bb, T, s));
        } else {
            CK(cudaStreamWaitEvent(s, v->join, 0));
            CK(launch_blend(V, FD, Bb, T, s));
        }
    }
    PHASE(8);
#undef PHASE
    if (phases) {
        CK(cudaEventRecord(v->ev1, s));
        v->timed_pending = true;
    }
    return ADGI_OK;
}

void finish_update(adgi_volume v, const FrameDev& fd, const adgi_frame* f)
{
    if (fd.F.even) v->last_even = (int64_t)f->frame;
    v->frames += 1;
}

}  // namespace

int adgi_update(adgi_volume v, const adgi_frame* f)
{
    FrameDev fd;
    int rc = prepare_update(v, f, fd, nullptr);
    if (rc) return rc;
    rc = enqueue_update(v, fd, v->stream, v->timing, nullptr);
    if (rc) return rc;
    finish_update(v, fd, f);
    return ADGI_OK;
}

// One rank's share of a probe-slab split update: the steps of
// enqueue_update (deterministic allocation) with the probe work restricted
// to [p0, p1); the allocation and the clip classes cover every probe.
int adgi_update_slab(adgi_volume v, const adgi_frame* f, int32_t step, int32_t p0, int32_t p1)
{
    if (!v || !f) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if (v->desc.sampler != 0 || v->desc.atlas_fp16 == 3)
        return fail(ADGI_ERR_INVALID_ARG, "the slab split takes sampler 0 with FP32 or half atlases");
    if (p0 < 0 || p0 > p1 || p1 > v->V.P) return fail(ADGI_ERR_INVALID_ARG, "probe range outside [0, P]");
    if (step < 0 || step > 2) return fail(ADGI_ERR_INVALID_ARG, "step must be 0, 1 or 2");
    if (step > 0 && (v->slab_step != step - 1 || v->slab_frame != f->frame || v->slab_p0 != p0 || v->slab_p1 != p1))
        return fail(ADGI_ERR_INVALID_ARG, "slab steps must run 0, 1, 2 on one frame and one probe range");
    cudaStream_t s = v->stream;
    if (step == 0) {
        int rc = prepare_update(v, f, v->slab_fd, nullptr);
        if (rc) return rc;
        v->slab_frame = f->frame;
        v->slab_p0 = p0;
        v->slab_p1 = p1;
    }
    v->slab_step = -1;  // until this step is enqueued
    const FrameDev& fd = v->slab_fd;
    const VolConst& V = v->V;
    VolConst Vs = v->V;
    Vs.p_lo = p0;
    Vs.p_hi = p1;
    const Tuning& T = v->tune;
    SceneDev S = scene_view(v);
    const FrameDev* FD = v->fdev;
    ShadeWork W{v->vis, v->jobs, v->job_light, v->job_count, (unsigned)std::min<size_t>(v->job_cap, 0xFFFFFFFFu),
                v->shadow_blocks, v->shadow_ctr};
    ChangeBufs C{v->pil_hit, v->pil_lum, v->lut_v, v->lut_c, v->qv,  v->qr,  v->qv_even, v->qr_even,
                 v->amp_v,   v->amp_r,   v->age_v, v->age_r, v->trv, v->trr, v->G,       v->W, v->qd, v->vout_even};
    BlendBufs Bb{v->off,  v->sf,  v->pil_rec, v->m_rec,
                 v->irr,  v->dep, v->dep_n,   carve_blend_plan(v->plan, V.rays_max - 8, V.Ti, V.Td), v->tex_src};
    const bool cosg = v->desc.blend_mode == 1;
    if (step == 0) {
        CK(launch_set_frame(v->fdev, fd, s));
        if (v->nd > 0 && v->dyn_dirty) {
            CK(fill_tri_orig(v->verts, v->idx, v->dlist, v->nv, v->nd, v->tri_orig, s));
            int rc = build_moving(v, s);
            if (rc) return rc;
        }
        v->dyn_dirty = false;
        if (!cosg) {  // the blend plan on the side stream; step 2 joins it before the blend
            CK(cudaEventRecord(v->fork, s));
            CK(cudaStreamWaitEvent(v->side, v->fork, 0));
            CK(launch_blend_plan(V, v->fdev, v->sf, Bb.plan, v->side));
            CK(cudaEventRecord(v->join, v->side));
        }
        CK(cudaMemsetAsync(v->shadow_ctr, 0, 8, s));
        CK(launch_classify(V, FD, v->lut_c, v->cls, s));
        CK(launch_pilot_trace(Vs, FD, S, v->pil_hit, v->job_count + 2, T, s));
        CK(launch_shade(Vs, FD, S, 0, (uint32_t)(p1 - p0) * kPilots, nullptr, nullptr, v->irr, v->dep, v->pil_hit,
                        v->pil_rec, v->pil_lum, W, T, s));
        CK(launch_change(Vs, FD, C, s, 1));
    } else if (step == 1) {
        CK(launch_change(Vs, FD, C, s, 2));
    } else {
        CK(launch_allocate(v->W, V.P, V.rays_avg, V.m0, V.rays_max, v->n, v->off, s, v->cls));
        CK(launch_main_trace(Vs, FD, S, v->off, v->sf, v->R_main, v->m_hit, v->job_count + 3, T, s));
        CK(launch_shade(Vs, FD, S, 1, v->R_main, v->off, v->sf, v->irr, v->dep, v->m_hit, v->m_rec, nullptr, W, T, s));
        if (cosg) {
            CK(launch_blend_cos(Vs, FD, Bb, T, s));
        } else {
            CK(cudaStreamWaitEvent(s, v->join, 0));
            CK(launch_blend(Vs, FD, Bb, T, s));
        }
        adgi_frame fcopy = *f;
        finish_update(v, fd, &fcopy);
    }
    v->slab_step = step;
    return ADGI_OK;
}

int adgi_slab_copy(adgi_volume v, int32_t which, int32_t p0, int32_t p1, void* dev_buf, int32_t into)
{
    if (!v || !dev_buf) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if (p0 < 0 || p0 > p1 || p1 > v->V.P) return fail(ADGI_ERR_INVALID_ARG, "probe range outside [0, P]");
    const size_t ti2 = (size_t)v->V.Ti * v->V.Ti, td2 = (size_t)v->V.Td * v->V.Td;
    size_t per = 0;
    char* base = nullptr;
    switch (which) {
    case ADGI_STATE_W: per = 4; base = (char*)v->W; break;
    case ADGI_STATE_TRV: per = 16; base = (char*)v->trv; break;
    case ADGI_STATE_TRR: per = 16; base = (char*)v->trr; break;
    case ADGI_STATE_G: per = 32; base = (char*)v->G; break;
    case ADGI_STATE_IRR: per = ti2 * (v->V.fp16 == 3 ? 4 : v->V.fp16 ? 8 : 16); base = (char*)v->irr; break;
    case ADGI_STATE_DEP: per = td2 * (v->V.fp16 ? 4 : 8); base = (char*)v->dep; break;
    case ADGI_STATE_DEP_N: per = td2; base = (char*)v->dep_n; break;
    default: return fail(ADGI_ERR_INVALID_ARG, "adgi_slab_copy: state not per probe");
    }
    const size_t n = per * (size_t)(p1 - p0);
    if (n == 0) return ADGI_OK;
    char* at = base + per * (size_t)p0;
    CK(cudaMemcpyAsync(into ? at : dev_buf, into ? dev_buf : at, n, cudaMemcpyDeviceToDevice, v->stream));
    return ADGI_OK;
}

int adgi_slab_bytes(adgi_volume v, int32_t which, int32_t p0, int32_t p1, uint64_t* bytes)
{
    if (!v || !bytes) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if (p0 < 0 || p0 > p1 || p1 > v->V.P) return fail(ADGI_ERR_INVALID_ARG, "probe range outside [0, P]");
    uint64_t all = 0;
    if (which != ADGI_STATE_W && which != ADGI_STATE_TRV && which != ADGI_STATE_TRR && which != ADGI_STATE_G &&
        which != ADGI_STATE_IRR && which != ADGI_STATE_DEP && which != ADGI_STATE_DEP_N)
        return fail(ADGI_ERR_INVALID_ARG, "adgi_slab_bytes: state not per probe");
    int rc = adgi_state_bytes(v, which, &all);
    if (rc) return rc;
    *bytes = all / (uint64_t)v->V.P * (uint64_t)(p1 - p0);
    return ADGI_OK;
}

namespace {

cudaError_t capture_end(cudaStream_t s, cudaGraph_t* g)
{
    cudaGraph_t tmp = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &tmp);
    *g = tmp;
    return e;
}

}  // namespace

int adgi_update_graph(adgi_volume v, const adgi_frame* f)
{
    FrameDev fd;
    bool stale = false;
    int rc = prepare_update(v, f, fd, &stale);
    if (rc) return rc;
    cudaStream_t s = v->stream;
    if (stale || !v->graph_ok) {
        if (v->gexec) cudaGraphExecDestroy(v->gexec);
        if (v->graph) cudaGraphDestroy(v->graph);
        v->gexec = nullptr;
        v->graph = nullptr;
        v->graph_ok = false;
        if (!v->cap_stream) CK(cudaStreamCreateWithFlags(&v->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamSynchronize(s));  // preparation work queued on the volume's stream
        CK(cudaStreamBeginCapture(v->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_update(v, fd, v->cap_stream, false, &v->gset);
        cudaGraph_t g = nullptr;
        cudaError_t e = capture_end(v->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(ADGI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        v->graph = g;
        CK(cudaGraphInstantiate(&v->gexec, v->graph, 0));
        v->graph_ok = true;
    } else {
        cudaKernelNodeParams kp;
        void* args[2];
        FrameDev* dst = v->fdev;
        set_frame_node_params(&dst, &fd, &kp, args);
        CK(cudaGraphExecKernelNodeSetParams(v->gexec, v->gset, &kp));
    }
    CK(cudaGraphLaunch(v->gexec, s));
    finish_update(v, fd, f);
    v->dyn_dirty = false;
    return ADGI_OK;
}

struct adgi_batch_s {
    std::vector<adgi_volume> vols;
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> setn;
    bool ok = false;
};

namespace {
void free_batch(adgi_batch b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t st : b->side)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}
}  // namespace

int adgi_batch_create(const adgi_volume* vols, int32_t n, void* cuda_stream, adgi_batch* out)
{
    if (!out || !vols || n <= 0 || n > 4096) return fail(ADGI_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!vols[i]) return fail(ADGI_ERR_INVALID_ARG, "NULL volume in batch");
        for (int j = 0; j < i; ++j)
            if (vols[j] == vols[i]) return fail(ADGI_ERR_INVALID_ARG, "a volume appears twice in the batch");
    }
    adgi_batch b = new adgi_batch_s();
    b->vols.assign(vols, vols + n);
    b->stream = (cudaStream_t)cuda_stream;
    b->side.assign(n, nullptr);
    b->join.assign(n, nullptr);
    b->setn.assign(n, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return fail(ADGI_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
    }
    *out = b;
    return ADGI_OK;
}

int adgi_batch_update(adgi_batch b, const adgi_frame* frames)
{
    if (!b || !frames) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    const int n = (int)b->vols.size();
    std::vector<FrameDev> fd(n);
    bool stale = !b->ok;
    for (int i = 0; i < n; ++i) {
        bool st = false;
        int rc = prepare_update(b->vols[i], &frames[i], fd[i], &st);
        if (rc) return rc;
        stale = stale || st;
    }
    if (stale) {
        // a static-part rebuild may have been queued on a volume's own stream
        for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(b->vols[i]->stream));
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        b->ok = false;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = ADGI_OK;
        cudaError_t e = cudaEventRecord(b->fork, b->stream);
        for (int i = 0; i < n && !rc && e == cudaSuccess; ++i) {
            e = cudaStreamWaitEvent(b->side[i], b->fork, 0);
            if (e == cudaSuccess) rc = enqueue_update(b->vols[i], fd[i], b->side[i], false, &b->setn[i]);
            if (!rc && e == cudaSuccess) e = cudaEventRecord(b->join[i], b->side[i]);
            if (!rc && e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = capture_end(b->stream, &g);
        if (rc || e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc) return rc;
            return fail(ADGI_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        b->graph = g;
        CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
        b->ok = true;
    } else {
        for (int i = 0; i < n; ++i) {
            cudaKernelNodeParams kp;
            void* args[2];
            FrameDev* dst = b->vols[i]->fdev;
            set_frame_node_params(&dst, &fd[i], &kp, args);
            CK(cudaGraphExecKernelNodeSetParams(b->exec, b->setn[i], &kp));
        }
    }
    CK(cudaGraphLaunch(b->exec, b->stream));
    for (int i = 0; i < n; ++i) {
        finish_update(b->vols[i], fd[i], &frames[i]);
        b->vols[i]->dyn_dirty = false;
    }
    return ADGI_OK;
}

int adgi_batch_destroy(adgi_batch b)
{
    if (!b) return ADGI_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return ADGI_OK;
}

// ---- the batched update as one persistent launch per tick (tick.cu)

struct adgi_tick_s {
    std::vector<adgi_volume> vols;
    cudaStream_t stream = nullptr;
    std::vector<cudaEvent_t> vol_ev;  // each volume's stream, joined before a tick
    cudaEvent_t done = nullptr;       // the last tick has read the staged frames
    FrameDev* h_fd = nullptr;         // pinned staging of the frame descriptors
    int* h_rb = nullptr;              // pinned staging: moving parts rebuilt inside the tick
    int* d_rb = nullptr;
    unsigned char* d_sort = nullptr;  // [n][kTickRebuildMax x 12 B] the moving parts' Morton sorts
    uint32_t* d_chunk = nullptr;      // the volumes' chunk_p arrays, one after the other
    TickCtl* d_ctl = nullptr;
    TickVol* d_vols = nullptr;
    uint32_t* d_pre = nullptr;
    int* d_cvol = nullptr;
    unsigned long long* d_scr = nullptr;
    int n_chunks = 0;
    unsigned grid = 0;
    size_t smem = 0;
    bool tables_ok = false;
    bool launched = false;
};

namespace {
void free_tick_tables(adgi_tick t)
{
    cudaFree(t->d_vols);
    cudaFree(t->d_pre);
    cudaFree(t->d_cvol);
    cudaFree(t->d_scr);
    t->d_vols = nullptr;
    t->d_pre = nullptr;
    t->d_cvol = nullptr;
    t->d_scr = nullptr;
    t->tables_ok = false;
}

void free_tick(adgi_tick t)
{
    if (!t) return;
    free_tick_tables(t);
    cudaFree(t->d_ctl);
    cudaFree(t->d_rb);
    cudaFree(t->d_sort);
    cudaFree(t->d_chunk);
    if (t->h_fd) cudaFreeHost(t->h_fd);
    if (t->h_rb) cudaFreeHost(t->h_rb);
    for (cudaEvent_t e : t->vol_ev)
        if (e) cudaEventDestroy(e);
    if (t->done) cudaEventDestroy(t->done);
    delete t;
}

TickVol tick_vol_of(adgi_tick t, int i)
{
    adgi_volume v = t->vols[i];
    TickVol T;
    std::memset(&T, 0, sizeof(T));
    T.w.V = v->V;
    T.w.V.p_lo = 0;
    T.w.V.p_hi = v->V.P;
    T.w.S = scene_view(v);
    T.w.FD = v->fdev;
    T.w.off = v->off;
    T.w.sf = v->sf;
    T.w.pil_hit = v->pil_hit;
    T.w.m_hit = v->m_hit;
    T.w.Wk = ShadeWork{v->vis, v->jobs, v->job_light, v->job_count,
                       (unsigned)std::min<size_t>(v->job_cap, 0xFFFFFFFFu), 0u, v->shadow_ctr};
    T.lut_c = v->lut_c;
    T.cls = v->cls;
    T.pil_rec = v->pil_rec;
    T.pil_lum = v->pil_lum;
    T.m_rec = v->m_rec;
    T.n = v->n;
    T.off = v->off;
    T.C = ChangeBufs{v->pil_hit, v->pil_lum, v->lut_v, v->lut_c, v->qv,  v->qr,  v->qv_even, v->qr_even,
                     v->amp_v,   v->amp_r,   v->age_v, v->age_r, v->trv, v->trr, v->G,       v->W, v->qd, v->vout_even};
    T.B = BlendBufs{v->off, v->sf,  v->pil_rec, v->m_rec,
                    v->irr, v->dep, v->dep_n,   carve_blend_plan(v->plan, v->V.rays_max - 8, v->V.Ti, v->V.Td),
                    v->tex_src};
    T.avg = v->V.rays_avg;
    T.m0 = v->V.m0;
    T.rmax = v->V.rays_max;
    T.verts = v->verts;
    T.idx = v->idx;
    T.dlist = v->dlist;
    T.nv = v->nv;
    T.nd = v->nd;
    T.node_off = moving_node_off(v);
    T.tri_off = moving_tri_off(v);
    T.eps = v->eps;
    T.tri_orig = v->tri_orig;
    T.tri_in = v->dbvh.bufs.tri_in;
    T.keys = v->dbvh.bufs.keys[0];
    T.vals = v->dbvh.bufs.vals[0];
    T.par_int = v->dbvh.bufs.par_int;
    T.par_leaf = v->dbvh.bufs.par_leaf;
    T.flags = v->dbvh.bufs.flags;
    T.w.chunk_p = nullptr;  // set by build_tick_tables
    T.sort_k = reinterpret_cast<uint64_t*>(t->d_sort + (size_t)12 * kTickRebuildMax * i);
    T.sort_v = reinterpret_cast<uint32_t*>(T.sort_k + kTickRebuildMax);
    return T;
}

// (Re)build the device tables: per-volume parameters, the phases' virtual
// blocks, the allocation chunks, the grid and its shared memory.
int build_tick_tables(adgi_tick t, std::vector<TickVol>& hv)
{
    CK(cudaStreamSynchronize(t->stream));  // no tick may still read the old tables
    free_tick_tables(t);
    const int n = (int)t->vols.size();
    std::vector<uint32_t> pre((size_t)kTickPhases * (n + 1), 0u);
    std::vector<int> cvol;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        adgi_volume v = t->vols[i];
        uint32_t cnt[kTickPhases];
        tick_phase_blocks(v->V, v->R_main, v->nd, cnt);
        for (int ph = 0; ph < kTickPhases; ++ph) {
            const uint64_t x = (uint64_t)pre[(size_t)ph * (n + 1) + i] + cnt[ph];
            if (x > 0x7FFFFFFFull) return fail(ADGI_ERR_INVALID_ARG, "tick: too much work for one launch");
            pre[(size_t)ph * (n + 1) + i + 1] = (uint32_t)x;
        }
        hv[i].chunk0 = (int)cvol.size();
        for (int c = 0; c < (v->V.P + kTickChunk - 1) / kTickChunk; ++c) cvol.push_back(i);
        smem = std::max(smem, tick_smem_bytes(v->V));
    }
    // the chunk-to-probe arrays (R_main / 32 + 2 entries a volume)
    {
        size_t total = 0;
        std::vector<size_t> at(n);
        for (int i = 0; i < n; ++i) {
            at[i] = total;
            total += (size_t)t->vols[i]->R_main / 32 + 2;
        }
        cudaFree(t->d_chunk);
        t->d_chunk = nullptr;
        size_t b = 0;
        if (dalloc(&t->d_chunk, total, &b) != cudaSuccess) return fail(ADGI_ERR_OOM, "tick chunk table");
        for (int i = 0; i < n; ++i) hv[i].w.chunk_p = t->d_chunk + at[i];
    }
    const unsigned grid = tick_grid_blocks(smem);
    if (grid == 0) return fail(ADGI_ERR_CUDA, "tick: no resident grid for the persistent kernel");
    if (cvol.size() > (size_t)kTickOwn * grid)
        return fail(ADGI_ERR_INVALID_ARG, "tick: more probes than one persistent grid allocates");
    size_t b = 0;
    if (dalloc(&t->d_vols, (size_t)n, &b) != cudaSuccess || dalloc(&t->d_pre, pre.size(), &b) != cudaSuccess ||
        dalloc(&t->d_cvol, cvol.size(), &b) != cudaSuccess ||
        dalloc(&t->d_scr, (size_t)kTickScratch * cvol.size(), &b) != cudaSuccess) {
        free_tick_tables(t);
        return fail(ADGI_ERR_OOM, "tick tables");
    }
    CK(cudaMemcpyAsync(t->d_vols, hv.data(), sizeof(TickVol) * n, cudaMemcpyHostToDevice, t->stream));
    CK(cudaMemcpyAsync(t->d_pre, pre.data(), sizeof(uint32_t) * pre.size(), cudaMemcpyHostToDevice, t->stream));
    CK(cudaMemcpyAsync(t->d_cvol, cvol.data(), sizeof(int) * cvol.size(), cudaMemcpyHostToDevice, t->stream));
    CK(cudaStreamSynchronize(t->stream));  // the host vectors are freed on return
    t->n_chunks = (int)cvol.size();
    t->grid = grid;
    t->smem = smem;
    t->tables_ok = true;
    return ADGI_OK;
}
}  // namespace

int adgi_tick_create(const adgi_volume* vols, int32_t n, void* cuda_stream, adgi_tick* out)
{
    if (!out || !vols || n <= 0 || n > 4096) return fail(ADGI_ERR_INVALID_ARG, "bad tick arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!vols[i]) return fail(ADGI_ERR_INVALID_ARG, "NULL volume in tick");
        for (int j = 0; j < i; ++j)
            if (vols[j] == vols[i]) return fail(ADGI_ERR_INVALID_ARG, "a volume appears twice in the tick");
        if (vols[i]->desc.sampler != 0 || vols[i]->desc.blend_mode != 0)
            return fail(ADGI_ERR_INVALID_ARG, "tick: only the deterministic allocation with the texel blend");
    }
    adgi_tick t = new adgi_tick_s();
    t->vols.assign(vols, vols + n);
    t->stream = (cudaStream_t)cuda_stream;
    t->vol_ev.assign(n, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&t->vol_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&t->h_fd, sizeof(FrameDev) * n);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&t->h_rb, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->d_rb, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->d_sort, (size_t)12 * kTickRebuildMax * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->d_ctl, sizeof(TickCtl));
    if (e == cudaSuccess) {
        TickCtl c;
        std::memset(&c, 0, sizeof(c));
        c.limit_ns = 2000000000ull;  // 2 s: far beyond any phase of a tick
        c.stall = -1;
        e = cudaMemcpy(t->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_tick(t);
        return fail(ADGI_ERR_CUDA, std::string("tick: ") + cudaGetErrorString(e));
    }
    *out = t;
    return ADGI_OK;
}

int adgi_tick_update(adgi_tick t, const adgi_frame* frames)
{
    if (!t || !frames) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    const int n = (int)t->vols.size();
    std::vector<FrameDev> fd(n);
    bool stale = !t->tables_ok;  // a buffer the tables name may have moved
    for (int i = 0; i < n; ++i) {
        bool st = false;
        int rc = prepare_update(t->vols[i], &frames[i], fd[i], &st);
        if (rc) return rc;
        stale = stale || st;
    }
    // work queued on the volumes' own streams (scene uploads, rebuilds) first
    for (int i = 0; i < n; ++i) {
        if (t->vols[i]->stream == t->stream) continue;
        CK(cudaEventRecord(t->vol_ev[i], t->vols[i]->stream));
        CK(cudaStreamWaitEvent(t->stream, t->vol_ev[i], 0));
    }
    // moving parts whose vertices moved: rebuilt inside the launch (up to
    // kTickRebuildMax triangles), else before it
    if (t->launched) CK(cudaEventSynchronize(t->done));  // the staging buffers are rewritten below
    int any_rb = 0;
    for (int i = 0; i < n; ++i) {
        adgi_volume v = t->vols[i];
        t->h_rb[i] = 0;
        if (v->nd > 0 && v->dyn_dirty) {
            if (v->nd <= kTickRebuildMax) {
                t->h_rb[i] = 1;
                any_rb = 1;
            } else {
                CK(fill_tri_orig(v->verts, v->idx, v->dlist, v->nv, v->nd, v->tri_orig, t->stream));
                int rc = build_moving(v, t->stream);
                if (rc) return rc;
            }
            v->dyn_dirty = false;
        }
    }
    if (stale) {
        std::vector<TickVol> hv(n);
        for (int i = 0; i < n; ++i) hv[i] = tick_vol_of(t, i);
        int rc = build_tick_tables(t, hv);
        if (rc) return rc;
    }
    std::memcpy(t->h_fd, fd.data(), sizeof(FrameDev) * n);
    CK(cudaMemcpyAsync(t->d_rb, t->h_rb, sizeof(int) * n, cudaMemcpyHostToDevice, t->stream));
    for (int i = 0; i < n; ++i)  // each volume's own descriptor, as the plain update leaves it
        CK(cudaMemcpyAsync(t->vols[i]->fdev, t->h_fd + i, sizeof(FrameDev), cudaMemcpyHostToDevice, t->stream));
    CK(cudaMemsetAsync(t->d_ctl, 0, offsetof(TickCtl, limit_ns), t->stream));
    CK(launch_tick(t->d_vols, n, t->d_pre, t->d_cvol, t->n_chunks, t->d_scr, t->d_ctl, t->d_rb, any_rb, t->grid,
                   t->smem, t->stream));
    CK(cudaEventRecord(t->done, t->stream));
    t->launched = true;
    for (int i = 0; i < n; ++i) finish_update(t->vols[i], fd[i], &frames[i]);
    return ADGI_OK;
}

int adgi_tick_sync(adgi_tick t)
{
    if (!t) return fail(ADGI_ERR_INVALID_ARG, "NULL tick");
    CK(cudaStreamSynchronize(t->stream));
    int status = 0;
    CK(cudaMemcpy(&status, &t->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status == kTickTimedOut) return fail(ADGI_ERR_TIMEOUT, "tick: a grid barrier wait gave up");
    if (status != 0) return fail(ADGI_ERR_CUDA, "tick: bad status");
    return ADGI_OK;
}

int adgi_tick_set_wait(adgi_tick t, uint64_t limit_ns, int32_t stall_barrier)
{
    if (!t || limit_ns == 0 || limit_ns > 60000000000ull || stall_barrier < -1)
        return fail(ADGI_ERR_INVALID_ARG, "bad tick wait arguments");
    CK(cudaStreamSynchronize(t->stream));
    const unsigned long long lim = limit_ns;
    const int st = stall_barrier;
    CK(cudaMemcpy(&t->d_ctl->limit_ns, &lim, sizeof(lim), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(&t->d_ctl->stall, &st, sizeof(st), cudaMemcpyHostToDevice));
    return ADGI_OK;
}

int adgi_tick_info(adgi_tick t, uint32_t* grid_blocks, uint32_t* smem_bytes, uint32_t* chunks)
{
    if (!t) return fail(ADGI_ERR_INVALID_ARG, "NULL tick");
    if (grid_blocks) *grid_blocks = t->grid;
    if (smem_bytes) *smem_bytes = (uint32_t)t->smem;
    if (chunks) *chunks = (uint32_t)t->n_chunks;
    return ADGI_OK;
}

int adgi_tick_phase_ns(adgi_tick t, uint64_t* out, int32_t n)
{
    if (!t || !out || n < 0) return fail(ADGI_ERR_INVALID_ARG, "bad tick phase arguments");
    CK(cudaStreamSynchronize(t->stream));
    unsigned long long st[1 + kTickStamps];
    CK(cudaMemcpy(st, &t->d_ctl->t_start, sizeof(st), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) out[i] = i < kTickStamps && st[i + 1] >= st[0] ? st[i + 1] - st[0] : 0;
    return ADGI_OK;
}

int adgi_tick_destroy(adgi_tick t)
{
    if (!t) return ADGI_OK;
    cudaStreamSynchronize(t->stream);
    free_tick(t);
    return ADGI_OK;
}

int adgi_set_tuning(adgi_volume v, const adgi_tuning* t)
{
    if (!v || !t) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    auto okb = [](int x) { return x == 32 || x == 64 || x == 128 || x == 256; };
    if (!okb(t->trace_block) || !okb(t->shade_block) || !okb(t->blend_block) || t->shadow_blocks_per_sm < 0 ||
        t->shadow_blocks_per_sm > 64)
        return fail(ADGI_ERR_INVALID_ARG, "block sizes must be 32, 64, 128 or 256");
    v->tune.trace_block = t->trace_block;
    v->tune.shade_block = t->shade_block;
    v->tune.blend_block = t->blend_block;
    v->tune.shadow_mult = t->shadow_blocks_per_sm;
    v->graph_ok = false;
    return ADGI_OK;
}

int adgi_get_tuning(adgi_volume v, adgi_tuning* t)
{
    if (!v || !t) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    std::memset(t, 0, sizeof(*t));
    t->trace_block = v->tune.trace_block;
    t->shade_block = v->tune.shade_block;
    t->blend_block = v->tune.blend_block;
    t->shadow_blocks_per_sm = v->tune.shadow_mult;
    return ADGI_OK;
}

int adgi_autotune(adgi_volume v, const adgi_frame* f, int32_t reps, adgi_tuning* out)
{
    if (!v || !f) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if (v->frames == 0) return fail(ADGI_ERR_INVALID_ARG, "autotune needs one update first");
    if (v->desc.sampler == 1 || v->desc.blend_mode == 1)
        return fail(ADGI_ERR_INVALID_ARG, "autotune: not available with the Metropolis sampler or the cosine gather");
    if (reps < 1) reps = 1;
    FrameDev fd;
    int rc = prepare_update(v, f, fd, nullptr);
    if (rc) return rc;
    cudaStream_t s = v->stream;
    const VolConst& V = v->V;
    SceneDev S = scene_view(v);
    CK(launch_set_frame(v->fdev, fd, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timed = [&](auto&& body, float* ms) -> int {
        cudaError_t e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = body();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        if (e != cudaSuccess) return fail(ADGI_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        *ms /= (float)reps;
        return ADGI_OK;
    };
    const int blocks[3] = {64, 128, 256};
    Tuning best = v->tune;
    float t_trace = 1e30f, t_shade = 1e30f, t_blend = 1e30f;
    for (int b : blocks) {  // nearest-hit traversal
        Tuning T = best;
        T.trace_block = b;
        float ms = 0.f;
        rc = timed([&] { return launch_main_trace(V, v->fdev, S, v->off, v->sf, v->R_main, v->m_hit, v->job_count + 3, T, s); }, &ms);
        if (rc) break;
        if (ms < t_trace) {
            t_trace = ms;
            best.trace_block = b;
        }
    }
    const int mults[4] = {0, 2, 4, 8};
    for (int b : blocks) {  // shading wavefront (shadow grid per SM, prep/finish blocks)
        for (int m : mults) {
            if (rc) break;
            Tuning T = best;
            T.shade_block = b;
            T.shadow_mult = m;
            ShadeWork W{v->vis, v->jobs, v->job_light, v->job_count, (unsigned)std::min<size_t>(v->job_cap, 0xFFFFFFFFu),
                        shadow_grid_blocks(m), v->shadow_ctr};
            float ms = 0.f;
            rc = timed([&] {
                return launch_shade(V, v->fdev, S, 1, v->R_main, v->off, v->sf, v->irr, v->dep, v->m_hit, v->m_rec,
                                    nullptr, W, T, s);
            }, &ms);
            if (!rc && ms < t_shade) {
                t_shade = ms;
                best.shade_block = b;
                best.shadow_mult = m;
            }
        }
    }
    // blend: trials run on the live atlases, which are restored afterwards
    uint64_t bi = 0, bd = 0, bn = 0;
    adgi_state_bytes(v, ADGI_STATE_IRR, &bi);
    adgi_state_bytes(v, ADGI_STATE_DEP, &bd);
    adgi_state_bytes(v, ADGI_STATE_DEP_N, &bn);
    void* keep = nullptr;
    if (!rc && cudaMalloc(&keep, bi + bd + bn) != cudaSuccess) rc = fail(ADGI_ERR_OOM, "autotune snapshot");
    if (!rc) {
        char* k = (char*)keep;
        CK(cudaMemcpyAsync(k, v->irr, bi, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(k + bi, v->dep, bd, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(k + bi + bd, v->dep_n, bn, cudaMemcpyDeviceToDevice, s));
        BlendBufs Bb{v->off,  v->sf,  v->pil_rec, v->m_rec,
                 v->irr,  v->dep, v->dep_n,   carve_blend_plan(v->plan, V.rays_max - 8, V.Ti, V.Td), v->tex_src};
        const int wblocks[3] = {32, 64, 128};  // 1, 2 or 4 probe tiles (warps) per CTA
        for (int b : wblocks) {
            if (rc) break;
            Tuning T = best;
            T.blend_block = b;
            float ms = 0.f;
            rc = timed([&] { return launch_blend(V, v->fdev, Bb, T, s); }, &ms);
            if (!rc && ms < t_blend) {
                t_blend = ms;
                best.blend_block = b;
            }
        }
        cudaMemcpyAsync(v->irr, k, bi, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(v->dep, k + bi, bd, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(v->dep_n, k + bi + bd, bn, cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
    }
    if (keep) cudaFree(keep);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    v->tune = best;
    v->graph_ok = false;
    if (out) {
        adgi_get_tuning(v, out);
        out->ms_trace = t_trace;
        out->ms_shade = t_shade;
        out->ms_blend = t_blend;
    }
    return ADGI_OK;
}

int adgi_query_irradiance(adgi_volume v, const float* pos, const float* nrm, int32_t n, float* out, int32_t on_device)
{
    if (!v || n < 0 || (n > 0 && (!pos || !nrm || !out))) return fail(ADGI_ERR_INVALID_ARG, "bad query arguments");
    if (n == 0) return ADGI_OK;
    cudaStream_t s = v->stream;
    if (on_device) {
        CK(launch_query(v->V, v->irr, v->dep, pos, nrm, n, out, s));
        return ADGI_OK;
    }
    if (n > v->q_cap) {
        cudaFree(v->q_buf);
        v->q_buf = nullptr;
        size_t dummy = 0;
        if (dalloc(&v->q_buf, 9 * (size_t)n, &dummy) != cudaSuccess) return fail(ADGI_ERR_OOM, "query buffer");
        v->q_cap = n;
    }
    float* dp = v->q_buf;
    float* dn = dp + 3 * (size_t)n;
    float* dout = dn + 3 * (size_t)n;
    CK(cudaMemcpyAsync(dp, pos, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dn, nrm, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
    CK(launch_query(v->V, v->irr, v->dep, dp, dn, n, dout, s));
    CK(cudaMemcpyAsync(out, dout, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ADGI_OK;
}

int adgi_get_stats(adgi_volume v, adgi_stats* out)
{
    if (!v || !out) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    CK(cudaStreamSynchronize(v->stream));
    std::memset(out, 0, sizeof(*out));
    out->frames = v->frames;
    out->rays_per_update = v->desc.sampler == 1 ? (uint64_t)v->V.P * 8u + 2u * (uint64_t)v->mh_B
                                                : (uint64_t)v->V.P * (uint64_t)v->V.rays_avg;
    if (v->V.dyn) {  // plus the last update's dynamic rays
        uint32_t nd = 0;
        CK(cudaMemcpy(&nd, v->dyn_off + v->V.P, 4, cudaMemcpyDeviceToHost));
        out->rays_per_update += nd;
    }
    out->pilot_rays = (uint64_t)v->V.P * 8u;
    unsigned long long sc = 0;
    CK(cudaMemcpy(&sc, v->shadow_ctr, 8, cudaMemcpyDeviceToHost));
    out->shadow_rays = sc;
    int ef = 0;
    CK(cudaMemcpy(&ef, v->err, 4, cudaMemcpyDeviceToHost));
    if (ef) return fail(ADGI_ERR_CUDA, "device anomaly flags set: " + std::to_string(ef));
    out->bvh_nodes = (uint32_t)((v->ns > 1 ? v->ns - 1 : 0) + (v->nd > 1 ? v->nd - 1 : 0));
    out->n_tris = (uint32_t)v->nt;
    out->device_bytes = v->bytes + v->sbvh.bytes() + v->dbvh.bytes();
    out->kernels_launched = adgi::kernels_launched();
    if (v->timed_pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, v->ev0, v->ev1));
        out->ms_last_update = ms;
        for (int i = 0; i < 8; ++i) CK(cudaEventElapsedTime(&out->ms_phase[i], v->ph[i], v->ph[i + 1]));
        for (int i = 0; i < 2; ++i) CK(cudaEventElapsedTime(&out->ms_shadow[i], v->shq[2 * i], v->shq[2 * i + 1]));
        if (v->desc.sampler != 1 && v->desc.blend_mode != 1)
            CK(cudaEventElapsedTime(&out->ms_blend_plan, v->plq[0], v->plq[1]));
    }
    return ADGI_OK;
}

int adgi_state_bytes(adgi_volume v, int32_t which, uint64_t* bytes)
{
    if (!v || !bytes) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if ((which == ADGI_STATE_BVH_NODES || which == ADGI_STATE_BVH_TRIS || which == ADGI_STATE_MOVING_BVH_NODES ||
         which == ADGI_STATE_MOVING_BVH_TRIS) && v->has_scene) {
        int rc = ensure_bvh(v, v->stream);  // sizes depend on the static/moving split
        if (rc) return rc;
    }
    const uint64_t P = (uint64_t)v->V.P, R = v->R_main;
    const uint64_t ti2 = (uint64_t)v->V.Ti * v->V.Ti, td2 = (uint64_t)v->V.Td * v->V.Td;
    switch (which) {
    case ADGI_STATE_W:
    case ADGI_STATE_N: *bytes = 4 * P; break;
    case ADGI_STATE_OFF: *bytes = 4 * (P + 1); break;
    case ADGI_STATE_QV:
    case ADGI_STATE_QR:
    case ADGI_STATE_TRV:
    case ADGI_STATE_TRR: *bytes = 2 * 8 * P; break;
    case ADGI_STATE_PILOT_HIT: *bytes = 8 * 8 * P; break;
    case ADGI_STATE_PILOT_REC: *bytes = 16 * 8 * P; break;
    case ADGI_STATE_PILOT_LUM: *bytes = 4 * 8 * P; break;
    case ADGI_STATE_MAIN_HIT: *bytes = 8 * R; break;
    case ADGI_STATE_MAIN_REC: *bytes = 16 * R; break;
    case ADGI_STATE_IRR: *bytes = P * ti2 * (v->V.fp16 == 3 ? 4 : v->V.fp16 ? 8 : 16); break;
    case ADGI_STATE_DEP: *bytes = P * td2 * (v->V.fp16 ? 4 : 8); break;
    case ADGI_STATE_DEP_N: *bytes = P * td2; break;
    case ADGI_STATE_G: *bytes = 4 * 8 * P; break;
    case ADGI_STATE_DEP_MOMENTS:
        if (v->V.fp16 == 3) return fail(ADGI_ERR_INVALID_ARG, "DEP_MOMENTS: packed atlases hold codes (read DEP)");
        *bytes = P * td2 * 16;
        break;
    case ADGI_STATE_ROT: *bytes = 36; break;
    case ADGI_STATE_BVH_NODES: *bytes = 64 * (uint64_t)(v->ns > 1 ? v->ns - 1 : 1); break;
    case ADGI_STATE_BVH_TRIS: *bytes = 48 * (uint64_t)v->ns; break;
    case ADGI_STATE_MOVING_BVH_NODES: *bytes = 64 * (uint64_t)(v->nd > 1 ? v->nd - 1 : 1); break;
    case ADGI_STATE_MOVING_BVH_TRIS: *bytes = 48 * (uint64_t)v->nd; break;
    case ADGI_STATE_MH_CHAINS:
    case ADGI_STATE_MH_SAMPLES:
    case ADGI_STATE_MH_ORDER:
    case ADGI_STATE_MH_OFF:
    case ADGI_STATE_MH_HIT_NEG:
        if (v->desc.sampler != 1) return fail(ADGI_ERR_INVALID_ARG, "not a Metropolis volume");
        *bytes = which == ADGI_STATE_MH_CHAINS    ? 32 * (uint64_t)v->mh_C
                 : which == ADGI_STATE_MH_SAMPLES ? 16 * (uint64_t)v->mh_B
                 : which == ADGI_STATE_MH_ORDER   ? 4 * (uint64_t)v->mh_B
                 : which == ADGI_STATE_MH_OFF     ? 4 * (P + 1)
                                                  : 8 * (uint64_t)v->mh_B;
        break;
    case ADGI_STATE_QD: *bytes = 4 * 8 * P; break;
    case ADGI_STATE_CLS: *bytes = P; break;
    case ADGI_STATE_DYN_CHAINS:
    case ADGI_STATE_DYN_SAMPLES:
    case ADGI_STATE_DYN_CELLS:
    case ADGI_STATE_DYN_FIRST:
    case ADGI_STATE_DYN_INCL:
    case ADGI_STATE_DYN_OFF:
    case ADGI_STATE_DYN_HIT:
    case ADGI_STATE_DYN_REC: {
        if (!v->V.dyn) return fail(ADGI_ERR_INVALID_ARG, "no dynamic chains in this volume");
        const uint64_t cells = 8 * (uint64_t)v->dyn_pp;
        *bytes = which == ADGI_STATE_DYN_CHAINS    ? 32 * (uint64_t)v->dyn_Cd
                 : which == ADGI_STATE_DYN_SAMPLES ? 16 * (uint64_t)v->dyn_Bd
                 : which == ADGI_STATE_DYN_CELLS   ? 4 * (uint64_t)v->dyn_Bd
                 : which == ADGI_STATE_DYN_FIRST   ? 4 * cells
                 : which == ADGI_STATE_DYN_INCL    ? cells
                 : which == ADGI_STATE_DYN_OFF     ? 4 * (P + 1)
                 : which == ADGI_STATE_DYN_HIT     ? 8 * (uint64_t)v->dyn_Rd
                                                   : 16 * (uint64_t)v->dyn_Rd;
        break;
    }
    default: return fail(ADGI_ERR_INVALID_ARG, "unknown state");
    }
    return ADGI_OK;
}

int adgi_read_state(adgi_volume v, int32_t which, void* dst, uint64_t bytes)
{
    if (v && (which == ADGI_STATE_BVH_NODES || which == ADGI_STATE_BVH_TRIS || which == ADGI_STATE_MOVING_BVH_NODES ||
              which == ADGI_STATE_MOVING_BVH_TRIS) && v->has_scene) {
        int rc = ensure_bvh(v, v->stream);
        if (rc) return rc;
    }
    uint64_t need = 0;
    int rc = adgi_state_bytes(v, which, &need);
    if (rc) return rc;
    if (!dst || bytes != need) return fail(ADGI_ERR_INVALID_ARG, "destination size mismatch");
    CK(cudaStreamSynchronize(v->stream));
    if (which == ADGI_STATE_ROT) {
        std::memcpy(dst, v->R, 36);
        return ADGI_OK;
    }
    if (which == ADGI_STATE_DEP_MOMENTS) {  // {mean, variance} -> {mean, variance + mean^2} in FP64
        const size_t n = (size_t)v->V.P * v->V.Td * v->V.Td;
        double* out = static_cast<double*>(dst);
        if (v->V.fp16) {
            std::vector<__half> h(2 * n);
            CK(cudaMemcpy(h.data(), v->dep, h.size() * sizeof(__half), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < n; ++i) {
                const double m = (double)__half2float(h[2 * i]), var = (double)__half2float(h[2 * i + 1]);
                out[2 * i] = m;
                out[2 * i + 1] = var + m * m;
            }
        } else {
            std::vector<float> f(2 * n);
            CK(cudaMemcpy(f.data(), v->dep, f.size() * sizeof(float), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < n; ++i) {
                const double m = (double)f[2 * i], var = (double)f[2 * i + 1];
                out[2 * i] = m;
                out[2 * i + 1] = var + m * m;
            }
        }
        return ADGI_OK;
    }
    const void* src = nullptr;
    int count_tris = -1;
    switch (which) {
    case ADGI_STATE_W: src = v->W; break;
    case ADGI_STATE_N: src = v->n; break;
    case ADGI_STATE_OFF: src = v->off; break;
    case ADGI_STATE_QV: src = v->qv; break;
    case ADGI_STATE_QR: src = v->qr; break;
    case ADGI_STATE_TRV: src = v->trv; break;
    case ADGI_STATE_TRR: src = v->trr; break;
    case ADGI_STATE_PILOT_HIT: src = v->pil_hit; break;
    case ADGI_STATE_PILOT_REC: src = v->pil_rec; break;
    case ADGI_STATE_PILOT_LUM: src = v->pil_lum; break;
    case ADGI_STATE_MAIN_HIT: src = v->m_hit; break;
    case ADGI_STATE_MAIN_REC: src = v->m_rec; break;
    case ADGI_STATE_IRR: src = v->irr; break;
    case ADGI_STATE_DEP: src = v->dep; break;
    case ADGI_STATE_DEP_N: src = v->dep_n; break;
    case ADGI_STATE_BVH_NODES: src = v->sbvh.nodes; count_tris = v->ns; break;
    case ADGI_STATE_BVH_TRIS: src = v->sbvh.tri_v; count_tris = v->ns; break;
    case ADGI_STATE_MOVING_BVH_NODES: src = v->sbvh.nodes + moving_node_off(v); count_tris = v->nd; break;
    case ADGI_STATE_MOVING_BVH_TRIS: src = v->sbvh.tri_v + 3 * (size_t)moving_tri_off(v); count_tris = v->nd; break;
    case ADGI_STATE_MH_CHAINS: src = v->mh_chain; break;
    case ADGI_STATE_MH_SAMPLES: src = v->mh_smp; break;
    case ADGI_STATE_MH_ORDER: src = v->mh_ord; break;
    case ADGI_STATE_MH_OFF: src = v->mh_off; break;
    case ADGI_STATE_MH_HIT_NEG: src = v->mh_hitn; break;
    case ADGI_STATE_QD: src = v->qd; break;
    case ADGI_STATE_CLS: src = v->cls; break;
    case ADGI_STATE_G: src = v->G; break;
    case ADGI_STATE_DYN_CHAINS: src = v->dyn_chain; break;
    case ADGI_STATE_DYN_SAMPLES: src = v->dyn_smp; break;
    case ADGI_STATE_DYN_CELLS: src = v->dyn_cell; break;
    case ADGI_STATE_DYN_FIRST: src = v->dyn_first; break;
    case ADGI_STATE_DYN_INCL: src = v->dyn_incl; break;
    case ADGI_STATE_DYN_OFF: src = v->dyn_off; break;
    case ADGI_STATE_DYN_HIT: src = v->dyn_hit; break;
    case ADGI_STATE_DYN_REC: src = v->dyn_rec; break;
    }
    bool nodes = which == ADGI_STATE_BVH_NODES || which == ADGI_STATE_MOVING_BVH_NODES;
    if (count_tris >= 0 && (count_tris == 0 || (nodes && count_tris < 2))) {
        std::memset(dst, 0, bytes);  // no tree (0 or 1 triangle)
        return ADGI_OK;
    }
    if (bytes) CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    if (which == ADGI_STATE_MOVING_BVH_NODES) {  // references back to the moving tree's own indices
        const int no = moving_node_off(v), to = moving_tri_off(v);
        for (size_t i = 0; i < bytes / sizeof(BNode); ++i) {
            int* c = reinterpret_cast<int*>(static_cast<char*>(dst) + i * sizeof(BNode) + offsetof(BNode, d));
            for (int k = 0; k < 2; ++k) c[k] = c[k] >= 0 ? c[k] - no : ~(~c[k] - to);
        }
    }
    return ADGI_OK;
}

int adgi_write_atlas(adgi_volume v, const void* irr, const void* dep, const uint8_t* dep_n)
{
    if (!v) return fail(ADGI_ERR_INVALID_ARG, "volume is NULL");
    uint64_t b;
    CK(cudaStreamSynchronize(v->stream));
    if (irr) {
        adgi_state_bytes(v, ADGI_STATE_IRR, &b);
        CK(cudaMemcpy(v->irr, irr, b, cudaMemcpyHostToDevice));
    }
    if (dep) {
        adgi_state_bytes(v, ADGI_STATE_DEP, &b);
        CK(cudaMemcpy(v->dep, dep, b, cudaMemcpyHostToDevice));
    }
    if (dep_n) {
        adgi_state_bytes(v, ADGI_STATE_DEP_N, &b);
        CK(cudaMemcpy(v->dep_n, dep_n, b, cudaMemcpyHostToDevice));
    }
    return ADGI_OK;
}

int adgi_trace_closest(adgi_volume v, const float* o, const float* d, int32_t n, float tmin, float tmax, float* t_out,
                       int32_t* tri_out)
{
    if (!v || n < 0 || (n > 0 && (!o || !d || !t_out || !tri_out))) return fail(ADGI_ERR_INVALID_ARG, "bad arguments");
    if (!v->has_scene) return fail(ADGI_ERR_NO_SCENE, "no scene");
    {
        int rc = ensure_bvh(v, v->stream);
        if (rc) return rc;
    }
    SceneDev S = scene_view(v);
    CK(launch_trace_list(S, o, d, n, tmin, tmax, t_out, tri_out, v->stream));
    return ADGI_OK;
}

int adgi_count_traversal(adgi_volume v, const adgi_frame* f, uint64_t* counts)
{
    if (!v || !f || !counts) return fail(ADGI_ERR_INVALID_ARG, "NULL argument");
    if (!v->has_scene) return fail(ADGI_ERR_NO_SCENE, "no scene");
    if (f->n_lights < 0 || f->n_lights > kMaxLights || (f->n_lights > 0 && !f->lights))
        return fail(ADGI_ERR_INVALID_ARG, "bad light list");
    cudaStream_t s = v->stream;
    float Rsave[9];
    std::memcpy(Rsave, v->R, sizeof(Rsave));
    int64_t le = v->last_even;
    // the last update's pair state: the frame after an even frame saw it
    if ((f->frame & 1u) == 1u && v->last_even == (int64_t)f->frame) v->last_even = (int64_t)f->frame - 1;
    FrameDev fd;
    fd.F = frame_const(v, f);
    v->last_even = le;
    std::memcpy(v->R, Rsave, sizeof(Rsave));
    fd.L.n = f->n_lights;
    for (int i = 0; i < f->n_lights; ++i) {
        fd.L.l[i].kind = f->lights[i].kind;
        for (int k = 0; k < 3; ++k) {
            fd.L.l[i].v[k] = f->lights[i].pos_or_dir[k];
            fd.L.l[i].rgb[k] = f->lights[i].rgb[k];
        }
    }
    unsigned long long* d = nullptr;
    size_t dummy = 0;
    if (dalloc(&d, 12, &dummy) != cudaSuccess) return fail(ADGI_ERR_OOM, "counter buffer");
    cudaError_t e = cudaMemsetAsync(d, 0, 96, s);
    if (e == cudaSuccess) e = launch_set_frame(v->fdev, fd, s);
    if (e == cudaSuccess)
        e = v->desc.sampler == 1 ? launch_count(v->V, v->fdev, scene_view(v), v->off, v->sf, 2 * v->mh_B, d, s, v->mh_smp_g)
                                 : launch_count(v->V, v->fdev, scene_view(v), v->off, v->sf, v->R_main, d, s);
    unsigned long long h[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 96, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ADGI_ERR_CUDA, std::string("count: ") + cudaGetErrorString(e));
    for (int i = 0; i < 12; ++i) counts[i] = h[i];
    return ADGI_OK;
}

int adgi_build_bvh(const float* verts, int32_t nv, const int32_t* idx, int32_t nt, float eps, void* nodes_out,
                   void* tris_out, void* cuda_stream)
{
    if (nv < 0 || nt < 0 || (nt > 0 && (nv <= 0 || !verts || !idx || !nodes_out || !tris_out)) || !(eps >= 0.0f))
        return fail(ADGI_ERR_INVALID_ARG, "bad arguments");
    if (nt == 0) return ADGI_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BvhBufs B;
    size_t sb = carve_bvh_scratch(nullptr, nt, B);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, sb, s);
    if (e != cudaSuccess) return fail(ADGI_ERR_OOM, std::string("scratch: ") + cudaGetErrorString(e));
    carve_bvh_scratch(scratch, nt, B);
    B.tri_v = (float4*)tris_out;
    B.nodes = (BNode*)nodes_out;
    int root = -1;
    e = cudaMemsetAsync(B.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = build_lbvh(B, verts, idx, nv, nt, eps, B.err, s, &root, nullptr);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ADGI_ERR_CUDA, std::string("build: ") + cudaGetErrorString(e));
    if (herr & kErrIndex) return fail(ADGI_ERR_INVALID_ARG, "triangle index outside [0, n_verts)");
    if (herr) return fail(ADGI_ERR_CUDA, "device anomaly flags set: " + std::to_string(herr));
    return ADGI_OK;
}

int adgi_allocate_rays(const uint32_t* W, int32_t P, int32_t avg, int32_t rmin, int32_t rmax, uint32_t* n_out,
                       uint32_t* off_out, void* cuda_stream)
{
    if (!W || !n_out || !off_out || P <= 0) return fail(ADGI_ERR_INVALID_ARG, "bad arguments");
    int m0 = rmin > 8 ? rmin : 8;
    if (avg < m0 || avg > rmax || rmax > 4096 || (int64_t)P * avg >= ((int64_t)1 << 31))
        return fail(ADGI_ERR_INVALID_ARG, "budget cannot be met");
    CK(launch_allocate(W, P, avg, m0, rmax, n_out, off_out, (cudaStream_t)cuda_stream));
    return ADGI_OK;
}

}  // extern "C"
