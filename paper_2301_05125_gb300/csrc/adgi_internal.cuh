// adgi_internal.cuh -- device data layout and inline device code shared by the
// library's kernels (sm_103a).  Nothing here is shared with the CPU oracle.
//
// Exactness: every floating-point step whose result becomes an integer or a
// discrete decision (ray directions, the watertight hit test, shadow
// visibility, the lit test, the quantised heuristics, texel binning) is
// written with the *_rn intrinsics, which are never fused or reordered, so it
// reproduces IEEE single precision bit for bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "../../include/adgi.h"

namespace adgi {

constexpr int kPilots = 8;
constexpr int kMaxLights = 64;
constexpr uint32_t kMiss = 0xFFFFFFFFu;
constexpr uint32_t kBackBit = 0x80000000u;

// ----------------------------------------------------------------- device data
struct Light {
    int kind;
    float v[3];
    float rgb[3];
};

// BVH node: the boxes of both children (so one fetch decides both) and the
// child references; a child >= 0 is an internal node, < 0 is ~(triangle slot).
struct __align__(16) BNode {
    float4 a;  // c0.lo.xyz, c0.hi.x
    float4 b;  // c0.hi.yz, c1.lo.xy
    float4 c;  // c1.lo.z, c1.hi.xyz
    int4 d;    // left, right, -, -
};

// The scene: a static part (quality BVH, built once) and a moving part
// (linear BVH, rebuilt when vertices move), in one node array and one
// triangle array.  The static part's ns triangles occupy slots [0, ns) and
// its internal nodes [0, ns-1); the moving part's triangles follow at slot
// ns and its nodes at node max(ns-1, 0), with child references relocated
// to these global indices, so a traversal needs no per-part pointers.  Hits
// are ranked over both by (t, original triangle index).
constexpr int kWideEmpty = (int)0x80000000;  // an unused child slot of a 4-wide node
constexpr int kWide4Stack = 160;             // entries of the 4-wide traversal stack (>= the binary one's)

struct SceneDev {
    const float4* w4;       // 4-wide tree of the static part (7 float4 a node), or null: the binary tree
    const BNode* nodes;     // internal nodes of both parts
    const float4* tri_v;    // both parts' triangles in BVH order, .w of v0 = original index
    int root[2];            // root node of each part's tree (-1: fewer than two triangles)
    int leaf[2];            // slot of a part's only triangle (-1: none, or a tree)
    int max_iter;           // traversal step limit (a correct tree needs fewer node visits)
    int n_tris;
    int n_verts;
    const float4* tri_orig; // [n_tris*3] vertices in original order (shading normal)
    const float* albedo;    // [n_tris*3]
    int* err;               // anomaly flags (kErr*), 0 when all is well
};

constexpr int kErrTraversal = 1;  // a traversal exceeded max_iter
constexpr int kErrRayRange = 2;   // a probe's ray range exceeded the buffers
constexpr int kErrBvh = 4;        // the bottom-up box pass exceeded its depth bound
constexpr int kErrIndex = 8;      // a triangle referenced a vertex outside the array

struct FrameConst {
    uint64_t pilot_key;     // sm(sm(seed) ^ pair)
    float R[9];             // main-ray rotation
    float sky[3];
    int n_lights;
    int even;               // first frame of a pair: pilots are blended
    int pair_valid;         // the previous frame was the first of this pair
    int has_camera;
    float cam[3];
    float cam_k;
    uint64_t mh_key;        // Metropolis counters of this frame: sm(sm(seed ^ 'METRO') ^ frame)
    uint64_t dyn_key;       // the dynamic chains' counters: sm(sm(seed ^ 'DYNAM') ^ frame)
    int has_clip;           // clip volumes from clip[] (with has_camera)
    float clip[16];         // row-major view-projection
};

struct VolConst {
    float origin[3], spacing[3];
    int dims[3];
    int P;
    int n_irr, n_dep, Ti, Td;
    float tmin;             // (float)(1e-4 * s)
    float depth_max;
    float qv_scale;         // (float)(256 / s)
    float qc_scale;         // (float)(64 / s)
    float var_min;          // (float)(1e-6 * s^2): the Chebyshev minimum variance
    float var_rel;          // optional further floor var_rel * mu2 (0: none)
    float hyst;
    int theta;
    int m0, rays_max, rays_avg;
    int fp16;               // atlas storage: 0 FP32, 1 FP16 (RN), 2 FP16 (SR), 3 packed 32-bit codes
    const float* ctab;      // packed code values: [512] 9-bit, [256] 8-bit, [8192] 13-bit mean, [8192] 13-bit square
    float s_f;              // (float) cage diagonal: the packed visibility normaliser
    uint32_t R_main;        // main-ray buffer length
    int* err;               // anomaly flags (kErr*)
    int dyn;                // dynamic chains on (Metropolis mode with dyn_ratio > 0)
    float hyst_dyn;         // hysteresis of the dynamic rays' batch step
    const uint8_t* cls;     // [P] clip volume of this frame: 2 V_in, 1 V_out - V_in, 0 outside
    int p_lo, p_hi;         // probes this launch works on: [0, P), or one rank's slab of a split update
};

// This frame's dynamic rays (dynamic chains over virtual proxies), grouped
// by probe: probe p sends, for every octant o whose proxy cell is traced,
// one ray through the centre of each irradiance texel listed for o.
struct DynRays {
    const uint32_t* off;      // [P+1] first dynamic ray of each probe; off[P] = rays this frame
    const uint8_t* incl;      // [Pp*8] 1: the cell (proxy, octant) is traced
    const int* ntex;          // [8] texels whose centre lies in each octant
    const int* tex_t;         // [8][n_irr^2] their tile indices
    const float4* tex_dir;    // [8][n_irr^2] their centre directions
    int dp[3];                // proxy grid
};

// ----------------------------------------------------------------- exact FP32
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float dot3x(float ax, float ay, float az, float bx, float by, float bz)
{
    return fa(fa(fm(ax, bx), fm(ay, by)), fm(az, bz));
}

__host__ __device__ __forceinline__ uint64_t splitmix(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// probe position (FP32): origin + spacing * index
__device__ __forceinline__ float3 probe_pos(const VolConst& V, int p)
{
    int ix = p % V.dims[0];
    int iy = (p / V.dims[0]) % V.dims[1];
    int iz = p / (V.dims[0] * V.dims[1]);
    return make_float3(fa(V.origin[0], fm(V.spacing[0], (float)ix)), fa(V.origin[1], fm(V.spacing[1], (float)iy)),
                       fa(V.origin[2], fm(V.spacing[2], (float)iz)));
}

// q_c of probe p (Eq. cameraD): 1023 within cam_k of the camera, else the
// LUT bin of width s/64 at the distance beyond cam_k; 1023 without a camera
__device__ __forceinline__ uint32_t qc_of_probe(const VolConst& V, const FrameConst& F,
                                                const uint16_t* __restrict__ lut_c, int p)
{
    if (!F.has_camera) return 1023u;
    float3 pp = probe_pos(V, p);
    float dx = fs(pp.x, F.cam[0]), dy = fs(pp.y, F.cam[1]), dz = fs(pp.z, F.cam[2]);
    float dist = fsq(dot3x(dx, dy, dz, dx, dy, dz));
    if (dist < F.cam_k) return 1023u;
    float q = fm(fs(dist, F.cam_k), V.qc_scale);
    uint32_t i = q < 4095.0f ? (uint32_t)floorf(q) : 4095u;
    return __ldg(lut_c + i);
}

// Pilot direction of (probe, octant) for the frame pair encoded in key:
// a uniform point of the octant's simplex from a 64-bit hash, normalised.
__device__ __forceinline__ float3 pilot_dir(uint64_t key, uint32_t probe, int o)
{
    uint64_t h = splitmix(key ^ ((uint64_t)probe * 8u + (uint64_t)o));
    const float k24 = 5.9604644775390625e-08f;
    float u1 = fm(__uint2float_rn((uint32_t)(h >> 40)), k24);
    float u2 = fm(__uint2float_rn((uint32_t)((h >> 16) & 0xFFFFFFu)), k24);
    if (fa(u1, u2) > 1.0f) {
        float a = fs(1.0f, u2), b = fs(1.0f, u1);
        u1 = a;
        u2 = b;
    }
    float x = u1, y = u2, z = fs(fs(1.0f, u1), u2);
    if (o & 1) x = -x;
    if (o & 2) y = -y;
    if (o & 4) z = -z;
    float l = fsq(dot3x(x, y, z, x, y, z));
    return make_float3(fd(x, l), fd(y, l), fd(z, l));
}

__device__ __forceinline__ float3 rotate(const float* R, float4 s)
{
    return make_float3(fa(fa(fm(R[0], s.x), fm(R[1], s.y)), fm(R[2], s.z)),
                       fa(fa(fm(R[3], s.x), fm(R[4], s.y)), fm(R[5], s.z)),
                       fa(fa(fm(R[6], s.x), fm(R[7], s.y)), fm(R[8], s.z)));
}

// ----------------------------------------------------------------- octahedral
__device__ __forceinline__ float sgnf(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ float2 oct_encode_x(float3 w)
{
    float l1 = fa(fa(fabsf(w.x), fabsf(w.y)), fabsf(w.z));
    float px = fd(w.x, l1), py = fd(w.y, l1);
    if (w.z < 0.0f) {
        float qx = fm(fs(1.0f, fabsf(py)), sgnf(px));
        float qy = fm(fs(1.0f, fabsf(px)), sgnf(py));
        px = qx;
        py = qy;
    }
    return make_float2(px, py);
}

// unit direction of octahedral coordinates (ux, uy), exact FP32
__device__ __forceinline__ float3 oct_decode_x(float ux, float uy)
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

// direction through the centre of interior texel (cx, cy) of an n x n
// octahedral grid: u = (c + 1/2)/n * 2 - 1 per axis, FP32 in that order
__device__ __forceinline__ float3 texel_centre_dir(int cx, int cy, int n)
{
    const float fn = (float)n;
    return oct_decode_x(fs(fm(fd(fa((float)cx, 0.5f), fn), 2.0f), 1.0f), fs(fm(fd(fa((float)cy, 0.5f), fn), 2.0f), 1.0f));
}

// nearest interior texel, as row*(n+2)+col with both in 1..n
__device__ __forceinline__ int texel_of(float2 p, int n)
{
    float fn = (float)n;
    int cx = (int)floorf(fm(fm(fa(p.x, 1.0f), 0.5f), fn));
    int cy = (int)floorf(fm(fm(fa(p.y, 1.0f), 0.5f), fn));
    cx = min(max(cx, 0), n - 1);
    cy = min(max(cy, 0), n - 1);
    return (cy + 1) * (n + 2) + (cx + 1);
}

// ----------------------------------------------------------------- watertight
struct WRay {
    float ox, oy, oz;
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ float comp(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ WRay wray(float3 o, float3 d)
{
    WRay r;
    r.ox = o.x;
    r.oy = o.y;
    r.oz = o.z;
    int kz = 0;
    float m = fabsf(d.x);
    if (fabsf(d.y) > m) {
        kz = 1;
        m = fabsf(d.y);
    }
    if (fabsf(d.z) > m) kz = 2;
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    float dz = comp(d.x, d.y, d.z, kz);
    if (dz < 0.0f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    r.Sx = fd(comp(d.x, d.y, d.z, kx), dz);
    r.Sy = fd(comp(d.x, d.y, d.z, ky), dz);
    r.Sz = fd(1.0f, dz);
    return r;
}

// Woop-Benthin-Wald watertight test.  Returns true when the ray's line crosses
// the triangle, with t and det; det > 0 is a front-face hit.
__device__ __forceinline__ bool wtri(const WRay& r, float4 A4, float4 B4, float4 C4, float& t, float& det)
{
    float ax = fs(A4.x, r.ox), ay = fs(A4.y, r.oy), az = fs(A4.z, r.oz);
    float bx = fs(B4.x, r.ox), by = fs(B4.y, r.oy), bz = fs(B4.z, r.oz);
    float cx = fs(C4.x, r.ox), cy = fs(C4.y, r.oy), cz = fs(C4.z, r.oz);
    float akz = comp(ax, ay, az, r.kz), bkz = comp(bx, by, bz, r.kz), ckz = comp(cx, cy, cz, r.kz);
    float Ax = fs(comp(ax, ay, az, r.kx), fm(r.Sx, akz));
    float Ay = fs(comp(ax, ay, az, r.ky), fm(r.Sy, akz));
    float Bx = fs(comp(bx, by, bz, r.kx), fm(r.Sx, bkz));
    float By = fs(comp(bx, by, bz, r.ky), fm(r.Sy, bkz));
    float Cx = fs(comp(cx, cy, cz, r.kx), fm(r.Sx, ckz));
    float Cy = fs(comp(cx, cy, cz, r.ky), fm(r.Sy, ckz));
    float U = fs(fm(Cx, By), fm(Cy, Bx));
    float V = fs(fm(Ax, Cy), fm(Ay, Cx));
    float W = fs(fm(Bx, Ay), fm(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = __double2float_rn(__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx)));
        V = __double2float_rn(__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx)));
        W = __double2float_rn(__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax)));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    det = fa(fa(U, V), W);
    if (det == 0.0f) return false;
    float Az = fm(r.Sz, akz), Bz = fm(r.Sz, bkz), Cz = fm(r.Sz, ckz);
    float T = fa(fa(fm(U, Az), fm(V, Bz)), fm(W, Cz));
    t = fd(T, det);
    return true;
}

// Conservative slab test of one box against [0, lim]; NaNs (0 * inf) drop out
// of fminf/fmaxf, which keeps the test conservative.
__device__ __forceinline__ bool slab(float lox, float loy, float loz, float hix, float hiy, float hiz, float3 o,
                                     float3 inv, float lim, float& tnear)
{
    float tx0 = (lox - o.x) * inv.x, tx1 = (hix - o.x) * inv.x;
    float ty0 = (loy - o.y) * inv.y, ty1 = (hiy - o.y) * inv.y;
    float tz0 = (loz - o.z) * inv.z, tz1 = (hiz - o.z) * inv.z;
    float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), lim));
    tnear = tn;
    return tn <= tf;
}

constexpr float kBoxSlack = 1.0001f;  // pruning slack on the best t (conservative)
// LBVH depth is at most 95 (63 key bits + 32 index bits); a PLOC tree can be
// deeper, so its builder checks the depth against kMaxDepth.  The near-first
// traversal stack holds at most one pending entry per level.
constexpr int kMaxDepth = 96;
constexpr int kStack = kMaxDepth;
static_assert(kWide4Stack >= kStack, "one stack array serves both traversals");

// A load of data that an earlier phase of the same launch may have written.
// The ordinary kernels take the read-only (non-coherent) path; the
// persistent batched tick (tick.cu), whose phases follow one another inside
// one launch, takes a plain coherent load, which its grid barriers order.
template <bool kLive, typename T>
__device__ __forceinline__ T ldl(const T* p)
{
    if constexpr (kLive)
        return *p;
    else
        return __ldg(p);
}

// Traversal of the two-part scene as one flat loop over one stack of
// global node indices.  The loop has no early exit, so the lanes of a warp
// reconverge every iteration.

// One traversal in flight.  Closest hit: t in (tmin, tmax], ranked by
// (t, original index) -- a strict order, so the result does not depend on
// the traversal order.  Any hit: t in (tmin, tmax), stops at the first.
// The state is scalars only, so it can live in registers; the node stack is
// a separate local array.
struct Trav {
    WRay wr;
    float3 o, inv, oi;      // oi = o * inv: slab tests as one FMA per plane
    float tmin, tmax, lim;  // lim: box pruning bound
    float t_best, best_det;
    int best_orig;
    bool found;
    int sp, iter;
    int next;  // the node to visit next (-1: take the stack top); saves a push and a pop per single-child step
};

// Conservative slab test of one box against [0, lim] with the plane
// distances as fma(plane, 1/d, -o/d): the rounding of o/d moves a plane by
// about 2^-24 |o|, far inside the boxes' enlargement (>= 1e-5 of the
// largest coordinate), so no box that the ray enters is culled.  NaNs
// (0 * inf) drop out of fminf/fmaxf, which keeps the test conservative.
__device__ __forceinline__ bool slab_fma(float lox, float loy, float loz, float hix, float hiy, float hiz, float3 inv,
                                         float3 oi, float lim, float& tnear)
{
    float tx0 = fmaf(lox, inv.x, -oi.x), tx1 = fmaf(hix, inv.x, -oi.x);
    float ty0 = fmaf(loy, inv.y, -oi.y), ty1 = fmaf(hiy, inv.y, -oi.y);
    float tz0 = fmaf(loz, inv.z, -oi.z), tz1 = fmaf(hiz, inv.z, -oi.z);
    float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), lim));
    tnear = tn;
    return tn <= tf;
}

// the triangle at slot `slot` of the BVH-ordered array (kLive: it may have
// been written earlier in the same launch, see ldl)
template <bool kLive = false>
__device__ __forceinline__ void trav_tri(Trav& T, const float4* tri_v, int slot, bool any, uint32_t* ntri)
{
    if (ntri) ++*ntri;
    const float4* tv = tri_v + 3 * (size_t)slot;
    float4 A = ldl<kLive>(tv), Bv = ldl<kLive>(tv + 1), C = ldl<kLive>(tv + 2);
    float tt, det;
    if (!wtri(T.wr, A, Bv, C, tt, det) || !(tt > T.tmin)) return;
    if (any) {
        if (tt < T.tmax) T.found = true;
        return;
    }
    const int orig = __float_as_int(A.w);
    const bool better = T.found ? (tt < T.t_best || (tt == T.t_best && orig < T.best_orig)) : (tt <= T.tmax);
    if (better) {
        T.found = true;
        T.t_best = tt;
        T.best_orig = orig;
        T.best_det = det;
    }
}

// set up a traversal; single-triangle parts are tested here, trees pushed
// (the static part's only when it has no 4-wide tree: that one is walked
// by trav4 beforehand).  kLive: the moving part may have been rebuilt
// earlier in the same launch (its nodes and triangles are read with ldl).
template <bool kLive = false>
__device__ __forceinline__ void trav_init(Trav& T, int* stack, const SceneDev& S, float3 o, float3 d, float tmin,
                                          float tmax, bool any, uint32_t* ntri = nullptr)
{
    T.wr = wray(o, d);
    T.o = o;
    // The box test uses 1/d with components below 1e-20 in magnitude raised
    // to +-1e-20: a zero component would make o * inv infinite and the FMA
    // slab form inf - inf = NaN, rejecting every box (axis-aligned rays: an
    // axis-aligned sun, texel-centre directions on the octahedral diamond).
    // The raised component moves the ray by 1e-20 t along that axis, far
    // below the boxes' enlargement, so the test stays conservative; the
    // triangle test keeps the exact direction.
    const float kTiny = 1e-20f;
    const float dx = fabsf(d.x) < kTiny ? copysignf(kTiny, d.x) : d.x;
    const float dy = fabsf(d.y) < kTiny ? copysignf(kTiny, d.y) : d.y;
    const float dz = fabsf(d.z) < kTiny ? copysignf(kTiny, d.z) : d.z;
    T.inv = make_float3(1.0f / dx, 1.0f / dy, 1.0f / dz);
    T.oi = make_float3(o.x * T.inv.x, o.y * T.inv.y, o.z * T.inv.z);
    T.next = -1;
    T.tmin = tmin;
    T.tmax = tmax;
    T.lim = any ? (isinf(tmax) ? tmax : tmax * kBoxSlack) : tmax * kBoxSlack;
    T.t_best = tmax;
    T.best_det = 0.0f;
    T.best_orig = 0x7FFFFFFF;
    T.found = false;
    T.sp = 0;
    T.iter = 0;
    if (S.n_tris == 0) return;
    for (int pi = 1; pi >= (S.w4 ? 1 : 0); --pi) {
        const int root = pi ? S.root[1] : S.root[0], leaf = pi ? S.leaf[1] : S.leaf[0];
        if (root >= 0)
            stack[T.sp++] = root;
        else if (leaf >= 0)
            trav_tri<kLive>(T, S.tri_v, leaf, any, ntri);
    }
    if (any && T.found) T.sp = 0;
}

// one node visit; false once the traversal is over
template <bool kLive = false>
__device__ __forceinline__ bool trav_step(Trav& T, int* stack, const SceneDev& S, bool any,
                                          uint32_t* nbox = nullptr, uint32_t* ntri = nullptr)
{
    if (T.next < 0 && T.sp <= 0) return false;
    if (++T.iter > S.max_iter) {
        atomicOr(S.err, kErrTraversal);
        T.sp = 0;
        T.next = -1;
        return false;
    }
    if (nbox) *nbox += 2;
    const int e = T.next >= 0 ? T.next : stack[--T.sp];
    T.next = -1;
    const BNode* nd = S.nodes + e;
    float4 a = ldl<kLive>(&nd->a), b = ldl<kLive>(&nd->b), c = ldl<kLive>(&nd->c);
    int4 ch = ldl<kLive>(&nd->d);
    const float lim = any ? T.lim : T.t_best * kBoxSlack;
    float t0, t1;
    const bool h0 = slab_fma(a.x, a.y, a.z, a.w, b.x, b.y, T.inv, T.oi, lim, t0);
    const bool h1 = slab_fma(b.z, b.w, c.x, c.y, c.z, c.w, T.inv, T.oi, lim, t1);
    if (h0 && ch.x < 0) trav_tri<kLive>(T, S.tri_v, ~ch.x, any, ntri);
    if (h1 && ch.y < 0) trav_tri<kLive>(T, S.tri_v, ~ch.y, any, ntri);
    const bool i0 = h0 && ch.x >= 0, i1 = h1 && ch.y >= 0;
    if (i0 && i1) {  // the near child next, the far one on the stack
        const bool first0 = t0 <= t1;
        if (T.sp < kStack + 2) {
            stack[T.sp++] = first0 ? ch.y : ch.x;
            T.next = first0 ? ch.x : ch.y;
        } else {
            atomicOr(S.err, kErrTraversal);  // cannot happen: depths are bounded by the builders
        }
    } else if (i0 || i1) {
        T.next = i0 ? ch.x : ch.y;
    }
    if (any && T.found) {  // a blocker ends a shadow ray
        T.sp = 0;
        T.next = -1;
    }
    return T.next >= 0 || T.sp > 0;
}

__device__ __forceinline__ uint32_t trav_hit(const Trav& T)
{
    return T.found ? ((uint32_t)T.best_orig | (T.best_det < 0.0f ? kBackBit : 0u)) : kMiss;
}

// One visit of the static part's 4-wide tree: node `node`, the traversal's
// stack and its depth sp, the ray's direction signs (sx, sy, sz: 0 positive,
// 1 negative).  Returns the node to visit next, or -1 once the static part is
// done (an any-hit traversal: also when it found a blocker).
__device__ __forceinline__ int trav4_visit(Trav& T, int* stack, int& sp, int node, const SceneDev& S, bool any,
                                           int sx, int sy, int sz, uint32_t* nbox, uint32_t* ntri)
{
    if (++T.iter > S.max_iter) {
        atomicOr(S.err, kErrTraversal);
        return -1;
    }
    if (nbox) *nbox += 4;
    const float4* N = S.w4 + 7 * (size_t)node;
    const float4 nx = __ldg(N + sx), fx = __ldg(N + 1 - sx);
    const float4 ny = __ldg(N + 2 + sy), fy = __ldg(N + 3 - sy);
    const float4 nz = __ldg(N + 4 + sz), fz = __ldg(N + 5 - sz);
    const int4 rf = __ldg(reinterpret_cast<const int4*>(N + 6));
    const float lim = any ? T.lim : T.t_best * kBoxSlack;
    float key[4];
    int ref[4] = {rf.x, rf.y, rf.z, rf.w};
    const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, fxs[4] = {fx.x, fx.y, fx.z, fx.w};
    const float nys[4] = {ny.x, ny.y, ny.z, ny.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w};
    const float nzs[4] = {nz.x, nz.y, nz.z, nz.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
    const float inf = __int_as_float(0x7F800000);
    uint32_t leaves = 0;  // closest hit: hit leaf children, tested below in one loop (one divergent region, not four)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float tn = fmaxf(fmaxf(fmaf(nxs[k], T.inv.x, -T.oi.x), fmaf(nys[k], T.inv.y, -T.oi.y)),
                               fmaxf(fmaf(nzs[k], T.inv.z, -T.oi.z), 0.0f));
        const float tf = fminf(fminf(fmaf(fxs[k], T.inv.x, -T.oi.x), fmaf(fys[k], T.inv.y, -T.oi.y)),
                               fminf(fmaf(fzs[k], T.inv.z, -T.oi.z), lim));
        const bool hit = tn <= tf;
        if (any) {  // any hit: each hit leaf at once (a blocker ends the search below)
            if (hit && ref[k] < 0) trav_tri(T, S.tri_v, ~ref[k], true, ntri);
        } else if (hit && ref[k] < 0) {
            leaves |= 1u << k;
        }
        key[k] = hit && ref[k] >= 0 ? tn : inf;
    }
    if (any && T.found) return -1;
    while (leaves) {
        const int k = __ffs(leaves) - 1;
        leaves &= leaves - 1u;
        const int r = k == 0 ? rf.x : k == 1 ? rf.y : k == 2 ? rf.z : rf.w;
        trav_tri(T, S.tri_v, ~r, any, ntri);
        if (any && T.found) return -1;
    }
    // the hit internal children nearest first: a sorting network on (key, ref)
    // (for an any-hit traversal only the nearest is put first)
#define ADGI_CSWAP(i, j)                                  \
    if (key[j] < key[i]) {                                \
        const float tk = key[i];                          \
        key[i] = key[j];                                  \
        key[j] = tk;                                      \
        const int tr = ref[i];                            \
        ref[i] = ref[j];                                  \
        ref[j] = tr;                                      \
    }
    ADGI_CSWAP(0, 1)
    ADGI_CSWAP(2, 3)
    ADGI_CSWAP(0, 2)
    if (!any) {  // any hit: the nearest first is enough (measured: the full order costs more than it saves)
        ADGI_CSWAP(1, 3)
        ADGI_CSWAP(1, 2)
    }
#undef ADGI_CSWAP
    if (key[0] < inf) {
        if (sp + 3 > kWide4Stack) {  // the builder bounds the depth, so this cannot happen
            atomicOr(S.err, kErrTraversal);
            return -1;
        }
        if (key[3] < inf) stack[sp++] = ref[3];
        if (key[2] < inf) stack[sp++] = ref[2];
        if (key[1] < inf) stack[sp++] = ref[1];
        return ref[0];
    }
    return sp == 0 ? -1 : stack[--sp];
}

// One visit of the static part's 4-wide tree without its leaf tests: node
// `node`, the traversal's stack and its depth sp, the ray's direction signs
// (sx, sy, sz: 0 positive, 1 negative).  The hit leaf children go to
// *leaves (bit k: slot k); of the hit internal children the first in the
// order below is returned and the others pushed.  Returns -1 when no
// internal child is hit and the stack is empty.
__device__ __forceinline__ int trav4_inner(Trav& T, int* stack, int& sp, int node, const SceneDev& S, bool any,
                                           int sx, int sy, int sz, uint32_t* nbox, uint32_t& leaves)
{
    leaves = 0;
    if (++T.iter > S.max_iter) {
        atomicOr(S.err, kErrTraversal);
        sp = 0;
        return -1;
    }
    if (nbox) *nbox += 4;
    const float4* N = S.w4 + 7 * (size_t)node;
    const float4 nx = __ldg(N + sx), fx = __ldg(N + 1 - sx);
    const float4 ny = __ldg(N + 2 + sy), fy = __ldg(N + 3 - sy);
    const float4 nz = __ldg(N + 4 + sz), fz = __ldg(N + 5 - sz);
    const int4 rf = __ldg(reinterpret_cast<const int4*>(N + 6));
    const float lim = any ? T.lim : T.t_best * kBoxSlack;
    float key[4];
    int ref[4] = {rf.x, rf.y, rf.z, rf.w};
    const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, fxs[4] = {fx.x, fx.y, fx.z, fx.w};
    const float nys[4] = {ny.x, ny.y, ny.z, ny.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w};
    const float nzs[4] = {nz.x, nz.y, nz.z, nz.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
    const float inf = __int_as_float(0x7F800000);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float tn = fmaxf(fmaxf(fmaf(nxs[k], T.inv.x, -T.oi.x), fmaf(nys[k], T.inv.y, -T.oi.y)),
                               fmaxf(fmaf(nzs[k], T.inv.z, -T.oi.z), 0.0f));
        const float tf = fminf(fminf(fmaf(fxs[k], T.inv.x, -T.oi.x), fmaf(fys[k], T.inv.y, -T.oi.y)),
                               fminf(fmaf(fzs[k], T.inv.z, -T.oi.z), lim));
        const bool hit = tn <= tf;
        if (hit && ref[k] < 0) leaves |= 1u << k;
        key[k] = hit && ref[k] >= 0 ? (any ? tn - tf : tn) : inf;
    }
    // the hit internal children in order: a sorting network on (key, ref).
    // Closest hit: nearest entry first.  Any hit: only the first place is
    // sorted, and it goes to the child holding the longest stretch of the
    // ray (tn - tf least), the likeliest to hold a blocker (measured: shadow
    // rays 2-7 % faster than nearest first).
#define ADGI_CSWAP(i, j)                                  \
    if (key[j] < key[i]) {                                \
        const float tk = key[i];                          \
        key[i] = key[j];                                  \
        key[j] = tk;                                      \
        const int tr = ref[i];                            \
        ref[i] = ref[j];                                  \
        ref[j] = tr;                                      \
    }
    ADGI_CSWAP(0, 1)
    ADGI_CSWAP(2, 3)
    ADGI_CSWAP(0, 2)
    if (!any) {  // any hit: the nearest first is enough (measured: the full order costs more than it saves)
        ADGI_CSWAP(1, 3)
        ADGI_CSWAP(1, 2)
    }
#undef ADGI_CSWAP
    if (key[0] < inf) {
        if (sp + 3 > kWide4Stack) {  // the builder bounds the depth, so this cannot happen
            atomicOr(S.err, kErrTraversal);
            sp = 0;
            return -1;
        }
        if (key[3] < inf) stack[sp++] = ref[3];
        if (key[2] < inf) stack[sp++] = ref[2];
        if (key[1] < inf) stack[sp++] = ref[1];
        return ref[0];
    }
    return sp == 0 ? -1 : stack[--sp];
}

// The triangles of the hit leaf children `leaves` of wide node `node`
// (an any-hit traversal stops at the first blocker).
__device__ __forceinline__ void trav4_leaves(Trav& T, int node, uint32_t leaves, const SceneDev& S, bool any,
                                             uint32_t* ntri)
{
    const int4 rf = __ldg(reinterpret_cast<const int4*>(S.w4 + 7 * (size_t)node + 6));
    while (leaves) {
        const int k = __ffs(leaves) - 1;
        leaves &= leaves - 1u;
        const int r = k == 0 ? rf.x : k == 1 ? rf.y : k == 2 ? rf.z : rf.w;
        trav_tri(T, S.tri_v, ~r, any, ntri);
        if (any && T.found) return;
    }
}

// The static part's 4-wide tree (T set up by trav_init): from the root, each
// visit tests the four child boxes with the near / far planes of each axis
// read by the sign of the ray direction (so an entry distance is a max and an
// exit distance a min of three FMAs) and continues with the nearest hit
// internal child; the other hit internal children are pushed, farthest
// first (closest hit).
//   Closest hit: the hit leaf children's triangles are tested in the visit
//   that finds them, so the pruning bound shrinks at once.
//   Any hit (shadow rays): the triangle tests are postponed.  A lane keeps
//   the leaf sets of up to two visits and goes on visiting inner nodes
//   until every lane of the warp still traversing has one (or is done);
//   then they test their leaves together, so the 55-operation triangle
//   tests run with most lanes busy; the traversal stops at the first
//   blocker.  (Measured on both benchmark scenes: shadow rays 4-12 %
//   faster this way; the nearest-hit trace 20-30 % slower, since its pruning
//   bound waits for the postponed tests.)
// The pruning bound and the (t, index) ranking are those of trav_step, and
// the hit is the least (t, index) over the same candidates, so it is the
// same in any visiting order.
__device__ __forceinline__ void trav4(Trav& T, int* stack, const SceneDev& S, bool any, uint32_t* nbox = nullptr,
                                      uint32_t* ntri = nullptr)
{
    const int sx = T.inv.x >= 0.0f ? 0 : 1, sy = T.inv.y >= 0.0f ? 0 : 1, sz = T.inv.z >= 0.0f ? 0 : 1;
    int node = 0, sp = 0;
    if (!any) {
        while (node >= 0) node = trav4_visit(T, stack, sp, node, S, false, sx, sy, sz, nbox, ntri);
        return;
    }
    int p0 = 0, p1 = 0;        // wide nodes with pending leaf tests
    uint32_t m0 = 0, m1 = 0;   // and their hit leaf children
    for (;;) {
        while (node >= 0 && m1 == 0) {
            const int cur = node;
            uint32_t lm;
            node = trav4_inner(T, stack, sp, cur, S, true, sx, sy, sz, nbox, lm);
            if (lm) {
                if (m0 == 0) {
                    p0 = cur;
                    m0 = lm;
                } else {
                    p1 = cur;
                    m1 = lm;
                }
            }
            if (__all_sync(__activemask(), m0 != 0 || node < 0)) break;
        }
        if (m0 == 0) return;  // no leaves pending and (the loop ended) no node left
        trav4_leaves(T, p0, m0, S, true, ntri);
        m0 = 0;
        if (m1 && !T.found) trav4_leaves(T, p1, m1, S, true, ntri);
        m1 = 0;
        if (T.found) return;
    }
}

// nearest hit with t in (tmin, tmax] (one thread, one ray); kLive: as for
// trav_init
template <bool kLive = false>
__device__ __forceinline__ void trace_closest(const SceneDev& S, float3 o, float3 d, float tmin, float tmax,
                                              float& t_best, uint32_t& hit_best, uint32_t* nbox = nullptr,
                                              uint32_t* ntri = nullptr)
{
    Trav T;
    int stack[kWide4Stack + 2];  // the moving part's root sits below the 4-wide traversal's entries
    trav_init<kLive>(T, stack, S, o, d, tmin, tmax, false, ntri);
    if (S.w4) {  // the static part's 4-wide tree first, then the moving part's binary tree
        const int sp = T.sp;  // the moving part's root, pushed by trav_init, waits below
        int* st = stack + sp;
        trav4(T, st, S, false, nbox, ntri);
        T.sp = sp;
    }
    while (trav_step<kLive>(T, stack, S, false, nbox, ntri)) {
    }
    t_best = T.t_best;
    hit_best = trav_hit(T);
}

// any hit with t in (tlo, thi): shadow visibility (one thread, one ray)
template <bool kLive = false>
__device__ __forceinline__ bool trace_any(const SceneDev& S, float3 o, float3 d, float tlo, float thi,
                                          uint32_t* nbox = nullptr, uint32_t* ntri = nullptr)
{
    Trav T;
    int stack[kWide4Stack + 2];  // the moving part's root sits below the 4-wide traversal's entries
    trav_init<kLive>(T, stack, S, o, d, tlo, thi, true, ntri);
    if (S.w4 && !T.found) {
        const int sp = T.sp;
        trav4(T, stack + sp, S, true, nbox, ntri);
        T.sp = T.found ? 0 : sp;
    }
    while (trav_step<kLive>(T, stack, S, true, nbox, ntri)) {
    }
    return T.found;
}


// ----------------------------------------------------------------- atlas access
// Packed texels (the paper's 32-bit codecs): irradiance R bits 0-8, G 9-17,
// B 18-25, count 26-31; visibility mean bits 0-12, mean square 13-25, count
// 26-31, both in units of the cage diagonal s.  A code stands for the value
// of its table entry.
constexpr int kCt9 = 0, kCt8 = 512, kCtM = 768, kCtQ = 768 + 8192, kCtSize = 768 + 2 * 8192;

__device__ __forceinline__ float4 irr_unpack(const float* __restrict__ ct, uint32_t c)
{
    return make_float4(__ldg(ct + kCt9 + (c & 511u)), __ldg(ct + kCt9 + ((c >> 9) & 511u)),
                       __ldg(ct + kCt8 + ((c >> 18) & 255u)), (float)(c >> 26));
}

// {mean, variance} in world units from a packed visibility texel
__device__ __forceinline__ float2 dep_unpack(const float* __restrict__ ct, float s, uint32_t c)
{
    const float m = __ldg(ct + kCtM + (c & 8191u)) * s;
    const float q = __ldg(ct + kCtQ + ((c >> 13) & 8191u)) * (s * s);
    return make_float2(m, fmaxf(q - m * m, 0.0f));
}

__device__ __forceinline__ float4 irr_load(const VolConst& V, const void* irr, size_t idx)
{
    if (V.fp16 == 3) return irr_unpack(V.ctab, reinterpret_cast<const uint32_t*>(irr)[idx]);
    if (V.fp16) {
        const __half2* h = reinterpret_cast<const __half2*>(irr) + 2 * idx;
        float2 a = __half22float2(h[0]), b = __half22float2(h[1]);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    return reinterpret_cast<const float4*>(irr)[idx];
}

// depth texel as {mean, variance}
__device__ __forceinline__ float2 dep_load(const VolConst& V, const void* dep, size_t idx)
{
    if (V.fp16 == 3) return dep_unpack(V.ctab, V.s_f, reinterpret_cast<const uint32_t*>(dep)[idx]);
    if (V.fp16) return __half22float2(reinterpret_cast<const __half2*>(dep)[idx]);
    return reinterpret_cast<const float2*>(dep)[idx];
}

// bilinear sample of a padded tile at direction w (octahedral coordinates)
template <int CH>
__device__ __forceinline__ void tile_bilinear(const VolConst& V, const void* base, size_t tile_off, int T, int n,
                                              float2 p, float* out)
{
    float fx = (1.0f + (p.x + 1.0f) * 0.5f * (float)n) - 0.5f;
    float fy = (1.0f + (p.y + 1.0f) * 0.5f * (float)n) - 0.5f;
    int x0 = min(max((int)floorf(fx), 0), n);
    int y0 = min(max((int)floorf(fy), 0), n);
    float ax = fminf(fmaxf(fx - (float)x0, 0.0f), 1.0f);
    float ay = fminf(fmaxf(fy - (float)y0, 0.0f), 1.0f);
    size_t i00 = tile_off + (size_t)(y0 * T + x0);
    if (CH == 3) {
        float4 v00 = irr_load(V, base, i00), v01 = irr_load(V, base, i00 + 1);
        float4 v10 = irr_load(V, base, i00 + T), v11 = irr_load(V, base, i00 + T + 1);
        out[0] = (1.0f - ay) * ((1.0f - ax) * v00.x + ax * v01.x) + ay * ((1.0f - ax) * v10.x + ax * v11.x);
        out[1] = (1.0f - ay) * ((1.0f - ax) * v00.y + ax * v01.y) + ay * ((1.0f - ax) * v10.y + ax * v11.y);
        out[2] = (1.0f - ay) * ((1.0f - ax) * v00.z + ax * v01.z) + ay * ((1.0f - ax) * v10.z + ax * v11.z);
    } else {
        float2 v00 = dep_load(V, base, i00), v01 = dep_load(V, base, i00 + 1);
        float2 v10 = dep_load(V, base, i00 + T), v11 = dep_load(V, base, i00 + T + 1);
        out[0] = (1.0f - ay) * ((1.0f - ax) * v00.x + ax * v01.x) + ay * ((1.0f - ax) * v10.x + ax * v11.x);
        out[1] = (1.0f - ay) * ((1.0f - ax) * v00.y + ax * v01.y) + ay * ((1.0f - ax) * v10.y + ax * v11.y);
    }
}

// FP32 coordinate of probe plane j along axis k (where the probes sit)
__device__ __forceinline__ float pcoord(const VolConst& V, int k, int j)
{
    return fa(V.origin[k], fm(V.spacing[k], (float)j));
}

// (o - pb) + t*d with the rounding errors of the product and the sum carried
// (FMA residual + two-sum), so the result has a small *relative* error even
// when the hit point sits next to a probe plane far from the world origin.
__device__ __forceinline__ float local_offset(float o, float pb, float t, float d)
{
    float a = fs(o, pb);  // probe planes: exact difference
    float p = fm(t, d);
    float e = __fmaf_rn(t, d, -p);
    float s = fa(a, p);
    float bb = fs(s, a);
    float err = fa(fs(a, fs(s, bb)), fs(p, bb));
    return fa(s, fa(e, err));
}

// Bilinear filter of depth texels {mean, variance}: filtered mean, and the
// filtered variance sum w var_t + sum w (mean_t - mean)^2 -- the variance of
// the filtered {d, d^2} moments, formed without cancellation.
__device__ __forceinline__ void filter_moments(float w00, float w01, float w10, float w11, float2 v00, float2 v01,
                                               float2 v10, float2 v11, float* mom)
{
    float mu = w00 * v00.x + w01 * v01.x + w10 * v10.x + w11 * v11.x;
    float d00 = v00.x - mu, d01 = v01.x - mu, d10 = v10.x - mu, d11 = v11.x - mu;
    float var = w00 * (v00.y + d00 * d00) + w01 * (v01.y + d01 * d01) + w10 * (v10.y + d10 * d10) +
                w11 * (v11.y + d11 * d11);
    mom[0] = mu;
    mom[1] = var;
}

// Depth moments of probe tile p at the direction of dv (not normalised:
// the octahedral map is scale invariant), FP32 bilinear fractions.
__device__ __forceinline__ void depth_moments(const VolConst& V, const void* dep, size_t tile, float dx, float dy,
                                              float dz, float* mom, float* cond)
{
    // the fractions only weight a bilinear lookup: fast division (2 ulp)
    float l1 = fabsf(dx) + fabsf(dy) + fabsf(dz);
    float px = __fdividef(dx, l1), py = __fdividef(dy, l1);
    if (dz < 0.0f) {
        float qx = (1.0f - fabsf(py)) * sgnf(px);
        float qy = (1.0f - fabsf(px)) * sgnf(py);
        px = qx;
        py = qy;
    }
    const int n = V.n_dep, T = V.Td;
    float fx = (1.0f + (px + 1.0f) * 0.5f * (float)n) - 0.5f;
    float fy = (1.0f + (py + 1.0f) * 0.5f * (float)n) - 0.5f;
    int x0 = min(max((int)floorf(fx), 0), n);
    int y0 = min(max((int)floorf(fy), 0), n);
    float ax = fminf(fmaxf(fx - (float)x0, 0.0f), 1.0f);
    float ay = fminf(fmaxf(fy - (float)y0, 0.0f), 1.0f);
    size_t i00 = tile + (size_t)(y0 * T + x0);
    float2 v00 = dep_load(V, dep, i00), v01 = dep_load(V, dep, i00 + 1);
    float2 v10 = dep_load(V, dep, i00 + T), v11 = dep_load(V, dep, i00 + T + 1);
    float w00 = (1.f - ax) * (1.f - ay), w01 = ax * (1.f - ay), w10 = (1.f - ax) * ay, w11 = ax * ay;
    filter_moments(w00, w01, w10, w11, v00, v01, v10, v11, mom);
    // conditioning of the filtered variance against the fractions: what a
    // texel adds to the variance per unit weight, over the floored variance
    float var = fmaxf(mom[1], fmaxf(V.var_rel * (mom[1] + mom[0] * mom[0]), V.var_min));
    float d00 = v00.x - mom[0], d01 = v01.x - mom[0], d10 = v10.x - mom[0], d11 = v11.x - mom[0];
    float s2 = fmaxf(fmaxf(v00.y + d00 * d00, v01.y + d01 * d01), fmaxf(v10.y + d10 * d10, v11.y + d11 * d11));
    *cond = __fdividef(s2, var);
}

// ---------------------------------------------------------------- double-float
// Unevaluated sums hi + lo of two floats (Dekker / Knuth error-free
// transformations), for the few quantities that need ~2^-44 relative precision.
struct df {
    float h, l;
};
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = fa(a, b);
    float bb = fs(s, a);
    return {s, fa(fs(a, fs(s, bb)), fs(b, bb))};
}
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = fa(a, b);
    return {s, fs(b, fs(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = fm(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, fa(s.l, fa(a.l, b.l)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_abs(df a) { return a.h < 0.0f ? df_neg(a) : a; }
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    df p = two_prod(a.h, b);
    return fast_two_sum(p.h, __fmaf_rn(a.l, b, p.l));
}
__device__ __forceinline__ df df_div(df a, df b)
{
    float q1 = fd(a.h, b.h);
    df r = df_add(a, df_neg(df_mul_f(b, q1)));
    float q2 = fd(r.h, b.h);
    return fast_two_sum(q1, q2);
}
// (o - p) + t*d as a double-float: exact inputs, error ~2^-44 relative
__device__ __forceinline__ df df_offset(float o, float p, float t, float d)
{
    return df_add(two_sum(o, -p), two_prod(t, d));
}

// The depth lookup with the direction and the bilinear fractions in
// double-float (for footprints where FP32 fractions would perturb the filtered
// variance): the offset is rebuilt exactly from (o, p, t, d).
static __device__ __noinline__ void depth_moments_precise(const VolConst& V, const void* dep, size_t tile,
                                                          const float* o, const float* p, float t, const float* d,
                                                          float* mom)
{
    df dx = df_offset(o[0], p[0], t, d[0]);
    df dy = df_offset(o[1], p[1], t, d[1]);
    df dz = df_offset(o[2], p[2], t, d[2]);
    df l1 = df_add(df_add(df_abs(dx), df_abs(dy)), df_abs(dz));
    df px = df_div(dx, l1), py = df_div(dy, l1);
    if (dz.h < 0.0f) {
        const df one = {1.0f, 0.0f};
        df qx = df_add(one, df_neg(df_abs(py)));
        df qy = df_add(one, df_neg(df_abs(px)));
        px = px.h >= 0.0f ? qx : df_neg(qx);
        py = py.h >= 0.0f ? qy : df_neg(qy);
    }
    const int n = V.n_dep, T = V.Td;
    const float hn = 0.5f * (float)n;
    df fx = df_add(df_mul_f(px, hn), {hn + 0.5f, 0.0f});
    df fy = df_add(df_mul_f(py, hn), {hn + 0.5f, 0.0f});
    float x0f = floorf(fx.h), y0f = floorf(fy.h);
    if (fx.h == x0f && fx.l < 0.0f) x0f -= 1.0f;
    if (fy.h == y0f && fy.l < 0.0f) y0f -= 1.0f;
    int x0 = min(max((int)x0f, 0), n);
    int y0 = min(max((int)y0f, 0), n);
    float ax = fminf(fmaxf(fa(fs(fx.h, (float)x0), fx.l), 0.0f), 1.0f);
    float ay = fminf(fmaxf(fa(fs(fy.h, (float)y0), fy.l), 0.0f), 1.0f);
    float bx = fminf(fmaxf(fs(fs((float)(x0 + 1), fx.h), fx.l), 0.0f), 1.0f);
    float by = fminf(fmaxf(fs(fs((float)(y0 + 1), fy.h), fy.l), 0.0f), 1.0f);
    size_t i00 = tile + (size_t)(y0 * T + x0);
    float2 v00 = dep_load(V, dep, i00), v01 = dep_load(V, dep, i00 + 1);
    float2 v10 = dep_load(V, dep, i00 + T), v11 = dep_load(V, dep, i00 + T + 1);
    float w00 = bx * by, w01 = ax * by, w10 = bx * ay, w11 = ax * ay;
    filter_moments(w00, w01, w10, w11, v00, v01, v10, v11, mom);
}

// 8-probe trilinear x Chebyshev irradiance query at x = o + t*d (the public
// query passes t = 0).  The cage is the one whose FP32 probe planes bracket x;
// offsets from each probe are formed without rounding x to world coordinates.
__device__ __forceinline__ float3 query_irr_at(const VolConst& V, const void* irr, const void* dep, float3 o, float t,
                                               float3 d, float3 nrm)
{
    float os[3] = {o.x, o.y, o.z}, ds[3] = {d.x, d.y, d.z};
    int b[3];
    float al[3], be[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float g = floorf((fa(os[k], fm(t, ds[k])) - V.origin[k]) / V.spacing[k]);
        int bi = (int)fminf(fmaxf(g, 0.0f), (float)(V.dims[k] - 2));
        float l = local_offset(os[k], pcoord(V, k, bi), t, ds[k]);
        if (bi > 0 && l < 0.0f) {
            --bi;
            l = local_offset(os[k], pcoord(V, k, bi), t, ds[k]);
        } else if (bi < V.dims[k] - 2) {
            float l2 = local_offset(os[k], pcoord(V, k, bi + 1), t, ds[k]);
            if (l2 >= 0.0f) {
                ++bi;
                l = l2;
            }
        }
        b[k] = bi;
        // both layer weights from the double-float offset l to plane b: alpha
        // = l/s and 1 - alpha = (s - l)/s, each with full relative precision
        // (1 - alpha formed in FP32 loses it next to the upper plane, where a
        // nearly empty lower-layer weight can still decide the normalised sum)
        const df lf = df_offset(os[k], pcoord(V, k, bi), t, ds[k]);
        const df rf = df_add({V.spacing[k], 0.0f}, df_neg(lf));
        al[k] = fminf(fmaxf(fa(lf.h, lf.l) / V.spacing[k], 0.0f), 1.0f);
        be[k] = fminf(fmaxf(fa(rf.h, rf.l) / V.spacing[k], 0.0f), 1.0f);
    }
    float nl = sqrtf(nrm.x * nrm.x + nrm.y * nrm.y + nrm.z * nrm.z);
    float3 nd = nl > 0.0f ? make_float3(nrm.x / nl, nrm.y / nl, nrm.z / nl) : make_float3(0.f, 0.f, 1.f);
    float2 pn = oct_encode_x(nd);
    float sum[3] = {0.f, 0.f, 0.f}, sumt[3] = {0.f, 0.f, 0.f}, sw = 0.f;
    const size_t ti2 = (size_t)V.Ti * V.Ti, td2 = (size_t)V.Td * V.Td;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        int o0 = c & 1, o1 = (c >> 1) & 1, o2 = (c >> 2) & 1;
        float wt = (o0 ? al[0] : be[0]) * (o1 ? al[1] : be[1]) * (o2 ? al[2] : be[2]);
        int ix = b[0] + o0, iy = b[1] + o1, iz = b[2] + o2;
        int p = ix + V.dims[0] * (iy + V.dims[1] * iz);
        float px = pcoord(V, 0, ix), py = pcoord(V, 1, iy), pz = pcoord(V, 2, iz);
        float dx = local_offset(os[0], px, t, ds[0]);
        float dy = local_offset(os[1], py, t, ds[1]);
        float dz = local_offset(os[2], pz, t, ds[2]);
        float dist = sqrtf(dx * dx + dy * dy + dz * dz);
        float mom[2] = {0.f, 0.f};
        if (dist > 0.f) {
            float cond;
            depth_moments(V, dep, (size_t)p * td2, dx, dy, dz, mom, &cond);
            if (cond > 128.0f) {  // FP32 fractions would move the variance by > ~6e-5
                const float pc[3] = {px, py, pz};
                depth_moments_precise(V, dep, (size_t)p * td2, os, pc, t, ds, mom);
            }
        }
        float wc = 1.f;
        if (dist > mom[0]) {
            // one-sided Chebyshev bound with the minimum variance 1e-6 s^2,
            // or var_rel * mu2 (mu2 = var + mean^2) where a volume asks for it
            float var = fmaxf(mom[1], fmaxf(V.var_rel * (mom[1] + mom[0] * mom[0]), V.var_min));
            float dd = dist - mom[0];
            wc = __fdividef(var, var + dd * dd);
        }
        float E[3];
        tile_bilinear<3>(V, irr, (size_t)p * ti2, V.Ti, V.n_irr, pn, E);
        float w = wt * wc;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sum[k] += w * E[k];
            sumt[k] += wt * E[k];
        }
        sw += w;
    }
    if (sw >= 1e-12f) return make_float3(sum[0] / sw, sum[1] / sw, sum[2] / sw);
    return make_float3(sumt[0], sumt[1], sumt[2]);
}

__device__ __forceinline__ float3 query_irr(const VolConst& V, const void* irr, const void* dep, float3 x, float3 nrm)
{
    return query_irr_at(V, irr, dep, x, 0.0f, make_float3(0.f, 0.f, 0.f), nrm);
}

__device__ __forceinline__ float3 query_irr_hit(const VolConst& V, const void* irr, const void* dep, float3 o, float t,
                                                float3 d, float3 nrm)
{
    return query_irr_at(V, irr, dep, o, t, d, nrm);
}

// Dynamic ray r: its probe p, irradiance texel t (tile index) and direction
// d; false beyond this frame's rays.
__device__ __forceinline__ bool dyn_ray_of(const VolConst& V, const DynRays& D, uint32_t r, int& p, int& t, float3& d)
{
    if (r >= __ldg(D.off + V.P)) return false;
    int lo = 0, hi = V.P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(D.off + mid) <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    p = lo;
    uint32_t j = r - __ldg(D.off + p);
    const int ix = p % V.dims[0], iy = (p / V.dims[0]) % V.dims[1], iz = p / (V.dims[0] * V.dims[1]);
    const int q = ix / 3 + D.dp[0] * (iy / 3 + D.dp[1] * (iz / 3));
    const int nn = V.n_irr * V.n_irr;
    for (int o = 0; o < 8; ++o) {
        if (!__ldg(D.incl + q * 8 + o)) continue;
        const uint32_t n = (uint32_t)__ldg(D.ntex + o);
        if (j < n) {
            t = __ldg(D.tex_t + o * nn + (int)j);
            const float4 w = __ldg(D.tex_dir + o * nn + (int)j);
            d = make_float3(w.x, w.y, w.z);
            return true;
        }
        j -= n;
    }
    return false;
}

}  // namespace adgi
