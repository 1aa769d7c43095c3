/*
 * adgi_oracle.c -- plain, slow CPU oracle of the ADGI per-frame probe update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no source, header, table or constant generator with the CUDA library; the
 * two are written independently from the paper (Datta, Goli, Zhang,
 * "Adaptive Dynamic Global Illumination", arXiv 2301.05125) and from the
 * published methods cited below.
 *
 * Two numeric paths:
 *   - an FP32 path for every floating-point computation whose result is turned
 *     into an integer or a discrete decision (pilot and main ray directions,
 *     ray/triangle hits and the hit index, shadow-ray visibility, the
 *     quantised heuristics q_v / q_r / q_c, texel binning).  It uses only
 *     IEEE +, -, *, / and sqrt, in the stated order, compiled with
 *     -ffp-contract=off, so any correct IEEE implementation gets the same bits;
 *   - an FP64 path for everything that is compared with a tolerance
 *     (shading, multi-bounce query, blending, the irradiance query).
 *
 * Section map (paper):
 *   Sec. 4.1 Eq. cameraD        -> q_c (camera distance heuristic f_c)
 *   Sec. 4.1 Eq. ProbeVis       -> q_v (f_v = exp(-2t/s), t = trace(p,-w))
 *   Sec. 4.1 "Incoming radiance"-> q_r (f_r = min(r,beta)/beta, beta = 5)
 *   Sec. 4.1 Eq. tempGradVis, tempGradIrr, Tr, spatial convolution
 *                               -> temporal trigger + 5x5x5 x octant sum
 *   Sec. 4.2 Eq. priorDynamic   -> f_d = f_c f_v (f_dv + mu f_dr), mu = 2
 *   Sec. 4.4 "Improving construction efficiency" -> pilot rays, AABB pattern
 *   Sec. 3.5 Alg. ApproxAlgo + Sec. 4.7 Alg. MovingAvgUpdate -> nearest-texel
 *                                 moving average with hysteresis
 *   Sec. 3.6 (MCMC analysis)    -> texel stores the texel-average of g
 *   Sec. 3.1 (DDGI background)  -> octahedral tiles with borders, 8-probe
 *                                 trilinear x Chebyshev query
 *   Sec. 3.4 (fixed sample budget) -> integer allocation under a fixed total
 * Published methods restated here: SplitMix64 (Steele, Lea, Flood, OOPSLA
 * 2014); watertight ray/triangle intersection (Woop, Benthin, Wald, JCGT
 * 2(1), 2013); spherical Fibonacci point sets (Keinert et al., 2015);
 * binned-SAH BVH construction (Wald, 2007).
 *
 * Parity pins: every exported function is pinned by a -m "not gpu" test in
 * tests/test_oracle_*.py against closed forms, invariants or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* SplitMix64 output function (Steele et al. 2014): one generator step from  */
/* state x.  Counter-based use: every random number the method draws is      */
/* sm(sm(sm(seed) ^ a) ^ b) for its own counters a, b.                        */
/* ------------------------------------------------------------------------ */
EXPORT uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t hash3(uint64_t a, uint64_t b, uint64_t c)
{
    return orc_splitmix64(orc_splitmix64(orc_splitmix64(a) ^ b) ^ c);
}

/* ------------------------------------------------------------------------ */
/* Pilot ray directions (Sec. 4.4): one stratified random direction per      */
/* octant; the directions depend on the frame pair floor(t/2) only, so the   */
/* two frames of a pair (A A B B C C ...) trace identical rays.              */
/* Octant index o = [x<0] | [y<0]<<1 | [z<0]<<2.                              */
/* ------------------------------------------------------------------------ */
EXPORT void orc_pilot_dir(uint64_t seed, uint64_t frame, uint32_t probe, int octant, float out[3])
{
    uint64_t pair = frame >> 1;
    uint64_t h = hash3(seed, pair, (uint64_t)probe * 8u + (uint64_t)octant);
    const float two_m24 = 5.9604644775390625e-08f; /* 2^-24 */
    float u1 = (float)(uint32_t)(h >> 40) * two_m24;
    float u2 = (float)(uint32_t)((h >> 16) & 0xFFFFFFu) * two_m24;
    if (u1 + u2 > 1.0f) {
        float a = 1.0f - u2;
        float b = 1.0f - u1;
        u1 = a;
        u2 = b;
    }
    float v[3];
    v[0] = u1;
    v[1] = u2;
    v[2] = (1.0f - u1) - u2;
    if (octant & 1) v[0] = -v[0];
    if (octant & 2) v[1] = -v[1];
    if (octant & 4) v[2] = -v[2];
    float len2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    float len = sqrtf(len2);
    out[0] = v[0] / len;
    out[1] = v[1] / len;
    out[2] = v[2] / len;
}

/* ------------------------------------------------------------------------ */
/* Per-frame random rotation of the main-ray pattern (DDGI's rotated         */
/* spiral, Sec. 3.1).  A uniform unit quaternion by rejection from the 4-ball */
/* in FP64, converted to a matrix in FP64 and rounded to FP32.               */
/* ------------------------------------------------------------------------ */
EXPORT void orc_frame_rotation(uint64_t seed, uint64_t frame, float R[9])
{
    const double two_m53 = 1.1102230246251565e-16; /* 2^-53 */
    double q[4] = {1.0, 0.0, 0.0, 0.0};
    for (uint64_t attempt = 0; attempt < 1000; ++attempt) {
        double c[4];
        for (int k = 0; k < 4; ++k) {
            uint64_t h = hash3(seed ^ 0x524F54ull, frame, attempt * 4u + (uint64_t)k);
            c[k] = ((double)(h >> 11) * two_m53) * 2.0 - 1.0;
        }
        double n2 = ((c[0] * c[0] + c[1] * c[1]) + c[2] * c[2]) + c[3] * c[3];
        if (n2 > 1e-6 && n2 <= 1.0) {
            double n = sqrt(n2);
            for (int k = 0; k < 4; ++k) q[k] = c[k] / n;
            break;
        }
    }
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double m[9];
    m[0] = 1.0 - 2.0 * (y * y + z * z);
    m[1] = 2.0 * (x * y - w * z);
    m[2] = 2.0 * (x * z + w * y);
    m[3] = 2.0 * (x * y + w * z);
    m[4] = 1.0 - 2.0 * (x * x + z * z);
    m[5] = 2.0 * (y * z - w * x);
    m[6] = 2.0 * (x * z - w * y);
    m[7] = 2.0 * (y * z + w * x);
    m[8] = 1.0 - 2.0 * (x * x + y * y);
    for (int k = 0; k < 9; ++k) R[k] = (float)m[k];
}

/* ------------------------------------------------------------------------ */
/* Spherical Fibonacci point set with m points (Keinert et al. 2015):        */
/* z_i = 1 - (2i+1)/m, phi_i = i * golden angle, golden angle = pi(3-sqrt5). */
/* cos/sin(phi_i) by the exact complex recurrence from cos/sin(golden angle) */
/* so only IEEE basic operations are used.  FP64, rounded to FP32.          */
/* ------------------------------------------------------------------------ */
static const double GA_COS = -0.7373688780783197;
static const double GA_SIN = 0.6754902942615238;

EXPORT void orc_sf_points(int m, float* out /* m*3 */)
{
    double c = 1.0, s = 0.0;
    for (int i = 0; i < m; ++i) {
        double z = 1.0 - (2.0 * (double)i + 1.0) / (double)m;
        double r2 = 1.0 - z * z;
        double r = r2 > 0.0 ? sqrt(r2) : 0.0;
        out[3 * i + 0] = (float)(r * c);
        out[3 * i + 1] = (float)(r * s);
        out[3 * i + 2] = (float)z;
        double cn = c * GA_COS - s * GA_SIN;
        double sn = s * GA_COS + c * GA_SIN;
        c = cn;
        s = sn;
    }
}

/* FP32 rotation d = R * v in a fixed order (row-major R). */
static void rotate_f32(const float R[9], const float v[3], float d[3])
{
    d[0] = (R[0] * v[0] + R[1] * v[1]) + R[2] * v[2];
    d[1] = (R[3] * v[0] + R[4] * v[1]) + R[5] * v[2];
    d[2] = (R[6] * v[0] + R[7] * v[1]) + R[8] * v[2];
}

/* ------------------------------------------------------------------------ */
/* Octahedral map (Sec. 3.1; DDGI's spherical mapping of probe texels).      */
/* encode: p = w.xy / (|x|+|y|+|z|); lower hemisphere folded outward with    */
/* sign(0) = +1.  decode is its inverse.  FP64 versions for the reference     */
/* path, an FP32 version for texel binning (a discrete decision).            */
/* ------------------------------------------------------------------------ */
static double sgn_d(double v) { return v >= 0.0 ? 1.0 : -1.0; }
static float sgn_f(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

EXPORT void orc_oct_encode(const double w[3], double p[2])
{
    double l1 = (fabs(w[0]) + fabs(w[1])) + fabs(w[2]);
    double px = w[0] / l1, py = w[1] / l1;
    if (w[2] < 0.0) {
        double qx = (1.0 - fabs(py)) * sgn_d(px);
        double qy = (1.0 - fabs(px)) * sgn_d(py);
        px = qx;
        py = qy;
    }
    p[0] = px;
    p[1] = py;
}

EXPORT void orc_oct_decode(const double p[2], double w[3])
{
    double x = p[0], y = p[1];
    double z = (1.0 - fabs(x)) - fabs(y);
    if (z < 0.0) {
        double nx = (1.0 - fabs(y)) * sgn_d(x);
        double ny = (1.0 - fabs(x)) * sgn_d(y);
        x = nx;
        y = ny;
    }
    double n = sqrt((x * x + y * y) + z * z);
    w[0] = x / n;
    w[1] = y / n;
    w[2] = z / n;
}

static void oct_encode_f32(const float w[3], float p[2])
{
    float l1 = (fabsf(w[0]) + fabsf(w[1])) + fabsf(w[2]);
    float px = w[0] / l1, py = w[1] / l1;
    if (w[2] < 0.0f) {
        float qx = (1.0f - fabsf(py)) * sgn_f(px);
        float qy = (1.0f - fabsf(px)) * sgn_f(py);
        px = qx;
        py = qy;
    }
    p[0] = px;
    p[1] = py;
}

/* Nearest interior texel of direction w in a tile with interior n x n and a */
/* one-texel border (Alg. ApproxAlgo: a sample updates the closest entry).   */
/* Returns row*(n+2)+col with row from p.y and col from p.x, both in 1..n.   */
EXPORT int orc_texel_of_dir(const float w[3], int n)
{
    float p[2];
    oct_encode_f32(w, p);
    float fn = (float)n;
    int cx = (int)floorf(((p[0] + 1.0f) * 0.5f) * fn);
    int cy = (int)floorf(((p[1] + 1.0f) * 0.5f) * fn);
    if (cx < 0) cx = 0;
    if (cx > n - 1) cx = n - 1;
    if (cy < 0) cy = 0;
    if (cy > n - 1) cy = n - 1;
    return (cy + 1) * (n + 2) + (cx + 1);
}

/* ------------------------------------------------------------------------ */
/* Watertight ray/triangle intersection (Woop, Benthin, Wald 2013), FP32.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    float o[3], d[3];
    int kx, ky, kz;
    float Sx, Sy, Sz;
} wray;

static void wray_setup(wray* r, const float o[3], const float d[3])
{
    for (int k = 0; k < 3; ++k) {
        r->o[k] = o[k];
        r->d[k] = d[k];
    }
    int kz = 0;
    if (fabsf(d[1]) > fabsf(d[kz])) kz = 1;
    if (fabsf(d[2]) > fabsf(d[kz])) kz = 2;
    int kx = kz + 1;
    if (kx == 3) kx = 0;
    int ky = kx + 1;
    if (ky == 3) ky = 0;
    if (d[kz] < 0.0f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    r->kx = kx;
    r->ky = ky;
    r->kz = kz;
    r->Sx = d[kx] / d[kz];
    r->Sy = d[ky] / d[kz];
    r->Sz = 1.0f / d[kz];
}

/* Returns 1 and (t, det) when the ray's line crosses the triangle; the caller */
/* applies its own t interval.  det < 0 <=> the ray meets the back face      */
/* (geometric normal (B-A)x(C-A) points along the ray); pinned by a test.    */
static int wtri(const wray* r, const float* A, const float* B, const float* C, float* t_out, float* det_out)
{
    float a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = A[k] - r->o[k];
        b[k] = B[k] - r->o[k];
        c[k] = C[k] - r->o[k];
    }
    const int kx = r->kx, ky = r->ky, kz = r->kz;
    float Ax = a[kx] - r->Sx * a[kz];
    float Ay = a[ky] - r->Sy * a[kz];
    float Bx = b[kx] - r->Sx * b[kz];
    float By = b[ky] - r->Sy * b[kz];
    float Cx = c[kx] - r->Sx * c[kz];
    float Cy = c[ky] - r->Sy * c[kz];
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        double CxBy = (double)Cx * (double)By, CyBx = (double)Cy * (double)Bx;
        double AxCy = (double)Ax * (double)Cy, AyCx = (double)Ay * (double)Cx;
        double BxAy = (double)Bx * (double)Ay, ByAx = (double)By * (double)Ax;
        U = (float)(CxBy - CyBx);
        V = (float)(AxCy - AyCx);
        W = (float)(BxAy - ByAx);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;
    float det = (U + V) + W;
    if (det == 0.0f) return 0;
    float Az = r->Sz * a[kz];
    float Bz = r->Sz * b[kz];
    float Cz = r->Sz * c[kz];
    float T = (U * Az + V * Bz) + W * Cz;
    *t_out = T / det;
    *det_out = det;
    return 1;
}

EXPORT int orc_intersect_tri(const float o[3], const float d[3], const float A[3], const float B[3],
                             const float C[3], float* t_out, float* det_out)
{
    wray r;
    wray_setup(&r, o, d);
    return wtri(&r, A, B, C, t_out, det_out);
}

/* ------------------------------------------------------------------------ */
/* Scene + CPU BVH.  The BVH only accelerates: its answer must equal brute   */
/* force exactly (pinned), so its boxes are enlarged and its pruning slack.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
    int left, right; /* children; leaf when count > 0 */
    int first, count;
} bnode;

typedef struct {
    int nt;
    const float* V;   /* vertices xyz */
    const int* I;     /* triangle indices */
    bnode* nodes;
    int n_nodes;
    int* order;       /* triangle ids in leaf order */
    double eps;       /* absolute box enlargement */
} cbvh;

static void tri_bounds(const float* V, const int* I, int t, double lo[3], double hi[3])
{
    for (int k = 0; k < 3; ++k) {
        lo[k] = 1e300;
        hi[k] = -1e300;
    }
    for (int v = 0; v < 3; ++v) {
        const float* p = V + 3 * (size_t)I[3 * (size_t)t + v];
        for (int k = 0; k < 3; ++k) {
            if (p[k] < lo[k]) lo[k] = p[k];
            if (p[k] > hi[k]) hi[k] = p[k];
        }
    }
}

typedef struct {
    double lo[3], hi[3], c[3];
} tbox;

static double area_of(const double lo[3], const double hi[3])
{
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    if (dx < 0 || dy < 0 || dz < 0) return 0.0;
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

static int bvh_build_rec(cbvh* b, tbox* tb, int* ids, int first, int count, int* next)
{
    int me = (*next)++;
    bnode* n = &b->nodes[me];
    for (int k = 0; k < 3; ++k) {
        n->lo[k] = 1e300;
        n->hi[k] = -1e300;
    }
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int i = first; i < first + count; ++i) {
        tbox* t = &tb[ids[i]];
        for (int k = 0; k < 3; ++k) {
            if (t->lo[k] < n->lo[k]) n->lo[k] = t->lo[k];
            if (t->hi[k] > n->hi[k]) n->hi[k] = t->hi[k];
            if (t->c[k] < clo[k]) clo[k] = t->c[k];
            if (t->c[k] > chi[k]) chi[k] = t->c[k];
        }
    }
    for (int k = 0; k < 3; ++k) {
        n->lo[k] -= b->eps;
        n->hi[k] += b->eps;
    }
    if (count <= 4) {
        n->left = n->right = -1;
        n->first = first;
        n->count = count;
        return me;
    }
    /* binned SAH over centroids, 16 bins per axis */
    enum { NB = 16 };
    int best_axis = -1, best_split = -1;
    double best_cost = 1e300;
    for (int ax = 0; ax < 3; ++ax) {
        double ext = chi[ax] - clo[ax];
        if (!(ext > 0.0)) continue;
        int cnt[NB] = {0};
        double blo[NB][3], bhi[NB][3];
        for (int i = 0; i < NB; ++i)
            for (int k = 0; k < 3; ++k) {
                blo[i][k] = 1e300;
                bhi[i][k] = -1e300;
            }
        for (int i = first; i < first + count; ++i) {
            tbox* t = &tb[ids[i]];
            int bi = (int)((t->c[ax] - clo[ax]) / ext * NB);
            if (bi >= NB) bi = NB - 1;
            if (bi < 0) bi = 0;
            cnt[bi]++;
            for (int k = 0; k < 3; ++k) {
                if (t->lo[k] < blo[bi][k]) blo[bi][k] = t->lo[k];
                if (t->hi[k] > bhi[bi][k]) bhi[bi][k] = t->hi[k];
            }
        }
        for (int s = 1; s < NB; ++s) {
            double llo[3] = {1e300, 1e300, 1e300}, lhi[3] = {-1e300, -1e300, -1e300};
            double rlo[3] = {1e300, 1e300, 1e300}, rhi[3] = {-1e300, -1e300, -1e300};
            int lc = 0, rc = 0;
            for (int i = 0; i < NB; ++i) {
                double* lo = i < s ? llo : rlo;
                double* hi = i < s ? lhi : rhi;
                if (i < s)
                    lc += cnt[i];
                else
                    rc += cnt[i];
                for (int k = 0; k < 3; ++k) {
                    if (blo[i][k] < lo[k]) lo[k] = blo[i][k];
                    if (bhi[i][k] > hi[k]) hi[k] = bhi[i][k];
                }
            }
            if (lc == 0 || rc == 0) continue;
            double cost = area_of(llo, lhi) * lc + area_of(rlo, rhi) * rc;
            if (cost < best_cost) {
                best_cost = cost;
                best_axis = ax;
                best_split = s;
            }
        }
    }
    int mid;
    if (best_axis < 0) {
        mid = first + count / 2; /* all centroids equal: split by position */
    } else {
        double ext = chi[best_axis] - clo[best_axis];
        int i = first, j = first + count - 1;
        while (i <= j) {
            tbox* t = &tb[ids[i]];
            int bi = (int)((t->c[best_axis] - clo[best_axis]) / ext * NB);
            if (bi >= NB) bi = NB - 1;
            if (bi < 0) bi = 0;
            if (bi < best_split) {
                ++i;
            } else {
                int tmp = ids[i];
                ids[i] = ids[j];
                ids[j] = tmp;
                --j;
            }
        }
        mid = i;
        if (mid == first || mid == first + count) mid = first + count / 2;
    }
    n->count = 0;
    n->first = -1;
    int l = bvh_build_rec(b, tb, ids, first, mid - first, next);
    int r = bvh_build_rec(b, tb, ids, mid, first + count - mid, next);
    b->nodes[me].left = l;
    b->nodes[me].right = r;
    return me;
}

static void cbvh_free(cbvh* b)
{
    free(b->nodes);
    free(b->order);
    b->nodes = NULL;
    b->order = NULL;
    b->n_nodes = 0;
}

static int cbvh_build(cbvh* b, const float* V, int nv, const int* I, int nt)
{
    cbvh_free(b);
    b->nt = nt;
    b->V = V;
    b->I = I;
    if (nt == 0) return 0;
    tbox* tb = (tbox*)malloc(sizeof(tbox) * (size_t)nt);
    int* ids = (int*)malloc(sizeof(int) * (size_t)nt);
    if (!tb || !ids) {
        free(tb);
        free(ids);
        return -1;
    }
    double slo[3] = {1e300, 1e300, 1e300}, shi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < 3; ++k) {
            double x = V[3 * (size_t)v + k];
            if (x < slo[k]) slo[k] = x;
            if (x > shi[k]) shi[k] = x;
        }
    double ext = 0.0, mag = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (shi[k] - slo[k] > ext) ext = shi[k] - slo[k];
        if (fabs(slo[k]) > mag) mag = fabs(slo[k]);
        if (fabs(shi[k]) > mag) mag = fabs(shi[k]);
    }
    b->eps = 1e-5 * (ext > mag ? ext : mag) + 1e-30;
    for (int t = 0; t < nt; ++t) {
        tri_bounds(V, I, t, tb[t].lo, tb[t].hi);
        for (int k = 0; k < 3; ++k) tb[t].c[k] = 0.5 * (tb[t].lo[k] + tb[t].hi[k]);
        ids[t] = t;
    }
    b->nodes = (bnode*)malloc(sizeof(bnode) * (size_t)(2 * nt));
    if (!b->nodes) {
        free(tb);
        free(ids);
        return -1;
    }
    int next = 0;
    bvh_build_rec(b, tb, ids, 0, nt, &next);
    b->n_nodes = next;
    b->order = ids;
    free(tb);
    return 0;
}

/* slab test in FP64 against [0, tlim]; conservative by the box enlargement */
static int box_hit(const bnode* n, const float o[3], const float d[3], double tlim)
{
    double tn = 0.0, tf = tlim;
    for (int k = 0; k < 3; ++k) {
        double ok = o[k], dk = d[k];
        if (dk == 0.0) {
            if (ok < n->lo[k] || ok > n->hi[k]) return 0;
            continue;
        }
        double inv = 1.0 / dk;
        double t0 = (n->lo[k] - ok) * inv, t1 = (n->hi[k] - ok) * inv;
        if (t0 > t1) {
            double t = t0;
            t0 = t1;
            t1 = t;
        }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
        if (tn > tf) return 0;
    }
    return 1;
}

typedef struct {
    float t;
    int tri;
    float det;
} hitrec;

/* nearest hit with t in (tmin, tmax]; ties on t broken by the smaller index */
static hitrec closest_brute(const float* V, const int* I, int nt, const float o[3], const float d[3], float tmin,
                            float tmax)
{
    wray r;
    wray_setup(&r, o, d);
    hitrec h = {tmax, -1, 0.0f};
    for (int t = 0; t < nt; ++t) {
        float tt, det;
        const int* ix = I + 3 * (size_t)t;
        if (!wtri(&r, V + 3 * (size_t)ix[0], V + 3 * (size_t)ix[1], V + 3 * (size_t)ix[2], &tt, &det)) continue;
        if (!(tt > tmin)) continue;
        if (h.tri < 0 ? !(tt <= tmax) : !(tt < h.t)) continue;
        h.t = tt;
        h.tri = t;
        h.det = det;
    }
    return h;
}

static hitrec closest_bvh(const cbvh* b, const float o[3], const float d[3], float tmin, float tmax)
{
    hitrec h = {tmax, -1, 0.0f};
    if (b->nt == 0) return h;
    wray r;
    wray_setup(&r, o, d);
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode* n = &b->nodes[stack[--sp]];
        double lim = (double)h.t * (1.0 + 1e-4) + 1e-30;
        if (!box_hit(n, o, d, lim)) continue;
        if (n->count > 0) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int t = b->order[i];
                const int* ix = b->I + 3 * (size_t)t;
                float tt, det;
                if (!wtri(&r, b->V + 3 * (size_t)ix[0], b->V + 3 * (size_t)ix[1], b->V + 3 * (size_t)ix[2], &tt, &det))
                    continue;
                if (!(tt > tmin)) continue;
                int better;
                if (h.tri < 0)
                    better = tt <= tmax;
                else
                    better = tt < h.t || (tt == h.t && t < h.tri);
                if (!better) continue;
                h.t = tt;
                h.tri = t;
                h.det = det;
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    return h;
}

/* any hit with t strictly inside (tlo, thi) */
static int anyhit_brute(const float* V, const int* I, int nt, const float o[3], const float d[3], float tlo, float thi)
{
    wray r;
    wray_setup(&r, o, d);
    for (int t = 0; t < nt; ++t) {
        float tt, det;
        const int* ix = I + 3 * (size_t)t;
        if (!wtri(&r, V + 3 * (size_t)ix[0], V + 3 * (size_t)ix[1], V + 3 * (size_t)ix[2], &tt, &det)) continue;
        if (tt > tlo && tt < thi) return 1;
    }
    return 0;
}

static int anyhit_bvh(const cbvh* b, const float o[3], const float d[3], float tlo, float thi)
{
    if (b->nt == 0) return 0;
    wray r;
    wray_setup(&r, o, d);
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    double lim = (double)thi * (1.0 + 1e-4) + 1e-30;
    if (isinf(thi)) lim = 1e300;
    while (sp) {
        const bnode* n = &b->nodes[stack[--sp]];
        if (!box_hit(n, o, d, lim)) continue;
        if (n->count > 0) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int t = b->order[i];
                const int* ix = b->I + 3 * (size_t)t;
                float tt, det;
                if (!wtri(&r, b->V + 3 * (size_t)ix[0], b->V + 3 * (size_t)ix[1], b->V + 3 * (size_t)ix[2], &tt, &det))
                    continue;
                if (tt > tlo && tt < thi) return 1;
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    return 0;
}

/* Stand-alone tracing entry points (used by the intersection pins). */
EXPORT void orc_trace_closest(const float* V, int nv, const int* I, int nt, int n_rays, const float* O, const float* D,
                              float tmin, float tmax, int use_bvh, float* t_out, int* tri_out, float* det_out)
{
    cbvh b;
    memset(&b, 0, sizeof(b));
    if (use_bvh) cbvh_build(&b, V, nv, I, nt);
    for (int i = 0; i < n_rays; ++i) {
        hitrec h = use_bvh ? closest_bvh(&b, O + 3 * (size_t)i, D + 3 * (size_t)i, tmin, tmax)
                           : closest_brute(V, I, nt, O + 3 * (size_t)i, D + 3 * (size_t)i, tmin, tmax);
        t_out[i] = h.t;
        tri_out[i] = h.tri;
        if (det_out) det_out[i] = h.det;
    }
    cbvh_free(&b);
}

EXPORT void orc_trace_any(const float* V, int nv, const int* I, int nt, int n_rays, const float* O, const float* D,
                          float tlo, float thi, int use_bvh, uint8_t* out)
{
    cbvh b;
    memset(&b, 0, sizeof(b));
    if (use_bvh) cbvh_build(&b, V, nv, I, nt);
    for (int i = 0; i < n_rays; ++i)
        out[i] = (uint8_t)(use_bvh ? anyhit_bvh(&b, O + 3 * (size_t)i, D + 3 * (size_t)i, tlo, thi)
                                   : anyhit_brute(V, I, nt, O + 3 * (size_t)i, D + 3 * (size_t)i, tlo, thi));
    cbvh_free(&b);
}

/* ------------------------------------------------------------------------ */
/* Ray allocation under a fixed total budget (Sec. 3.4: the number of        */
/* samples per frame is an input, independent of the probe count).  The     */
/* paper draws the samples with Metropolis chains; this oracle follows the  */
/* deterministic reading: integer proportional shares of the extra budget   */
/* by the change weight W_p, with per-probe caps, then the remainder one by */
/* one in probe-index order.                                                */
/*   n_p = m0 + extra_p, m0 = max(rays_min, 8), sum n_p = rays_avg * P.      */
/*   off[p] = exclusive prefix of the main-ray counts n_p - 8.               */
/* Returns 0, or -1 when the budget cannot be met.                           */
/* ------------------------------------------------------------------------ */
#define ORC_ALLOC_MAX_ITERS 64

/* Allocation restricted by the clip volumes (cls: 2 V_in, 1 V_out only, 0
   outside; NULL: every probe in V_in).  Only V_in probes take adaptive
   rays: n = m0 + extra in V_in, 8 (the pilots) in V_out - V_in, 0 outside.
   The adaptive budget stays (avg - 8) P; beyond the V_in floors, E =
   (avg - 8) P - (m0 - 8) |V_in| is spread over V_in as below, capped at
   rmax - m0 per probe (what the caps cannot hold stays unspent; the pilots
   of culled probes are saved, not reassigned).  With every probe in V_in
   this is exactly the plain rule. */
EXPORT int orc_allocate_masked(const uint32_t* W, const uint8_t* cls, int P, int avg, int rmin, int rmax,
                               uint32_t* n_out, uint32_t* off_out)
{
    if (P <= 0) return -1;
    int m0 = rmin > 8 ? rmin : 8;
    if (avg < m0 || avg > rmax || m0 > rmax) return -1;
    uint64_t cap = (uint64_t)(rmax - m0);
    uint64_t Pin = 0;
    for (int p = 0; p < P; ++p) Pin += !cls || cls[p] == 2;
    uint64_t E = (uint64_t)(avg - 8) * (uint64_t)P - (uint64_t)(m0 - 8) * Pin;
    if (E > Pin * cap) E = Pin * cap;
    uint64_t* extra = (uint64_t*)calloc((size_t)P, sizeof(uint64_t));
    uint8_t* inU = (uint8_t*)calloc((size_t)P, 1);
    if (!extra || !inU) {
        free(extra);
        free(inU);
        return -1;
    }
#define IN_VIN(p) (!cls || cls[p] == 2)
    uint64_t S = 0;
    for (int p = 0; p < P; ++p)
        if (IN_VIN(p)) S += W[p];
    if (S == 0) {
        if (Pin > 0) { /* uniform over V_in, the remainder to the lowest ranks */
            uint64_t q = E / Pin, r = E % Pin, rank = 0;
            for (int p = 0; p < P; ++p)
                if (IN_VIN(p)) extra[p] = q + (rank++ < r ? 1u : 0u);
        }
    } else {
        uint64_t Erem = E;
        for (int p = 0; p < P; ++p) inU[p] = IN_VIN(p) && W[p] > 0 && cap > 0;
        for (int it = 0; it < ORC_ALLOC_MAX_ITERS; ++it) {
            uint64_t SU = 0;
            for (int p = 0; p < P; ++p)
                if (inU[p]) SU += W[p];
            if (SU == 0 || Erem == 0) break;
            uint64_t given = 0;
            for (int p = 0; p < P; ++p) {
                if (!inU[p]) continue;
                uint64_t share = Erem * (uint64_t)W[p] / SU;
                uint64_t room = cap - extra[p];
                uint64_t a = share < room ? share : room;
                extra[p] += a;
                given += a;
            }
            if (given == 0) break;
            Erem -= given;
            for (int p = 0; p < P; ++p)
                if (inU[p] && extra[p] == cap) inU[p] = 0;
        }
        /* remainder: one ray each, probe-index order, probes with W > 0 first */
        while (Erem > 0) {
            int anyA = 0;
            for (int p = 0; p < P; ++p)
                if (IN_VIN(p) && W[p] > 0 && extra[p] < cap) {
                    anyA = 1;
                    break;
                }
            for (int p = 0; p < P && Erem > 0; ++p) {
                int elig = IN_VIN(p) && extra[p] < cap && (anyA ? W[p] > 0 : 1);
                if (elig) {
                    extra[p] += 1;
                    Erem -= 1;
                }
            }
        }
    }
    uint32_t acc = 0;
    for (int p = 0; p < P; ++p) {
        int c = cls ? cls[p] : 2;
        n_out[p] = (uint32_t)((c == 2 ? (uint64_t)m0 : (c == 1 ? 8u : 0u)) + extra[p]);
        if (off_out) off_out[p] = acc;
        acc += n_out[p] > 8u ? n_out[p] - 8u : 0u;
    }
    if (off_out) off_out[P] = acc;
#undef IN_VIN
    free(extra);
    free(inU);
    return 0;
}

EXPORT int orc_allocate(const uint32_t* W, int P, int avg, int rmin, int rmax, uint32_t* n_out, uint32_t* off_out)
{
    return orc_allocate_masked(W, NULL, P, avg, rmin, rmax, n_out, off_out);
}

/* ------------------------------------------------------------------------ */
/* Packed 32-bit atlases (Sec. "Probe irradiance cache", "Probe visibility   */
/* cache", appendix "Probe compression").  A channel value v >= 0 is coded   */
/* as u = min(ln(gamma v + 1), beta) / beta quantised to b bits by rounding  */
/* down; decoding is (exp(beta u) - 1) / gamma.  Irradiance texel: R9 G9 B8 */
/* (beta 5, gamma 15) and a 6-bit sample count N; visibility texel: the     */
/* mean distance and mean squared distance, both divided by the probe cage  */
/* diagonal s (and s^2), 13 bits each with (beta, gamma) = (5, 15) and      */
/* (8, 20), and N.  The code is exact through its thresholds: code k stands */
/* for t_k = (exp(beta k / (2^b - 1)) - 1) / gamma (FP64, rounded to FP32),  */
/* and v codes to the largest k with t_k <= v -- rounding down of u, with    */
/* the thresholds as the single definition of the boundaries.               */
/* Sample updates follow Alg. MovingAvgUpdate one sample at a time (as the  */
/* CAS loop of Alg. atmMvAvgUpd serialises them), in sample order:          */
/* V = v / (n + 1) + (n o) / (n + 1) in FP32 on the decoded o, then coded   */
/* again; N = min(n + 1, 63) (6 bits).                                      */
/* ------------------------------------------------------------------------ */
#define PK_NMAX 63u
typedef struct {
    int bits;
    uint32_t kmax;
    float t[8192];
} codec_tab;

static void codec_init(codec_tab* c, int bits, double beta, double gamma)
{
    c->bits = bits;
    c->kmax = (1u << bits) - 1u;
    for (uint32_t k = 0; k <= c->kmax; ++k)
        c->t[k] = (float)((exp(beta * (double)k / (double)c->kmax) - 1.0) / gamma);
}

static uint32_t codec_enc(const codec_tab* c, float v)
{
    if (!(v > 0.0f)) return 0u; /* negatives, zero and NaN code to 0 */
    uint32_t lo = 0, hi = c->kmax; /* t[lo] <= v */
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1u) / 2u;
        if (c->t[mid] <= v)
            lo = mid;
        else
            hi = mid - 1u;
    }
    return lo;
}

static float codec_dec(const codec_tab* c, uint32_t k) { return c->t[k <= c->kmax ? k : c->kmax]; }

/* one moving-average step on a decoded value (Alg. MovingAvgUpdate), FP32 */
static float mav_step(float o, float v, uint32_t n)
{
    float n1 = (float)(n + 1u);
    float a = v / n1;
    float b = ((float)n * o) / n1;
    return a + b;
}

static codec_tab g_c9, g_c8, g_c13m, g_c13q;
static pthread_once_t g_codec_once = PTHREAD_ONCE_INIT;
static void codec_tables_init(void)
{
    codec_init(&g_c9, 9, 5.0, 15.0);
    codec_init(&g_c8, 8, 5.0, 15.0);
    codec_init(&g_c13m, 13, 5.0, 15.0);
    codec_init(&g_c13q, 13, 8.0, 20.0);
}

static const codec_tab* codec_of(int which)
{
    pthread_once(&g_codec_once, codec_tables_init);
    switch (which) {
    case 0: return &g_c9;
    case 1: return &g_c8;
    case 2: return &g_c13m;
    default: return &g_c13q;
    }
}

/* which: 0 = 9-bit irradiance, 1 = 8-bit irradiance, 2 = 13-bit mean
   distance, 3 = 13-bit mean squared distance */
EXPORT uint32_t orc_codec_enc(int which, float v) { return codec_enc(codec_of(which), v); }
EXPORT float orc_codec_dec(int which, uint32_t k) { return codec_dec(codec_of(which), k); }
EXPORT float orc_codec_mav(float o, float v, uint32_t n) { return mav_step(o, v, n); }

/* packed texels: irradiance R bits 0-8, G 9-17, B 18-25, N 26-31;
   visibility mean bits 0-12, mean square 13-25, N 26-31 */
static uint32_t pk_irr_update(uint32_t code, const float v[3])
{
    const codec_tab *c9 = codec_of(0), *c8 = codec_of(1);
    uint32_t n = code >> 26;
    float o0 = codec_dec(c9, code & 511u), o1 = codec_dec(c9, (code >> 9) & 511u), o2 = codec_dec(c8, (code >> 18) & 255u);
    uint32_t k0 = codec_enc(c9, mav_step(o0, v[0], n));
    uint32_t k1 = codec_enc(c9, mav_step(o1, v[1], n));
    uint32_t k2 = codec_enc(c8, mav_step(o2, v[2], n));
    uint32_t nn = n + 1u < PK_NMAX ? n + 1u : PK_NMAX;
    return k0 | (k1 << 9) | (k2 << 18) | (nn << 26);
}

static uint32_t pk_dep_update(uint32_t code, float x)
{
    const codec_tab *cm = codec_of(2), *cq = codec_of(3);
    uint32_t n = code >> 26;
    float om = codec_dec(cm, code & 8191u), oq = codec_dec(cq, (code >> 13) & 8191u);
    uint32_t km = codec_enc(cm, mav_step(om, x, n));
    uint32_t kq = codec_enc(cq, mav_step(oq, x * x, n));
    uint32_t nn = n + 1u < PK_NMAX ? n + 1u : PK_NMAX;
    return km | (kq << 13) | (nn << 26);
}

/* Metropolis chain steps per frame, rejected initial steps, samples per chain */
#define MH_M 8
#define MH_K 2
#define MH_S (MH_M - MH_K - 1)
/* proposal sigmas of the static chains: half a probe spacing, sqrt(pi / 256) */
#define MH_SG 0.5f
#define MH_SU 0.11077321f
/* the dynamic chains step 3x and 6x farther (in proxy units: half a proxy) */
#define DYN_SG 0.5f
#define DYN_SU 0.66463926f

/* ------------------------------------------------------------------------ */
/* Volume state                                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    float origin[3], spacing[3];
    int dims[3];
    int n_irr, n_dep;     /* interior texel counts per side */
    int avg, rmin, rmax;  /* ray budget */
    float hyst;           /* hysteresis h */
    float depth_max;      /* depth clamp; <= 0 selects 1.5 * voxel diagonal */
    int theta;            /* temporal trigger decay length (frames) */
    int packed;           /* 1: 32-bit packed atlases (the paper's codecs) */
    int sampler;          /* 0: deterministic allocation; 1: Metropolis chains (static guide) */
    float alpha;          /* confidence alpha in the cache term of the guide (Eq. DDGIBays) */
    int blend_mode;       /* 0 nearest texel (Alg. ApproxAlgo); 1 DDGI cosine gather (Sec. 3.1)  */
    int dyn_ratio;        /* sampler = 1: > 0 adds the dynamic chains (Sec. "Adaptive sampling -  */
                          /* dynamic") with a static:dynamic budget split of dyn_ratio:1      */
    float hyst_dyn;       /* hysteresis of the dynamic rays' batch update */
    float var_rel;        /* Chebyshev minimum variance relative to mu2 (0: the absolute floor alone) */
} orc_desc;

typedef struct {
    int kind; /* 0 point, 1 directional (v = direction light travels) */
    float v[3];
    float rgb[3];
} orc_light;

typedef struct {
    uint64_t frame, seed;
    const orc_light* lights;
    int n_lights;
    float sky[3];
    int has_camera;
    float cam[3];
    float cam_k;
    int has_clip;    /* 1: clip volumes from the camera's view-projection matrix (Fig. TrCam(b)) */
    float clip[16];  /* row-major 4x4: clip = M (x, y, z, 1) */
} orc_frame;

typedef struct orc_vol {
    orc_desc d;
    int P, m0, Ti, Td; /* probes, min rays, tile sides */
    double s;          /* voxel diagonal (Eq. ProbeVis) */
    float tmin, depth_max, qv_scale, qc_scale;
    uint16_t lut_v[4096], lut_c[4096];
    int sf_M;
    float* sf; /* concatenated SF sets for m = 1..sf_M, set m at m(m-1)/2 */
    /* scene */
    int nv, nt;
    float* V;
    int* I;
    float* alb;
    cbvh bvh;
    int bvh_dirty;
    /* packed atlases (desc.packed): the codes are the state; irr/dep
       below then hold their decoded FP64 view, which the queries read */
    uint32_t* irr_pk; /* P * Ti*Ti */
    uint32_t* dep_pk; /* P * Td*Td */
    float s_f;        /* (float) s: the visibility normaliser */
    /* atlases, FP64 */
    double* irr;    /* P * Ti*Ti * 3 */
    uint8_t* irr_n; /* P * Ti*Ti */
    double* dep;    /* P * Td*Td * 2 */
    uint8_t* dep_n; /* P * Td*Td */
    /* change state, per probe and octant */
    uint16_t *qv_even, *qr_even, *qv, *qr;
    uint16_t *amp_v, *amp_r; /* trigger pulse heights */
    uint8_t *age_v, *age_r;  /* frames since the pulse */
    uint16_t *trv, *trr;     /* trigger outputs f_1, f_3 */
    int64_t last_even;
    /* last update's intermediates */
    uint32_t *W, *n, *off;
    float* pil_t;
    int* pil_tri;
    float* pil_lum;
    float* pil_dir;  /* P*8*3 */
    double* pil_rad; /* P*8*3 */
    double* pil_dep; /* P*8 */
    size_t R_main;
    float* m_t;
    int* m_tri;
    double* m_rad;
    double* m_dep;
    float R[9];
    int nthreads;
    /* Metropolis sampler (desc.sampler = 1) */
    size_t B;            /* samples per frame: (avg - 8) * P */
    size_t C;            /* chains: ceil(B / samples per chain) */
    int chains_live;     /* chain states initialised */
    float* ch_g;         /* C*3 grid coordinates */
    float* ch_u;         /* C*2 octahedral coordinates */
    int* smp_p;          /* B probe of each sample */
    float* smp_dir;      /* B*3 direction */
    float* smp_t;        /* B nearest hit along +w (inf on a miss) */
    int* smp_tri;
    float* smp_tn;       /* B nearest hit along -w */
    int* smp_trin;
    double* smp_rad;     /* B*3 radiance along +w */
    double* smp_dep;     /* B distance along -w (clamped) */
    uint32_t* smp_off;   /* P+1 first sample of each probe in smp_ord */
    uint32_t* smp_ord;   /* B sample indices grouped by probe, in sample order */
    uint32_t* qd;        /* P*8 dynamic weight q_d of each probe and octant (Eq. priorDynamic) */
    uint8_t* cls;        /* P clip volume of each probe this frame: 2 V_in, 1 V_out - V_in, 0 outside */
    uint8_t* vout_even;  /* P 1: the probe was in V_out on the last first-of-pair frame */
    /* dynamic chains over virtual proxies (desc.dyn_ratio > 0) */
    int Dp[3], Pp;       /* proxy grid: ceil(dims / 3) */
    size_t Cd, Bd;       /* dynamic chains, dynamic samples per frame (5 per chain) */
    size_t Rd;           /* dynamic ray budget per frame */
    int dyn_live;
    float* dch_g;        /* Cd*3 proxy-grid coordinates */
    float* dch_u;        /* Cd*2 octahedral coordinates */
    int* dsm_q;          /* Bd proxy of each dynamic sample */
    float* dsm_dir;      /* Bd*3 */
    int* dsm_cell;       /* Bd proxy*8 + octant, -1 where the target is 0 */
    uint32_t* dfirst;    /* Pp*8 first dynamic sample of each cell (UINT32_MAX: unmarked) */
    int* dmark;          /* marked cells in first-sample order */
    int n_marked, n_incl;/* marked cells; the leading ones within the ray budget */
    uint8_t* dincl;      /* Pp*8 1: the cell's rays are traced this frame */
    int ntex[8];         /* irradiance interior texels whose centre lies in each octant */
    int* tex_t;          /* [8][n_irr^2] their tile indices, in texel order */
    float* tex_dir;      /* [8][n_irr^2][3] their centre directions (FP32) */
    uint32_t* doff;      /* P+1 dynamic rays of each probe */
    size_t Rdyn;         /* this frame's dynamic rays */
    int* d_p;            /* Rd probe of each dynamic ray */
    int* d_k;            /* Rd octant * n_irr^2 + index in the octant's texel list */
    float* d_t;
    int* d_tri;
    double* d_rad;       /* Rd*3 */
    double* d_dep;       /* Rd */
} orc_vol;

static void build_luts(orc_vol* v)
{
    /* q_v LUT: f_v = exp(-2 t / s) at the centre of distance bin i of width s/256 */
    for (int i = 0; i < 4096; ++i) {
        double f = exp(-2.0 * ((double)i + 0.5) / 256.0);
        v->lut_v[i] = (uint16_t)floor(1023.0 * f);
    }
    /* q_c LUT: f_c = exp(-(|p-c| - k)) at the centre of bin i of width s/64 */
    for (int i = 0; i < 4096; ++i) {
        double f = exp(-((double)i + 0.5) * v->s / 64.0);
        v->lut_c[i] = (uint16_t)floor(1023.0 * f);
    }
}

EXPORT void orc_luts(double s, uint16_t* lut_v, uint16_t* lut_c)
{
    orc_vol tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.s = s;
    build_luts(&tmp);
    memcpy(lut_v, tmp.lut_v, sizeof(tmp.lut_v));
    memcpy(lut_c, tmp.lut_c, sizeof(tmp.lut_c));
}

EXPORT void orc_destroy(orc_vol* v);
static void dyn_create(orc_vol* v);

EXPORT orc_vol* orc_create(const orc_desc* d, int nthreads)
{
    if (d->dims[0] < 2 || d->dims[1] < 2 || d->dims[2] < 2) return NULL;
    if (d->n_irr < 1 || d->n_dep < 1 || d->theta < 1) return NULL;
    int m0 = d->rmin > 8 ? d->rmin : 8;
    if (d->avg < m0 || d->avg > d->rmax) return NULL;
    if (!(d->var_rel >= 0.0f && d->var_rel < 1.0f)) return NULL;
    orc_vol* v = (orc_vol*)calloc(1, sizeof(orc_vol));
    v->d = *d;
    v->P = d->dims[0] * d->dims[1] * d->dims[2];
    v->m0 = m0;
    v->Ti = d->n_irr + 2;
    v->Td = d->n_dep + 2;
    double sx = d->spacing[0], sy = d->spacing[1], sz = d->spacing[2];
    v->s = sqrt((sx * sx + sy * sy) + sz * sz);
    v->tmin = (float)(1e-4 * v->s);
    v->depth_max = d->depth_max > 0.0f ? d->depth_max : (float)(1.5 * v->s);
    v->qv_scale = (float)(256.0 / v->s);
    v->qc_scale = (float)(64.0 / v->s);
    build_luts(v);
    v->sf_M = d->rmax - 8;
    if (v->sf_M > 0) {
        size_t tot = (size_t)v->sf_M * (size_t)(v->sf_M + 1) / 2;
        v->sf = (float*)malloc(sizeof(float) * 3 * tot);
        for (int m = 1; m <= v->sf_M; ++m) orc_sf_points(m, v->sf + 3 * ((size_t)m * (size_t)(m - 1) / 2));
    }
    size_t P = (size_t)v->P;
    v->s_f = (float)v->s;
    if (d->packed) {
        v->irr_pk = (uint32_t*)calloc(P * v->Ti * v->Ti, 4);
        v->dep_pk = (uint32_t*)calloc(P * v->Td * v->Td, 4);
    }
    v->irr = (double*)calloc(P * v->Ti * v->Ti * 3, sizeof(double));
    v->irr_n = (uint8_t*)calloc(P * v->Ti * v->Ti, 1);
    v->dep = (double*)calloc(P * v->Td * v->Td * 2, sizeof(double));
    v->dep_n = (uint8_t*)calloc(P * v->Td * v->Td, 1);
    v->qv_even = (uint16_t*)calloc(P * 8, 2);
    v->qr_even = (uint16_t*)calloc(P * 8, 2);
    v->trv = (uint16_t*)calloc(P * 8, 2);
    v->trr = (uint16_t*)calloc(P * 8, 2);
    v->amp_v = (uint16_t*)calloc(P * 8, 2);
    v->amp_r = (uint16_t*)calloc(P * 8, 2);
    v->age_v = (uint8_t*)malloc(P * 8);
    v->age_r = (uint8_t*)malloc(P * 8);
    memset(v->age_v, 255, P * 8);
    memset(v->age_r, 255, P * 8);
    v->qv = (uint16_t*)calloc(P * 8, 2);
    v->qr = (uint16_t*)calloc(P * 8, 2);
    v->qd = (uint32_t*)calloc(P * 8, 4);
    v->cls = (uint8_t*)malloc(P);
    memset(v->cls, 2, P);
    v->vout_even = (uint8_t*)calloc(P, 1);
    v->last_even = -2;
    v->W = (uint32_t*)calloc(P, 4);
    v->n = (uint32_t*)calloc(P, 4);
    v->off = (uint32_t*)calloc(P + 1, 4);
    v->pil_t = (float*)calloc(P * 8, 4);
    v->pil_tri = (int*)calloc(P * 8, 4);
    v->pil_lum = (float*)calloc(P * 8, 4);
    v->pil_dir = (float*)calloc(P * 8 * 3, 4);
    v->pil_rad = (double*)calloc(P * 8 * 3, 8);
    v->pil_dep = (double*)calloc(P * 8, 8);
    v->R_main = (size_t)(d->avg - 8) * P;
    v->m_t = (float*)calloc(v->R_main + 1, 4);
    v->m_tri = (int*)calloc(v->R_main + 1, 4);
    v->m_rad = (double*)calloc((v->R_main + 1) * 3, 8);
    v->m_dep = (double*)calloc(v->R_main + 1, 8);
    v->nthreads = nthreads > 0 ? nthreads : 1;
    if (d->sampler == 1) {
        if (d->packed) { /* the Metropolis mode blends with the batched moving average only */
            orc_destroy(v);
            return NULL;
        }
        v->B = v->R_main;
        if (d->dyn_ratio > 0) { /* budget split static:dynamic = r:1; a static sample costs two rays */
            size_t B = v->B, r = (size_t)d->dyn_ratio;
            v->B = B * r / (r + 1);
            v->Rd = 2 * (B - v->B);
        }
        v->C = (v->B + MH_S - 1) / MH_S;
        v->ch_g = (float*)calloc(v->C * 3 + 1, 4);
        v->ch_u = (float*)calloc(v->C * 2 + 1, 4);
        v->smp_p = (int*)calloc(v->B + 1, 4);
        v->smp_dir = (float*)calloc(v->B * 3 + 1, 4);
        v->smp_t = (float*)calloc(v->B + 1, 4);
        v->smp_tri = (int*)calloc(v->B + 1, 4);
        v->smp_tn = (float*)calloc(v->B + 1, 4);
        v->smp_trin = (int*)calloc(v->B + 1, 4);
        v->smp_rad = (double*)calloc(v->B * 3 + 1, 8);
        v->smp_dep = (double*)calloc(v->B + 1, 8);
        v->smp_off = (uint32_t*)calloc(P + 1, 4);
        v->smp_ord = (uint32_t*)calloc(v->B + 1, 4);
        if (d->dyn_ratio > 0) dyn_create(v);
    } else if (d->dyn_ratio != 0) { /* the dynamic chains belong to the Metropolis mode */
        orc_destroy(v);
        return NULL;
    }
    if (d->blend_mode != 0 && (d->blend_mode != 1 || d->sampler != 0 || d->packed)) {
        orc_destroy(v); /* the cosine gather blends the allocated rays into FP64 atlases */
        return NULL;
    }
    return v;
}

EXPORT void orc_destroy(orc_vol* v)
{
    if (!v) return;
    cbvh_free(&v->bvh);
    free(v->sf);
    free(v->V);
    free(v->I);
    free(v->alb);
    free(v->irr);
    free(v->irr_n);
    free(v->dep);
    free(v->dep_n);
    free(v->irr_pk);
    free(v->dep_pk);
    free(v->ch_g);
    free(v->ch_u);
    free(v->smp_p);
    free(v->smp_dir);
    free(v->smp_t);
    free(v->smp_tri);
    free(v->smp_tn);
    free(v->smp_trin);
    free(v->smp_rad);
    free(v->smp_dep);
    free(v->smp_off);
    free(v->smp_ord);
    free(v->qd);
    free(v->cls);
    free(v->vout_even);
    free(v->dch_g);
    free(v->dch_u);
    free(v->dsm_q);
    free(v->dsm_dir);
    free(v->dsm_cell);
    free(v->dfirst);
    free(v->dmark);
    free(v->dincl);
    free(v->tex_t);
    free(v->tex_dir);
    free(v->doff);
    free(v->d_p);
    free(v->d_k);
    free(v->d_t);
    free(v->d_tri);
    free(v->d_rad);
    free(v->d_dep);
    free(v->qv_even);
    free(v->qr_even);
    free(v->trv);
    free(v->trr);
    free(v->amp_v);
    free(v->amp_r);
    free(v->age_v);
    free(v->age_r);
    free(v->qv);
    free(v->qr);
    free(v->W);
    free(v->n);
    free(v->off);
    free(v->pil_t);
    free(v->pil_tri);
    free(v->pil_lum);
    free(v->pil_dir);
    free(v->pil_rad);
    free(v->pil_dep);
    free(v->m_t);
    free(v->m_tri);
    free(v->m_rad);
    free(v->m_dep);
    free(v);
}

EXPORT int orc_set_scene(orc_vol* v, const float* verts, int nv, const int* idx, int nt, const float* albedo)
{
    for (int t = 0; t < 3 * nt; ++t)
        if (idx[t] < 0 || idx[t] >= nv) return -1;
    free(v->V);
    free(v->I);
    free(v->alb);
    v->V = (float*)malloc(sizeof(float) * 3 * (size_t)(nv > 0 ? nv : 1));
    v->I = (int*)malloc(sizeof(int) * 3 * (size_t)(nt > 0 ? nt : 1));
    v->alb = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    memcpy(v->V, verts, sizeof(float) * 3 * (size_t)nv);
    memcpy(v->I, idx, sizeof(int) * 3 * (size_t)nt);
    memcpy(v->alb, albedo, sizeof(float) * 3 * (size_t)nt);
    v->nv = nv;
    v->nt = nt;
    v->bvh_dirty = 1;
    return 0;
}

EXPORT int orc_move_vertices(orc_vol* v, int first, int count, const float* verts)
{
    if (first < 0 || count < 0 || first + count > v->nv) return -1;
    memcpy(v->V + 3 * (size_t)first, verts, sizeof(float) * 3 * (size_t)count);
    v->bvh_dirty = 1;
    return 0;
}

/* probe position, FP32: origin + spacing * index */
static void probe_pos(const orc_vol* v, int p, float out[3])
{
    int ix = p % v->d.dims[0];
    int iy = (p / v->d.dims[0]) % v->d.dims[1];
    int iz = p / (v->d.dims[0] * v->d.dims[1]);
    out[0] = v->d.origin[0] + v->d.spacing[0] * (float)ix;
    out[1] = v->d.origin[1] + v->d.spacing[1] * (float)iy;
    out[2] = v->d.origin[2] + v->d.spacing[2] * (float)iz;
}

static void main_dir(const orc_vol* v, int m, int i, float d[3])
{
    const float* s = v->sf + 3 * ((size_t)m * (size_t)(m - 1) / 2 + (size_t)i);
    rotate_f32(v->R, s, d);
}

/* geometric normal, FP32, normalised: (B-A) x (C-A) / |.| */
static void tri_normal_f32(const orc_vol* v, int t, float n[3])
{
    const int* ix = v->I + 3 * (size_t)t;
    const float *A = v->V + 3 * (size_t)ix[0], *B = v->V + 3 * (size_t)ix[1], *C = v->V + 3 * (size_t)ix[2];
    float e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    float e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    float c[3];
    c[0] = e1[1] * e2[2] - e1[2] * e2[1];
    c[1] = e1[2] * e2[0] - e1[0] * e2[2];
    c[2] = e1[0] * e2[1] - e1[1] * e2[0];
    float l = sqrtf((c[0] * c[0] + c[1] * c[1]) + c[2] * c[2]);
    if (l > 0.0f) {
        n[0] = c[0] / l;
        n[1] = c[1] / l;
        n[2] = c[2] / l;
    } else {
        n[0] = 0.0f;
        n[1] = 0.0f;
        n[2] = 1.0f;
    }
}

static void tri_normal_f64(const orc_vol* v, int t, double n[3])
{
    const int* ix = v->I + 3 * (size_t)t;
    const float *A = v->V + 3 * (size_t)ix[0], *B = v->V + 3 * (size_t)ix[1], *C = v->V + 3 * (size_t)ix[2];
    double e1[3] = {(double)B[0] - A[0], (double)B[1] - A[1], (double)B[2] - A[2]};
    double e2[3] = {(double)C[0] - A[0], (double)C[1] - A[1], (double)C[2] - A[2]};
    double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double l = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (l > 0.0) {
        n[0] = c[0] / l;
        n[1] = c[1] / l;
        n[2] = c[2] / l;
    } else {
        n[0] = 0.0;
        n[1] = 0.0;
        n[2] = 1.0;
    }
}

static hitrec vol_closest(const orc_vol* v, const float o[3], const float d[3], float tmin, float tmax)
{
    return closest_bvh(&v->bvh, o, d, tmin, tmax);
}

/* ------------------------------------------------------------------------ */
/* Irradiance query (Sec. 3.1, DDGI lookup; Chebyshev visibility g_c of     */
/* Table "List of symbols"), FP64.                                          */
/* ------------------------------------------------------------------------ */
static void bilinear(const double* tile, int T, int n, int ch, const double dir[3], double* out)
{
    double p[2];
    orc_oct_encode(dir, p);
    double fx = (1.0 + (p[0] + 1.0) * 0.5 * n) - 0.5;
    double fy = (1.0 + (p[1] + 1.0) * 0.5 * n) - 0.5;
    int x0 = (int)floor(fx), y0 = (int)floor(fy);
    if (x0 < 0) x0 = 0;
    if (x0 > n) x0 = n;
    if (y0 < 0) y0 = 0;
    if (y0 > n) y0 = n;
    double ax = fx - x0, ay = fy - y0;
    if (ax < 0.0) ax = 0.0;
    if (ax > 1.0) ax = 1.0;
    if (ay < 0.0) ay = 0.0;
    if (ay > 1.0) ay = 1.0;
    for (int c = 0; c < ch; ++c) {
        double v00 = tile[(y0 * T + x0) * ch + c], v01 = tile[(y0 * T + x0 + 1) * ch + c];
        double v10 = tile[((y0 + 1) * T + x0) * ch + c], v11 = tile[((y0 + 1) * T + x0 + 1) * ch + c];
        out[c] = (1.0 - ay) * ((1.0 - ax) * v00 + ax * v01) + ay * ((1.0 - ax) * v10 + ax * v11);
    }
}

/* FP32 coordinate of probe plane j along axis k (where the probes sit) */
static double pcoord(const orc_vol* v, int k, int j)
{
    float c = v->d.origin[k] + v->d.spacing[k] * (float)j;
    return (double)c;
}

/* The probe cage holding x: along each axis the last probe plane at or below x
   (clamped to the grid), and the trilinear fraction from that plane. */
static void query_point(const orc_vol* v, const double x[3], const double nrm[3], double out[3])
{
    double a[3];
    int b[3];
    for (int k = 0; k < 3; ++k) {
        int n = v->d.dims[k];
        int bi = 0;
        while (bi < n - 2 && x[k] >= pcoord(v, k, bi + 1)) ++bi;
        b[k] = bi;
        double al = (x[k] - pcoord(v, k, bi)) / (double)v->d.spacing[k];
        if (al < 0.0) al = 0.0;
        if (al > 1.0) al = 1.0;
        a[k] = al;
    }
    double nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    double nd[3] = {0.0, 0.0, 1.0};
    if (nl > 0.0) {
        nd[0] = nrm[0] / nl;
        nd[1] = nrm[1] / nl;
        nd[2] = nrm[2] / nl;
    }
    double sum[3] = {0, 0, 0}, sumt[3] = {0, 0, 0}, sw = 0.0;
    double varmin = 1e-6 * v->s * v->s;
    for (int c = 0; c < 8; ++c) {
        int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double wt = 1.0;
        int ii[3];
        for (int k = 0; k < 3; ++k) {
            wt *= o[k] ? a[k] : 1.0 - a[k];
            ii[k] = b[k] + o[k];
        }
        int p = ii[0] + v->d.dims[0] * (ii[1] + v->d.dims[1] * ii[2]);
        float pp[3];
        probe_pos(v, p, pp);
        double dv[3] = {x[0] - pp[0], x[1] - pp[1], x[2] - pp[2]};
        double dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double dir[3] = {0.0, 0.0, 1.0};
        if (dist > 0.0) {
            dir[0] = dv[0] / dist;
            dir[1] = dv[1] / dist;
            dir[2] = dv[2] / dist;
        }
        double mom[2];
        bilinear(v->dep + (size_t)p * v->Td * v->Td * 2, v->Td, v->d.n_dep, 2, dir, mom);
        double wc = 1.0;
        if (dist > mom[0]) {
            /* one-sided Chebyshev bound P(d >= dist) <= var / (var + (dist - mu)^2)
               on the filtered moments (variance shadow maps, cited for g_c),
               var = mu2 - mu^2 raised to the minimum variance 1e-6 s^2; a
               volume may ask for a larger floor var_rel * mu2 */
            double var = mom[1] - mom[0] * mom[0];
            double vrel = (double)v->d.var_rel * mom[1];
            double vfloor = vrel > varmin ? vrel : varmin;
            if (var < vfloor) var = vfloor;
            double dd = dist - mom[0];
            wc = var / (var + dd * dd);
        }
        double E[3];
        bilinear(v->irr + (size_t)p * v->Ti * v->Ti * 3, v->Ti, v->d.n_irr, 3, nd, E);
        double w = wt * wc;
        for (int k = 0; k < 3; ++k) {
            sum[k] += w * E[k];
            sumt[k] += wt * E[k];
        }
        sw += w;
    }
    for (int k = 0; k < 3; ++k) out[k] = sw >= 1e-12 ? sum[k] / sw : sumt[k];
}

EXPORT void orc_query(const orc_vol* v, int n, const float* pos, const float* nrm, double* out)
{
    for (int i = 0; i < n; ++i) {
        double x[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        double nn[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        query_point(v, x, nn, out + 3 * (size_t)i);
    }
}

/* ------------------------------------------------------------------------ */
/* Shading of one ray.                                                       */
/* Direct light with shadow rays + multi-bounce albedo * Q_{t-1}(x, n)       */
/* (Sec. 4.1 "Incoming radiance"; Sec. 4.5 static sampling traces the       */
/* scene; DDGI multi-bounce, Sec. 3.1).  Visibility and the lit test are     */
/* FP32 decisions; magnitudes are FP64.  lum32 receives the FP32 luminance   */
/* of the direct-only radiance (the r of f_r).                              */
/* ------------------------------------------------------------------------ */
static const float LUM_R = 0.2126f, LUM_G = 0.7152f, LUM_B = 0.0722f;
static const float INV_PI_F = 0.31830987f;

static void shade_ray(const orc_vol* v, const orc_frame* fr, const float o[3], const float d[3], hitrec h,
                      double rad[3], double* depth, float* lum32)
{
    if (h.tri < 0) {
        for (int k = 0; k < 3; ++k) rad[k] = fr->sky[k];
        *depth = v->depth_max;
        if (lum32) *lum32 = (LUM_R * fr->sky[0] + LUM_G * fr->sky[1]) + LUM_B * fr->sky[2];
        return;
    }
    *depth = h.t < v->depth_max ? h.t : v->depth_max;
    if (h.det < 0.0f) { /* back face */
        rad[0] = rad[1] = rad[2] = 0.0;
        if (lum32) *lum32 = 0.0f;
        return;
    }
    float x[3], n[3], xs[3];
    for (int k = 0; k < 3; ++k) x[k] = o[k] + h.t * d[k];
    tri_normal_f32(v, h.tri, n);
    for (int k = 0; k < 3; ++k) xs[k] = x[k] + v->tmin * n[k];
    double n64[3];
    tri_normal_f64(v, h.tri, n64);
    double x64[3];
    for (int k = 0; k < 3; ++k) x64[k] = (double)o[k] + (double)h.t * (double)d[k];
    const float* alb = v->alb + 3 * (size_t)h.tri;
    double E[3] = {0, 0, 0};
    float E32[3] = {0.0f, 0.0f, 0.0f};
    for (int l = 0; l < fr->n_lights; ++l) {
        const orc_light* L = &fr->lights[l];
        float D[3];
        float thi;
        if (L->kind == 0) {
            for (int k = 0; k < 3; ++k) D[k] = L->v[k] - xs[k];
            thi = 1.0f;
        } else {
            for (int k = 0; k < 3; ++k) D[k] = -L->v[k];
            thi = INFINITY;
        }
        float ndD = (n[0] * D[0] + n[1] * D[1]) + n[2] * D[2];
        if (!(ndD > 0.0f)) continue;
        if (anyhit_bvh(&v->bvh, xs, D, 0.0f, thi)) continue;
        /* FP32 irradiance for the pilot luminance */
        float g32;
        if (L->kind == 0) {
            float Dx[3] = {L->v[0] - x[0], L->v[1] - x[1], L->v[2] - x[2]};
            float d2 = (Dx[0] * Dx[0] + Dx[1] * Dx[1]) + Dx[2] * Dx[2];
            float nd = (n[0] * Dx[0] + n[1] * Dx[1]) + n[2] * Dx[2];
            g32 = nd > 0.0f ? nd / (d2 * sqrtf(d2)) : 0.0f;
        } else {
            float l2 = (L->v[0] * L->v[0] + L->v[1] * L->v[1]) + L->v[2] * L->v[2];
            g32 = ndD / sqrtf(l2);
        }
        for (int k = 0; k < 3; ++k) E32[k] = E32[k] + L->rgb[k] * g32;
        /* FP64 irradiance */
        double g;
        if (L->kind == 0) {
            double Dx[3] = {(double)L->v[0] - x64[0], (double)L->v[1] - x64[1], (double)L->v[2] - x64[2]};
            double d2 = Dx[0] * Dx[0] + Dx[1] * Dx[1] + Dx[2] * Dx[2];
            double nd = n64[0] * Dx[0] + n64[1] * Dx[1] + n64[2] * Dx[2];
            g = nd > 0.0 ? nd / (d2 * sqrt(d2)) : 0.0;
        } else {
            double l2 = (double)L->v[0] * L->v[0] + (double)L->v[1] * L->v[1] + (double)L->v[2] * L->v[2];
            double nd = -(n64[0] * L->v[0] + n64[1] * L->v[1] + n64[2] * L->v[2]);
            g = nd > 0.0 ? nd / sqrt(l2) : 0.0;
        }
        for (int k = 0; k < 3; ++k) E[k] += (double)L->rgb[k] * g;
    }
    double Q[3];
    query_point(v, x64, n64, Q);
    for (int k = 0; k < 3; ++k) rad[k] = (double)alb[k] / M_PI * E[k] + (double)alb[k] * Q[k];
    if (lum32) {
        float r0 = (alb[0] * INV_PI_F) * E32[0];
        float r1 = (alb[1] * INV_PI_F) * E32[1];
        float r2 = (alb[2] * INV_PI_F) * E32[2];
        *lum32 = (LUM_R * r0 + LUM_G * r1) + LUM_B * r2;
    }
}

/* ------------------------------------------------------------------------ */
/* Blend (Alg. ApproxAlgo + Alg. MovingAvgUpdate, batch form): every sample */
/* of this frame updates its nearest texel; for a texel with k samples of   */
/* mean m and stored (V, n):  V' = V + w (m - V),  w = max(1 - h, k/(n+k)),  */
/* n' = min(n + k, 255).  Untouched texels keep their value.  Then the      */
/* one-texel octahedral border is refreshed from the interior.             */
/* ------------------------------------------------------------------------ */
/* one batched moving-average step of the texels with k > 0 samples (sums s):
   V += w (s/k - V), w = max(1 - h, k/(n + k)), n = min(n + k, 255) */
static void batch_apply(double* val, uint8_t* cnt, const double* s, const int* kk, int texels, int ch, double h)
{
    for (int t = 0; t < texels; ++t) {
        if (!kk[t]) continue;
        double k = kk[t], n = cnt[t];
        double w = k / (n + k);
        if (w < 1.0 - h) w = 1.0 - h;
        for (int c = 0; c < ch; ++c) val[t * ch + c] += w * (s[t * ch + c] / k - val[t * ch + c]);
        int nn = cnt[t] + kk[t];
        cnt[t] = (uint8_t)(nn > 255 ? 255 : nn);
    }
}

static void border_copy(double* tile, uint8_t* cnt, int n, int ch)
{
    int T = n + 2;
#define CP(di, dj, si, sj)                                                    \
    do {                                                                      \
        for (int c = 0; c < ch; ++c) tile[((di)*T + (dj)) * ch + c] = tile[((si)*T + (sj)) * ch + c]; \
        cnt[(di)*T + (dj)] = cnt[(si)*T + (sj)];                              \
    } while (0)
    for (int j = 1; j <= n; ++j) {
        CP(0, j, 1, n + 1 - j);
        CP(n + 1, j, n, n + 1 - j);
    }
    for (int i = 1; i <= n; ++i) {
        CP(i, 0, n + 1 - i, 1);
        CP(i, n + 1, n + 1 - i, n);
    }
    CP(0, 0, n, n);
    CP(0, n + 1, n, 1);
    CP(n + 1, 0, 1, n);
    CP(n + 1, n + 1, 1, 1);
#undef CP
}

/* octahedral border fold of a tile of codes (the same texel map as
   border_copy) */
static void border_copy_u32(uint32_t* tile, int n)
{
    int T = n + 2;
    for (int j = 1; j <= n; ++j) {
        tile[j] = tile[T + (n + 1 - j)];
        tile[(n + 1) * T + j] = tile[n * T + (n + 1 - j)];
    }
    for (int i = 1; i <= n; ++i) {
        tile[i * T] = tile[(n + 1 - i) * T + 1];
        tile[i * T + n + 1] = tile[(n + 1 - i) * T + n];
    }
    tile[0] = tile[n * T + n];
    tile[n + 1] = tile[n * T + 1];
    tile[(n + 1) * T] = tile[T + n];
    tile[(n + 1) * T + n + 1] = tile[T + 1];
}

/* the decoded view of probe p's packed tiles (what the queries read) */
static void decode_probe(orc_vol* v, int p)
{
    const int Ti = v->Ti, Td = v->Td;
    const codec_tab *c9 = codec_of(0), *c8 = codec_of(1), *cm = codec_of(2), *cq = codec_of(3);
    const double s = (double)v->s_f;
    for (int t = 0; t < Ti * Ti; ++t) {
        uint32_t c = v->irr_pk[(size_t)p * Ti * Ti + t];
        double* o = v->irr + ((size_t)p * Ti * Ti + t) * 3;
        o[0] = codec_dec(c9, c & 511u);
        o[1] = codec_dec(c9, (c >> 9) & 511u);
        o[2] = codec_dec(c8, (c >> 18) & 255u);
        v->irr_n[(size_t)p * Ti * Ti + t] = (uint8_t)(c >> 26);
    }
    for (int t = 0; t < Td * Td; ++t) {
        uint32_t c = v->dep_pk[(size_t)p * Td * Td + t];
        double* o = v->dep + ((size_t)p * Td * Td + t) * 2;
        o[0] = (double)codec_dec(cm, c & 8191u) * s;
        o[1] = (double)codec_dec(cq, (c >> 13) & 8191u) * s * s;
        v->dep_n[(size_t)p * Td * Td + t] = (uint8_t)(c >> 26);
    }
}

/* Packed blend: every sample, in sample order (pilots first, then SF index
   order), updates its nearest irradiance and visibility texel with one
   moving-average step on the codes; then the border fold. */
static void blend_probe_packed(orc_vol* v, int p, int use_pilots)
{
    const int Ti = v->Ti, Td = v->Td, ni = v->d.n_irr, nd = v->d.n_dep;
    uint32_t* irr = v->irr_pk + (size_t)p * Ti * Ti;
    uint32_t* dep = v->dep_pk + (size_t)p * Td * Td;
    const uint32_t mp = v->n[p] > 8u ? v->n[p] - 8u : 0u;
    const int total = (int)mp + (use_pilots ? 8 : 0);
    for (int j = 0; j < total; ++j) {
        float d[3];
        const double* rad;
        double ds;
        if (use_pilots && j < 8) {
            const float* pd = v->pil_dir + ((size_t)p * 8 + (size_t)j) * 3;
            d[0] = pd[0];
            d[1] = pd[1];
            d[2] = pd[2];
            rad = v->pil_rad + ((size_t)p * 8 + (size_t)j) * 3;
            ds = v->pil_dep[(size_t)p * 8 + (size_t)j];
        } else {
            int i = use_pilots ? j - 8 : j;
            main_dir(v, (int)mp, i, d);
            size_t r = (size_t)v->off[p] + (size_t)i;
            rad = v->m_rad + r * 3;
            ds = v->m_dep[r];
        }
        int ti = orc_texel_of_dir(d, ni);
        int td = orc_texel_of_dir(d, nd);
        float vr[3] = {(float)rad[0], (float)rad[1], (float)rad[2]};
        irr[ti] = pk_irr_update(irr[ti], vr);
        float x = (float)ds / v->s_f; /* distance in units of the cage diagonal */
        dep[td] = pk_dep_update(dep[td], x);
    }
    if (v->cls[p] == 1) { /* V_out - V_in: sample counts set down to 16 (catch-up) */
        for (int t = 0; t < Ti * Ti; ++t)
            if ((irr[t] >> 26) > 16u) irr[t] = (irr[t] & 0x03FFFFFFu) | (16u << 26);
        for (int t = 0; t < Td * Td; ++t)
            if ((dep[t] >> 26) > 16u) dep[t] = (dep[t] & 0x03FFFFFFu) | (16u << 26);
    }
    border_copy_u32(irr, ni);
    border_copy_u32(dep, nd);
    decode_probe(v, p);
}

static void blend_probe(orc_vol* v, int p, int use_pilots, double h)
{
    const int Ti = v->Ti, Td = v->Td, ni = v->d.n_irr, nd = v->d.n_dep;
    double* irr = v->irr + (size_t)p * Ti * Ti * 3;
    uint8_t* irn = v->irr_n + (size_t)p * Ti * Ti;
    double* dep = v->dep + (size_t)p * Td * Td * 2;
    uint8_t* den = v->dep_n + (size_t)p * Td * Td;
    double* si = (double*)calloc((size_t)Ti * Ti * 3, sizeof(double));
    int* ki = (int*)calloc((size_t)Ti * Ti, sizeof(int));
    double* sd = (double*)calloc((size_t)Td * Td * 2, sizeof(double));
    int* kd = (int*)calloc((size_t)Td * Td, sizeof(int));
    const uint32_t mp = v->n[p] > 8u ? v->n[p] - 8u : 0u;
    const int total = (int)mp + (use_pilots ? 8 : 0);
    for (int j = 0; j < total; ++j) {
        float d[3];
        const double* rad;
        double ds;
        if (use_pilots && j < 8) {
            const float* pd = v->pil_dir + ((size_t)p * 8 + (size_t)j) * 3;
            d[0] = pd[0];
            d[1] = pd[1];
            d[2] = pd[2];
            rad = v->pil_rad + ((size_t)p * 8 + (size_t)j) * 3;
            ds = v->pil_dep[(size_t)p * 8 + (size_t)j];
        } else {
            int i = use_pilots ? j - 8 : j;
            main_dir(v, (int)mp, i, d);
            size_t r = (size_t)v->off[p] + (size_t)i;
            rad = v->m_rad + r * 3;
            ds = v->m_dep[r];
        }
        int ti = orc_texel_of_dir(d, ni);
        int td = orc_texel_of_dir(d, nd);
        for (int c = 0; c < 3; ++c) si[ti * 3 + c] += rad[c];
        ki[ti] += 1;
        sd[td * 2 + 0] += ds;
        sd[td * 2 + 1] += ds * ds;
        kd[td] += 1;
    }
    batch_apply(irr, irn, si, ki, Ti * Ti, 3, h);
    batch_apply(dep, den, sd, kd, Td * Td, 2, h);
    if (v->cls[p] == 1) { /* V_out - V_in: sample counts set down to 16 (catch-up) */
        for (int t = 0; t < Ti * Ti; ++t)
            if (irn[t] > 16) irn[t] = 16;
        for (int t = 0; t < Td * Td; ++t)
            if (den[t] > 16) den[t] = 16;
    }
    border_copy(irr, irn, ni, 3);
    border_copy(dep, den, nd, 2);
    free(si);
    free(ki);
    free(sd);
    free(kd);
}

/* ------------------------------------------------------------------------ */
/* Heuristics (Sec. 4.1-4.2), integer form.                                 */
/*   q_v(p,o) = LUT_v[min(floor(t * 256/s), 4095)], t from the pilot ray of */
/*              the opposite octant 7-o (f_v uses trace(p, -w))              */
/*   q_r(p,o) = floor(1023 * min(lum, 5) / 5)                                */
/*   trigger Tr(., theta) (Fig. TrCam(a)): a pulse of height v starts a     */
/*            signal that decays linearly to 0 over theta frames,           */
/*            y = floor(v (theta - age) / theta); a new pulse replaces the  */
/*            running one when it is at least the current value.  Pulses    */
/*            are the deltas |q_t - q_{t-1}| taken on the second frame of   */
/*            each pair (identical rays, Sec. 4.4); ages advance every frame */
/*   f_D(p,o) = sum over the 5x5x5 probe box clipped to the grid and over    */
/*              o' in {o, o^1, o^2, o^4} of Tr(p', o')                       */
/*   q_d(p,o) = (q_c q_v (f_Dv + 2 f_Dr)) >> 20          (mu = 2)           */
/*   W_p      = min(sum_o q_d(p,o), 2^24 - 1)                                */
/* ------------------------------------------------------------------------ */
static uint32_t qt_of(const orc_vol* v, float t, int hit)
{
    if (!hit) return 4095u;
    float q = t * v->qv_scale;
    if (!(q < 4095.0f)) return 4095u;
    return (uint32_t)floorf(q);
}

static uint32_t qr_of(float lum)
{
    float c = lum < 5.0f ? lum : 5.0f;
    if (!(c > 0.0f)) return 0u;
    float q = floorf((c * 1023.0f) / 5.0f);
    if (q > 1023.0f) q = 1023.0f;
    return (uint32_t)q;
}

static uint32_t qc_of(const orc_vol* v, const orc_frame* fr, int p)
{
    if (!fr->has_camera) return 1023u;
    float pp[3];
    probe_pos(v, p, pp);
    float dx = pp[0] - fr->cam[0], dy = pp[1] - fr->cam[1], dz = pp[2] - fr->cam[2];
    float dist = sqrtf((dx * dx + dy * dy) + dz * dz);
    if (dist < fr->cam_k) return 1023u;
    float q = (dist - fr->cam_k) * v->qc_scale;
    uint32_t i = (q < 4095.0f) ? (uint32_t)floorf(q) : 4095u;
    return v->lut_c[i];
}

/* Clip volumes (Fig. TrCam(b), Sec. "Improving construction efficiency"):
   with the camera's view-projection matrix M, probe p is inside the
   extended frustum |clip_xy| <= L when w > 0, |c_x| <= L w and |c_y| <= L w
   ((c_x, c_y, -, w) = M (p, 1), FP32 in row order).  V_in: L = 1.2 and f_c
   >= 0.75; V_out: L = 1.4 and f_c >= 0.5, with f_c = q_c / 1023 (q_c >= 768,
   resp. >= 512).  Without a matrix every probe is in V_in. */
static int in_frustum(const float m[16], const float x[3], float L)
{
    float w = ((m[12] * x[0] + m[13] * x[1]) + m[14] * x[2]) + m[15];
    float cx = ((m[0] * x[0] + m[1] * x[1]) + m[2] * x[2]) + m[3];
    float cy = ((m[4] * x[0] + m[5] * x[1]) + m[6] * x[2]) + m[7];
    if (!(w > 0.0f)) return 0;
    float lw = L * w;
    return fabsf(cx) <= lw && fabsf(cy) <= lw;
}

static void classify(orc_vol* v, const orc_frame* fr)
{
    for (int p = 0; p < v->P; ++p) {
        if (!fr->has_clip) {
            v->cls[p] = 2;
            continue;
        }
        float x[3];
        probe_pos(v, p, x);
        uint32_t qc = qc_of(v, fr, p);
        if (qc >= 768u && in_frustum(fr->clip, x, 1.2f))
            v->cls[p] = 2;
        else if (qc >= 512u && in_frustum(fr->clip, x, 1.4f))
            v->cls[p] = 1;
        else
            v->cls[p] = 0;
    }
}

/* The change step of probes [p0, p1) in two parts: change_state (q_v, q_r,
   the pair gradient and the trigger Tr, from each probe's own pilot rays)
   and change_weights (the 5x5x5 x octant sum of Tr over the neighbours and
   the composition into q_d and W_p).  The weights read the neighbours' Tr,
   so with the probes split across ranks the Tr of the neighbouring planes
   must be present before change_weights runs. */
static void change_state(orc_vol* v, const orc_frame* fr, int p0, int p1)
{
    for (int p = p0; p < p1; ++p)
        for (int o = 0; o < 8; ++o) {
            size_t opp = (size_t)p * 8 + (size_t)(7 - o);
            v->qv[(size_t)p * 8 + o] = v->cls[p] ? v->lut_v[qt_of(v, v->pil_t[opp], v->pil_tri[opp] >= 0)] : 0;
            v->qr[(size_t)p * 8 + o] = v->cls[p] ? (uint16_t)qr_of(v->pil_lum[(size_t)p * 8 + o]) : 0;
        }
    const int theta = v->d.theta;
    const int even = (fr->frame & 1u) == 0;
    const int valid = !even && v->last_even == (int64_t)fr->frame - 1;
    for (size_t i = (size_t)p0 * 8; i < (size_t)p1 * 8; ++i) {
        const size_t pi = i / 8;
        if (v->cls[pi] == 0) { /* outside V_out: no heuristics; the state waits */
            v->trv[i] = v->trr[i] = 0;
            continue;
        }
        uint16_t* amp[2] = {&v->amp_v[i], &v->amp_r[i]};
        uint8_t* age[2] = {&v->age_v[i], &v->age_r[i]};
        uint16_t* out[2] = {&v->trv[i], &v->trr[i]};
        int delta[2] = {0, 0};
        if (!even && valid && v->vout_even[pi]) { /* both frames of the pair inside V_out */
            delta[0] = abs((int)v->qv[i] - (int)v->qv_even[i]);
            delta[1] = abs((int)v->qr[i] - (int)v->qr_even[i]);
        }
        for (int c = 0; c < 2; ++c) {
            int a = *age[c];
            if (a < theta) a += 1; /* the running pulse ages by one frame */
            int cur = a < theta ? (int)(((uint32_t)*amp[c] * (uint32_t)(theta - a)) / (uint32_t)theta) : 0;
            if (delta[c] > 0 && delta[c] >= cur) {
                *amp[c] = (uint16_t)delta[c];
                a = 0;
                cur = delta[c];
            }
            *age[c] = (uint8_t)(a < theta ? a : theta);
            *out[c] = (uint16_t)cur;
        }
        if (even) {
            v->qv_even[i] = v->qv[i];
            v->qr_even[i] = v->qr[i];
        }
    }
    if (even)
        for (int p = p0; p < p1; ++p) v->vout_even[p] = v->cls[p] >= 1;
    if (even) v->last_even = (int64_t)fr->frame;
}

static void change_weights(orc_vol* v, const orc_frame* fr, int p0, int p1)
{
    const int X = v->d.dims[0], Y = v->d.dims[1], Z = v->d.dims[2];
    for (int p = p0; p < p1; ++p) {
        int ix = p % X, iy = (p / X) % Y, iz = p / (X * Y);
        uint32_t qc = qc_of(v, fr, p);
        uint64_t Wp = 0;
        for (int o = 0; o < 8; ++o) {
            uint64_t fdv = 0, fdr = 0;
            for (int dz = -2; dz <= 2; ++dz)
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx) {
                        int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                        if (jx < 0 || jy < 0 || jz < 0 || jx >= X || jy >= Y || jz >= Z) continue;
                        size_t q = ((size_t)jx + (size_t)X * ((size_t)jy + (size_t)Y * (size_t)jz)) * 8;
                        const int nb[4] = {o, o ^ 1, o ^ 2, o ^ 4};
                        for (int k = 0; k < 4; ++k) {
                            fdv += v->trv[q + nb[k]];
                            fdr += v->trr[q + nb[k]];
                        }
                    }
            uint64_t qd = ((uint64_t)qc * (uint64_t)v->qv[(size_t)p * 8 + o] * (fdv + 2u * fdr)) >> 20;
            if (v->cls[p] != 2) qd = 0; /* only V_in probes take adaptive samples */
            v->qd[(size_t)p * 8 + o] = (uint32_t)(qd < 0xFFFFFFFFu ? qd : 0xFFFFFFFFu);
            Wp += qd;
        }
        v->W[p] = (uint32_t)(Wp < 0xFFFFFFu ? Wp : 0xFFFFFFu);
    }
}

static void change_detect(orc_vol* v, const orc_frame* fr)
{
    change_state(v, fr, 0, v->P);
    change_weights(v, fr, 0, v->P);
}

/* ------------------------------------------------------------------------ */
/* The per-frame update, in the paper's order (Fig. Method): pilot rays ->  */
/* heuristics -> allocation -> adaptive rays -> cache update.  All shading  */
/* reads the atlases as they were before this frame's blend.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_vol* v;
    const orc_frame* fr;
    int phase;
    int t0, t1;
} job;

/* ------------------------------------------------------------------------ */
/* Metropolis sampling of the adaptive rays (desc.sampler = 1).              */
/*   Guide (Eq. DDGIBays with the static heuristic of Sec. "Adaptive        */
/*   sampling - static"): h(x) = exp(min(alpha g(x) / f_s(x), 1)) f_s(x),    */
/*   f_s = f_c f_v = q_c q_v / 1023^2 (the 10-bit heuristics of the probe   */
/*   and octant of x), g = Rec. 709 luminance of the irradiance texel of x   */
/*   in the previous frame's atlas; h = 0 where f_s = 0.                     */
/*   State x = (grid coordinates g in [0, dims-1]^3, octahedral coordinates */
/*   u in [-1,1]^2); its probe is the nearest grid point, its direction the */
/*   decoded u.  Chains persist across frames (Alg. MarkovChainMT): each     */
/*   frame a chain re-evaluates h at its state and takes M = 8 random-walk  */
/*   steps (Alg. MetropolisStep): Gaussian proposal (sigma 0.5 probe        */
/*   spacings in position, sqrt(pi/256) in u), reflected into the domain;   */
/*   accept when eps <= min(h'/h, 1) (always when h = 0); the states after  */
/*   steps K+1..M-1 (K = 2) are the frame's samples.                         */
/*   Each sample traces its direction w for the irradiance texel at w and   */
/*   the opposite direction -w for the visibility texel at -w (the extra   */
/*   ray of Sec. "Adaptive sampling - static").                             */
/*   Random numbers: SplitMix64 counters; N(0,1) by a 4096-entry quantile   */
/*   table (Phi^-1((i+0.5)/4096), FP64 bisection on erfc, rounded to FP32)  */
/*   indexed by 12 random bits; exp(r), r in [0,1], by a 1024-entry table   */
/*   at r = floor(1023 r)/1023.  Every decision is FP32 with these tables,  */
/*   so two correct implementations agree bit for bit when alpha = 0.       */
/* ------------------------------------------------------------------------ */
static float g_nq[4096], g_ex[1024];
static pthread_once_t g_mh_once = PTHREAD_ONCE_INIT;
static void mh_tables_init(void)
{
    for (int i = 0; i < 4096; ++i) {
        double pr = ((double)i + 0.5) / 4096.0, lo = -10.0, hi = 10.0;
        for (int it = 0; it < 200; ++it) { /* Phi(x) = erfc(-x / sqrt 2) / 2 */
            double mid = 0.5 * (lo + hi);
            if (0.5 * erfc(-mid / sqrt(2.0)) < pr)
                lo = mid;
            else
                hi = mid;
        }
        g_nq[i] = (float)(0.5 * (lo + hi));
    }
    for (int k = 0; k < 1024; ++k) g_ex[k] = (float)exp((double)k / 1023.0);
}
EXPORT float orc_mh_normal_quantile(int i)
{
    pthread_once(&g_mh_once, mh_tables_init);
    return g_nq[i & 4095];
}
EXPORT float orc_mh_exp(int k)
{
    pthread_once(&g_mh_once, mh_tables_init);
    return g_ex[k & 1023];
}

static uint64_t mh_bits(uint64_t seed, uint64_t frame, uint64_t chain, uint64_t step, uint64_t comp)
{
    return hash3(seed ^ 0x4D4554524FULL, frame, (chain * (MH_M + 1) + step) * 8u + comp);
}
static float mh_uniform(uint64_t r) { return (float)(uint32_t)(r >> 40) * 5.9604644775390625e-08f; }
static float mh_normal(uint64_t r) { return g_nq[r >> 52]; }

/* reflect x into [lo, hi] (symmetric proposal), then clamp */
static float mh_reflect(float x, float lo, float hi)
{
    if (x < lo) x = lo + (lo - x);
    if (x > hi) x = hi - (x - hi);
    if (x < lo) x = lo;
    if (x > hi) x = hi;
    return x;
}

static int mh_probe(const orc_vol* v, const float g[3])
{
    int q[3];
    for (int k = 0; k < 3; ++k) {
        int i = (int)floorf(g[k] + 0.5f);
        if (i < 0) i = 0;
        if (i > v->d.dims[k] - 1) i = v->d.dims[k] - 1;
        q[k] = i;
    }
    return q[0] + v->d.dims[0] * (q[1] + v->d.dims[1] * q[2]);
}

/* direction of octahedral coordinates u (FP32, unit length) */
static void mh_dir(const float u[2], float w[3])
{
    float x = u[0], y = u[1];
    float z = (1.0f - fabsf(x)) - fabsf(y);
    if (z < 0.0f) {
        float nx = (1.0f - fabsf(y)) * sgn_f(x);
        float ny = (1.0f - fabsf(x)) * sgn_f(y);
        x = nx;
        y = ny;
    }
    float l = sqrtf((x * x + y * y) + z * z);
    w[0] = x / l;
    w[1] = y / l;
    w[2] = z / l;
}

/* h(x) under this frame's guide */
static float mh_guide(const orc_vol* v, const orc_frame* fr, const float g[3], const float u[2])
{
    int p = mh_probe(v, g);
    if (v->cls[p] != 2) return 0.0f; /* adaptive samples only inside V_in */
    float w[3];
    mh_dir(u, w);
    int o = (w[0] < 0.0f ? 1 : 0) | (w[1] < 0.0f ? 2 : 0) | (w[2] < 0.0f ? 4 : 0);
    uint32_t qc = qc_of(v, fr, p), qv = v->qv[(size_t)p * 8 + (size_t)o];
    float fs = (float)(qc * qv) * (1.0f / 1046529.0f); /* q_c q_v / 1023^2 */
    if (!(fs > 0.0f)) return 0.0f;
    int t = orc_texel_of_dir(w, v->d.n_irr);
    const double* e = v->irr + ((size_t)p * v->Ti * v->Ti + (size_t)t) * 3;
    float gl = (LUM_R * (float)e[0] + LUM_G * (float)e[1]) + LUM_B * (float)e[2];
    float r = (v->d.alpha * gl) / fs;
    if (!(r < 1.0f)) r = 1.0f;
    if (r < 0.0f) r = 0.0f;
    int k = (int)floorf(r * 1023.0f);
    return g_ex[k] * fs;
}

/* M random-walk steps (Alg. MetropolisStep) of a chain in state (g, u) of a
   dims grid, under guide(ctx, g, u), with proposal sigmas sg (grid units)
   and su (octahedral units) and random numbers hash3(key, frame, counter);
   the states after steps K+1..M-1 are written to samples (grid point,
   direction) from index first (up to limit). */
typedef float (*mh_guide_fn)(const void* ctx, const float g[3], const float u[2]);
static uint64_t mh_key_bits(uint64_t key, uint64_t frame, uint64_t chain, uint64_t step, uint64_t comp)
{
    return hash3(key, frame, (chain * (MH_M + 1) + step) * 8u + comp);
}
static void mh_walk(const int dims[3], uint64_t key, uint64_t frame, size_t c, float sg, float su, float* g, float* u,
                    mh_guide_fn guide, const void* ctx, int* smp_p, float* smp_dir, size_t first, size_t limit)
{
    float y = guide(ctx, g, u);
    for (int i = 0; i < MH_M; ++i) {
        float g2[3], u2[2];
        for (int k = 0; k < 3; ++k)
            g2[k] = mh_reflect(g[k] + sg * mh_normal(mh_key_bits(key, frame, c, (uint64_t)i, (uint64_t)k)), 0.0f,
                               (float)(dims[k] - 1));
        for (int k = 0; k < 2; ++k)
            u2[k] = mh_reflect(u[k] + su * mh_normal(mh_key_bits(key, frame, c, (uint64_t)i, (uint64_t)(3 + k))),
                               -1.0f, 1.0f);
        float y2 = guide(ctx, g2, u2);
        int accept = 1;
        if (y > 0.0f) {
            float mu = y2 / y;
            float eps = mh_uniform(mh_key_bits(key, frame, c, (uint64_t)i, 5u));
            if (mu < 1.0f && eps > mu) accept = 0;
        }
        if (accept) {
            for (int k = 0; k < 3; ++k) g[k] = g2[k];
            u[0] = u2[0];
            u[1] = u2[1];
            y = y2;
        }
        if (i > MH_K) { /* the state after step i is sample i - K - 1 of the chain */
            size_t sidx = first + (size_t)(i - MH_K - 1);
            if (sidx < limit) {
                int q[3];
                for (int k = 0; k < 3; ++k) {
                    int t = (int)floorf(g[k] + 0.5f);
                    q[k] = t < 0 ? 0 : (t > dims[k] - 1 ? dims[k] - 1 : t);
                }
                smp_p[sidx] = q[0] + dims[0] * (q[1] + dims[1] * q[2]);
                mh_dir(u, smp_dir + sidx * 3);
            }
        }
    }
}

typedef struct {
    const orc_vol* v;
    const orc_frame* fr;
} mh_vol_ctx;
static float mh_vol_guide(const void* ctx, const float g[3], const float u[2])
{
    const mh_vol_ctx* c = (const mh_vol_ctx*)ctx;
    return mh_guide(c->v, c->fr, g, u);
}

/* chain c of the volume: this frame's steps and samples */
static void mh_chain(orc_vol* v, const orc_frame* fr, size_t c)
{
    mh_vol_ctx ctx = {v, fr};
    mh_walk(v->d.dims, fr->seed ^ 0x4D4554524FULL, fr->frame, c, MH_SG, MH_SU, v->ch_g + c * 3, v->ch_u + c * 2,
            mh_vol_guide, &ctx, v->smp_p, v->smp_dir, c * MH_S, v->B);
}

/* Test hook: chains on a fixed guide h(probe, octant) given as a table
   (piecewise constant), for `frames` frames of M steps; counts[probe*8 +
   octant] receives the samples of frames >= skip. */
typedef struct {
    const int* dims;
    const float* table;
} mh_tab_ctx;
static float mh_tab_guide(const void* ctx, const float g[3], const float u[2])
{
    const mh_tab_ctx* c = (const mh_tab_ctx*)ctx;
    int q[3];
    for (int k = 0; k < 3; ++k) {
        int t = (int)floorf(g[k] + 0.5f);
        q[k] = t < 0 ? 0 : (t > c->dims[k] - 1 ? c->dims[k] - 1 : t);
    }
    float w[3];
    mh_dir(u, w);
    int o = (w[0] < 0.0f ? 1 : 0) | (w[1] < 0.0f ? 2 : 0) | (w[2] < 0.0f ? 4 : 0);
    return c->table[(size_t)(q[0] + c->dims[0] * (q[1] + c->dims[1] * q[2])) * 8 + (size_t)o];
}
EXPORT void orc_mh_run_table(const int dims[3], const float* table, int chains, int frames, int skip, uint64_t seed,
                             double* counts)
{
    pthread_once(&g_mh_once, mh_tables_init);
    mh_tab_ctx ctx = {dims, table};
    float* g = (float*)malloc(sizeof(float) * 3 * (size_t)chains);
    float* u = (float*)malloc(sizeof(float) * 2 * (size_t)chains);
    int* sp = (int*)malloc(sizeof(int) * MH_S);
    float* sd = (float*)malloc(sizeof(float) * 3 * MH_S);
    for (int c = 0; c < chains; ++c) {
        for (int k = 0; k < 3; ++k)
            g[c * 3 + k] = mh_uniform(mh_bits(seed ^ 0x494E4954ULL, 0, (uint64_t)c, MH_M, (uint64_t)k)) *
                           (float)(dims[k] - 1);
        for (int k = 0; k < 2; ++k)
            u[c * 2 + k] = mh_uniform(mh_bits(seed ^ 0x494E4954ULL, 0, (uint64_t)c, MH_M, (uint64_t)(3 + k))) * 2.0f - 1.0f;
    }
    for (int f = 0; f < frames; ++f)
        for (int c = 0; c < chains; ++c) {
            mh_walk(dims, seed ^ 0x4D4554524FULL, (uint64_t)f, (size_t)c, MH_SG, MH_SU, g + c * 3, u + c * 2,
                    mh_tab_guide, &ctx, sp, sd, 0, MH_S);
            if (f < skip) continue;
            for (int j = 0; j < MH_S; ++j) {
                const float* d = sd + 3 * j;
                int o = (d[0] < 0.0f ? 1 : 0) | (d[1] < 0.0f ? 2 : 0) | (d[2] < 0.0f ? 4 : 0);
                counts[(size_t)sp[j] * 8 + (size_t)o] += 1.0;
            }
        }
    free(g);
    free(u);
    free(sp);
    free(sd);
}

static void mh_init(orc_vol* v, uint64_t seed)
{
    for (size_t c = 0; c < v->C; ++c) {
        for (int k = 0; k < 3; ++k)
            v->ch_g[c * 3 + k] = mh_uniform(mh_bits(seed ^ 0x494E4954ULL, 0, c, MH_M, (uint64_t)k)) *
                                 (float)(v->d.dims[k] - 1);
        for (int k = 0; k < 2; ++k)
            v->ch_u[c * 2 + k] = mh_uniform(mh_bits(seed ^ 0x494E4954ULL, 0, c, MH_M, (uint64_t)(3 + k))) * 2.0f - 1.0f;
    }
    v->chains_live = 1;
}

static int octant_of(const float w[3]) { return (w[0] < 0.0f ? 1 : 0) | (w[1] < 0.0f ? 2 : 0) | (w[2] < 0.0f ? 4 : 0); }

/* direction through the centre of interior texel (cx, cy) of an n x n
   octahedral grid: u = (c + 1/2)/n * 2 - 1 per axis, FP32 in that order,
   decoded like a chain state */
static void texel_centre_dir(int cx, int cy, int n, float w[3])
{
    float u[2] = {(((float)cx + 0.5f) / (float)n) * 2.0f - 1.0f, (((float)cy + 0.5f) / (float)n) * 2.0f - 1.0f};
    mh_dir(u, w);
}

/* the centre direction of the texel a direction bins to (n x n interior) */
static void snap_to_texel(const float d[3], int n, float w[3])
{
    int t = orc_texel_of_dir(d, n), T = n + 2;
    texel_centre_dir(t % T - 1, t / T - 1, n, w);
}

/* trace and shade sample s: +w for radiance, -w for the visibility distance.
   With the dynamic chains on, a sample whose probe and octant carry a
   dynamic weight (q_d > 0) traces through texel centres instead: +w through
   the centre of its irradiance texel, -w through the centre of the
   visibility texel of -w (Sec. "Adaptive sampling - dynamic", last
   paragraph), so that it adds no sampling noise there. */
static void mh_sample_rays(orc_vol* v, const orc_frame* fr, size_t sidx)
{
    if (v->cls[v->smp_p[sidx]] != 2) { /* outside V_in: the sample is dropped (no rays, not blended) */
        v->smp_t[sidx] = v->smp_tn[sidx] = INFINITY;
        v->smp_tri[sidx] = v->smp_trin[sidx] = -1;
        v->smp_rad[sidx * 3] = v->smp_rad[sidx * 3 + 1] = v->smp_rad[sidx * 3 + 2] = 0.0;
        v->smp_dep[sidx] = v->depth_max;
        return;
    }
    float o[3];
    probe_pos(v, v->smp_p[sidx], o);
    const float* d0 = v->smp_dir + sidx * 3;
    float d[3] = {d0[0], d0[1], d0[2]}, dn[3] = {-d0[0], -d0[1], -d0[2]};
    if (v->d.dyn_ratio > 0 && v->qd[(size_t)v->smp_p[sidx] * 8 + (size_t)octant_of(d0)] > 0) {
        snap_to_texel(d0, v->d.n_irr, d);
        float m[3] = {-d0[0], -d0[1], -d0[2]};
        snap_to_texel(m, v->d.n_dep, dn);
    }
    hitrec h = vol_closest(v, o, d, v->tmin, INFINITY);
    v->smp_t[sidx] = h.tri >= 0 ? h.t : INFINITY;
    v->smp_tri[sidx] = h.tri;
    double dep_unused;
    shade_ray(v, fr, o, d, h, v->smp_rad + sidx * 3, &dep_unused, NULL);
    hitrec hn = vol_closest(v, o, dn, v->tmin, INFINITY);
    v->smp_tn[sidx] = hn.tri >= 0 ? hn.t : INFINITY;
    v->smp_trin[sidx] = hn.tri;
    v->smp_dep[sidx] = hn.tri >= 0 ? (hn.t < v->depth_max ? hn.t : v->depth_max) : v->depth_max;
}


/* ------------------------------------------------------------------------ */
/* Dynamic chains over virtual proxies (desc.dyn_ratio > 0; Sec. "Adaptive */
/* sampling - dynamic").                                                    */
/*   A proxy stands for a 3x3x3 block of probes (clipped at the grid end); */
/*   its value in octant o is the max of q_d over its probes (the coarsened */
/*   f_d), and the guide is that value with alpha = 0 (no cache term).     */
/*   The chains walk proxy-grid coordinates and octahedral coordinates with */
/*   steps 3x and 6x those of the static chains, 8 steps per frame, the     */
/*   states after steps 3..7 being the samples (as the static chains).      */
/*   A sample marks its (proxy, octant) cell when the guide there is > 0;   */
/*   a cell is marked once per frame, by its first sample.  Marked cells in */
/*   first-sample order are traced while the running ray count stays within */
/*   the dynamic budget; a traced cell sends, from each of its probes, one  */
/*   ray through the centre of every irradiance texel whose centre lies in  */
/*   the octant (deterministic directions).  Each such ray updates its      */
/*   irradiance texel and the visibility texel of its direction, in a       */
/*   second batched step after the static samples, with hysteresis          */
/*   hyst_dyn.  Budget: the adaptive samples B are split r:1; the static    */
/*   chains draw B_s = floor(B r/(r+1)) samples, the dynamic rays get the   */
/*   remaining 2(B - B_s) rays (a static sample traces two rays); there are */
/*   ceil(C_s / r) dynamic chains (the paper's 4096:1024 at r = 4).          */
/* ------------------------------------------------------------------------ */
#define DYN_KEY 0x44594E414DULL /* 'DYNAM' */

static void dyn_create(orc_vol* v)
{
    for (int k = 0; k < 3; ++k) v->Dp[k] = (v->d.dims[k] + 2) / 3;
    v->Pp = v->Dp[0] * v->Dp[1] * v->Dp[2];
    size_t r = (size_t)v->d.dyn_ratio;
    v->Cd = v->C ? (v->C + r - 1) / r : 0;
    v->Bd = v->Cd * MH_S;
    v->dch_g = (float*)calloc(v->Cd * 3 + 1, 4);
    v->dch_u = (float*)calloc(v->Cd * 2 + 1, 4);
    v->dsm_q = (int*)calloc(v->Bd + 1, 4);
    v->dsm_dir = (float*)calloc(v->Bd * 3 + 1, 4);
    v->dsm_cell = (int*)calloc(v->Bd + 1, 4);
    v->dfirst = (uint32_t*)calloc((size_t)v->Pp * 8, 4);
    v->dmark = (int*)calloc((size_t)v->Pp * 8, 4);
    v->dincl = (uint8_t*)calloc((size_t)v->Pp * 8, 1);
    const int n = v->d.n_irr, T = n + 2;
    v->tex_t = (int*)calloc((size_t)8 * n * n, 4);
    v->tex_dir = (float*)calloc((size_t)8 * n * n * 3, 4);
    for (int cy = 0; cy < n; ++cy)
        for (int cx = 0; cx < n; ++cx) {
            float w[3];
            texel_centre_dir(cx, cy, n, w);
            int o = octant_of(w), j = v->ntex[o]++;
            v->tex_t[o * n * n + j] = (cy + 1) * T + (cx + 1);
            memcpy(v->tex_dir + ((size_t)o * n * n + (size_t)j) * 3, w, sizeof(w));
        }
    v->doff = (uint32_t*)calloc((size_t)v->P + 1, 4);
    v->d_p = (int*)calloc(v->Rd + 1, 4);
    v->d_k = (int*)calloc(v->Rd + 1, 4);
    v->d_t = (float*)calloc(v->Rd + 1, 4);
    v->d_tri = (int*)calloc(v->Rd + 1, 4);
    v->d_rad = (double*)calloc(v->Rd * 3 + 1, 8);
    v->d_dep = (double*)calloc(v->Rd + 1, 8);
}

static void dyn_init(orc_vol* v, uint64_t seed)
{
    for (size_t c = 0; c < v->Cd; ++c) {
        for (int k = 0; k < 3; ++k)
            v->dch_g[c * 3 + k] =
                mh_uniform(mh_key_bits(seed ^ DYN_KEY ^ 0x494E4954ULL, 0, c, MH_M, (uint64_t)k)) * (float)(v->Dp[k] - 1);
        for (int k = 0; k < 2; ++k)
            v->dch_u[c * 2 + k] =
                mh_uniform(mh_key_bits(seed ^ DYN_KEY ^ 0x494E4954ULL, 0, c, MH_M, (uint64_t)(3 + k))) * 2.0f - 1.0f;
    }
    v->dyn_live = 1;
}

/* coarsened dynamic target of proxy q in octant o: max of q_d over its probes */
static uint32_t dyn_value(const orc_vol* v, int q, int o)
{
    const int X = v->d.dims[0], Y = v->d.dims[1], Z = v->d.dims[2];
    int qx = q % v->Dp[0], qy = (q / v->Dp[0]) % v->Dp[1], qz = q / (v->Dp[0] * v->Dp[1]);
    uint32_t m = 0;
    for (int z = 3 * qz; z < 3 * qz + 3 && z < Z; ++z)
        for (int y = 3 * qy; y < 3 * qy + 3 && y < Y; ++y)
            for (int x = 3 * qx; x < 3 * qx + 3 && x < X; ++x) {
                uint32_t w = v->qd[((size_t)x + (size_t)X * ((size_t)y + (size_t)Y * (size_t)z)) * 8 + (size_t)o];
                if (w > m) m = w;
            }
    return m;
}

static int dyn_proxy_of(const orc_vol* v, const float g[3])
{
    int q[3];
    for (int k = 0; k < 3; ++k) {
        int i = (int)floorf(g[k] + 0.5f);
        q[k] = i < 0 ? 0 : (i > v->Dp[k] - 1 ? v->Dp[k] - 1 : i);
    }
    return q[0] + v->Dp[0] * (q[1] + v->Dp[1] * q[2]);
}

static float dyn_guide(const void* ctx, const float g[3], const float u[2])
{
    const orc_vol* v = (const orc_vol*)ctx;
    float w[3];
    mh_dir(u, w);
    return (float)dyn_value(v, dyn_proxy_of(v, g), octant_of(w));
}

static void dyn_chain(orc_vol* v, const orc_frame* fr, size_t c)
{
    mh_walk(v->Dp, fr->seed ^ DYN_KEY, fr->frame, c, DYN_SG, DYN_SU, v->dch_g + c * 3, v->dch_u + c * 2, dyn_guide, v,
            v->dsm_q, v->dsm_dir, c * MH_S, v->Bd);
}

/* probes of proxy q inside V_in (index order) */
static int dyn_probes(const orc_vol* v, int q, int* out)
{
    const int X = v->d.dims[0], Y = v->d.dims[1], Z = v->d.dims[2];
    int qx = q % v->Dp[0], qy = (q / v->Dp[0]) % v->Dp[1], qz = q / (v->Dp[0] * v->Dp[1]), n = 0;
    for (int z = 3 * qz; z < 3 * qz + 3 && z < Z; ++z)
        for (int y = 3 * qy; y < 3 * qy + 3 && y < Y; ++y)
            for (int x = 3 * qx; x < 3 * qx + 3 && x < X; ++x) {
                int p = x + X * (y + Y * z);
                if (v->cls[p] == 2) out[n++] = p;
            }
    return n;
}

/* marks, the budget, and this frame's dynamic rays grouped by probe */
static void dyn_marks(orc_vol* v)
{
    const size_t cells = (size_t)v->Pp * 8;
    for (size_t k = 0; k < cells; ++k) v->dfirst[k] = UINT32_MAX;
    for (size_t sidx = 0; sidx < v->Bd; ++sidx) {
        const int o = octant_of(v->dsm_dir + sidx * 3), q = v->dsm_q[sidx];
        int cell = dyn_value(v, q, o) > 0 ? q * 8 + o : -1;
        v->dsm_cell[sidx] = cell;
        if (cell >= 0 && v->dfirst[cell] == UINT32_MAX) v->dfirst[cell] = (uint32_t)sidx;
    }
    /* marked cells in first-sample order (each sample marks at most one cell) */
    v->n_marked = 0;
    for (size_t sidx = 0; sidx < v->Bd; ++sidx) {
        int cell = v->dsm_cell[sidx];
        if (cell >= 0 && v->dfirst[cell] == (uint32_t)sidx) v->dmark[v->n_marked++] = cell;
    }
    memset(v->dincl, 0, cells);
    size_t used = 0;
    int pr[27];
    v->n_incl = 0;
    for (int m = 0; m < v->n_marked; ++m) {
        int cell = v->dmark[m];
        size_t rays = (size_t)dyn_probes(v, cell / 8, pr) * (size_t)v->ntex[cell % 8];
        if (used + rays > v->Rd) break;
        used += rays;
        v->dincl[cell] = 1;
        v->n_incl++;
    }
    /* rays grouped by probe: octants in order, texels in the octant's list order */
    const int X = v->d.dims[0], Y = v->d.dims[1], nn = v->d.n_irr * v->d.n_irr;
    size_t r = 0;
    for (int p = 0; p < v->P; ++p) {
        v->doff[p] = (uint32_t)r;
        if (v->cls[p] != 2) continue; /* dynamic rays only from V_in probes */
        int ix = p % X, iy = (p / X) % Y, iz = p / (X * Y);
        int q = (ix / 3) + v->Dp[0] * ((iy / 3) + v->Dp[1] * (iz / 3));
        for (int o = 0; o < 8; ++o) {
            if (!v->dincl[q * 8 + o]) continue;
            for (int j = 0; j < v->ntex[o]; ++j, ++r) {
                v->d_p[r] = p;
                v->d_k[r] = o * nn + j;
            }
        }
    }
    v->doff[v->P] = (uint32_t)r;
    v->Rdyn = r;
}

static void dyn_ray(orc_vol* v, const orc_frame* fr, size_t r)
{
    float o[3];
    probe_pos(v, v->d_p[r], o);
    const float* d = v->tex_dir + (size_t)v->d_k[r] * 3;
    hitrec h = vol_closest(v, o, d, v->tmin, INFINITY);
    v->d_t[r] = h.tri >= 0 ? h.t : INFINITY;
    v->d_tri[r] = h.tri;
    shade_ray(v, fr, o, d, h, v->d_rad + r * 3, v->d_dep + r, NULL);
}

/* the samples of each probe, in sample order (counting sort by probe) */
static void mh_group(orc_vol* v)
{
    memset(v->smp_off, 0, sizeof(uint32_t) * ((size_t)v->P + 1));
    for (size_t sidx = 0; sidx < v->B; ++sidx) v->smp_off[v->smp_p[sidx] + 1] += 1u;
    for (int p = 0; p < v->P; ++p) v->smp_off[p + 1] += v->smp_off[p];
    uint32_t* cur = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)v->P);
    memcpy(cur, v->smp_off, sizeof(uint32_t) * (size_t)v->P);
    for (size_t sidx = 0; sidx < v->B; ++sidx) v->smp_ord[cur[v->smp_p[sidx]]++] = (uint32_t)sidx;
    free(cur);
}

/* blend probe p: pilots (even frames), then its samples in sample order;
   irradiance texel at w, visibility texel at -w; the batched moving average
   of blend_probe */
static void mh_blend_probe(orc_vol* v, int p, int use_pilots, double h)
{
    const int Ti = v->Ti, Td = v->Td, ni = v->d.n_irr, nd = v->d.n_dep;
    double* irr = v->irr + (size_t)p * Ti * Ti * 3;
    uint8_t* irn = v->irr_n + (size_t)p * Ti * Ti;
    double* dep = v->dep + (size_t)p * Td * Td * 2;
    uint8_t* den = v->dep_n + (size_t)p * Td * Td;
    double* si = (double*)calloc((size_t)Ti * Ti * 3, sizeof(double));
    int* ki = (int*)calloc((size_t)Ti * Ti, sizeof(int));
    double* sd = (double*)calloc((size_t)Td * Td * 2, sizeof(double));
    int* kd = (int*)calloc((size_t)Td * Td, sizeof(int));
    if (use_pilots)
        for (int j = 0; j < 8; ++j) {
            const float* d = v->pil_dir + ((size_t)p * 8 + (size_t)j) * 3;
            const double* rad = v->pil_rad + ((size_t)p * 8 + (size_t)j) * 3;
            double ds = v->pil_dep[(size_t)p * 8 + (size_t)j];
            int ti = orc_texel_of_dir(d, ni), td = orc_texel_of_dir(d, nd);
            for (int c = 0; c < 3; ++c) si[ti * 3 + c] += rad[c];
            ki[ti] += 1;
            sd[td * 2 + 0] += ds;
            sd[td * 2 + 1] += ds * ds;
            kd[td] += 1;
        }
    for (uint32_t q = v->smp_off[p]; q < v->smp_off[p + 1] && v->cls[p] == 2; ++q) {
        size_t sidx = v->smp_ord[q];
        const float* d = v->smp_dir + sidx * 3;
        float dn[3] = {-d[0], -d[1], -d[2]};
        int ti = orc_texel_of_dir(d, ni), td = orc_texel_of_dir(dn, nd);
        for (int c = 0; c < 3; ++c) si[ti * 3 + c] += v->smp_rad[sidx * 3 + c];
        ki[ti] += 1;
        double ds = v->smp_dep[sidx];
        sd[td * 2 + 0] += ds;
        sd[td * 2 + 1] += ds * ds;
        kd[td] += 1;
    }
    batch_apply(irr, irn, si, ki, Ti * Ti, 3, h);
    batch_apply(dep, den, sd, kd, Td * Td, 2, h);
    if (v->d.dyn_ratio > 0) { /* then the dynamic rays of the probe, a second batch with hyst_dyn */
        memset(si, 0, sizeof(double) * (size_t)Ti * Ti * 3);
        memset(ki, 0, sizeof(int) * (size_t)Ti * Ti);
        memset(sd, 0, sizeof(double) * (size_t)Td * Td * 2);
        memset(kd, 0, sizeof(int) * (size_t)Td * Td);
        for (uint32_t r = v->doff[p]; r < v->doff[p + 1]; ++r) {
            const float* d = v->tex_dir + (size_t)v->d_k[r] * 3;
            int ti = orc_texel_of_dir(d, ni), td = orc_texel_of_dir(d, nd);
            for (int c = 0; c < 3; ++c) si[ti * 3 + c] += v->d_rad[(size_t)r * 3 + c];
            ki[ti] += 1;
            double ds = v->d_dep[r];
            sd[td * 2 + 0] += ds;
            sd[td * 2 + 1] += ds * ds;
            kd[td] += 1;
        }
        batch_apply(irr, irn, si, ki, Ti * Ti, 3, (double)v->d.hyst_dyn);
        batch_apply(dep, den, sd, kd, Td * Td, 2, (double)v->d.hyst_dyn);
    }
    if (v->cls[p] == 1) { /* V_out - V_in: sample counts set down to 16 (catch-up) */
        for (int t = 0; t < Ti * Ti; ++t)
            if (irn[t] > 16) irn[t] = 16;
        for (int t = 0; t < Td * Td; ++t)
            if (den[t] > 16) den[t] = 16;
    }
    border_copy(irr, irn, ni, 3);
    border_copy(dep, den, nd, 2);
    free(si);
    free(ki);
    free(sd);
    free(kd);
}

/* DDGI's cosine-gather blend (Sec. 3.1; the variant of the texel update):
   every ray of the probe contributes to every texel of its hemisphere.  For
   interior texel t with centre direction n_t (the FP32 decode of the texel
   centre, as the dynamic rays') and ray r of direction w_r, c = n_t . w_r
   (the test c > 0 in FP32, ((x x' + y y') + z z'); the weights in FP64,
   at least 0): the irradiance
   texel takes the c-weighted mean of the rays' radiance over c > 0, the
   visibility texel the c^50-weighted mean of {d, d^2} (DDGI's depth
   sharpness 50); k = the number of rays with c > 0 enters the batched
   moving average as the sample count (w = max(1 - h, k/(n + k))). */
#define COS_DEPTH_SHARPNESS 50
static void texel_centre_dir(int cx, int cy, int n, float w[3]);
static void blend_probe_cos(orc_vol* v, int p, int use_pilots, double h)
{
    const int Ti = v->Ti, Td = v->Td, ni = v->d.n_irr, nd = v->d.n_dep;
    double* irr = v->irr + (size_t)p * Ti * Ti * 3;
    uint8_t* irn = v->irr_n + (size_t)p * Ti * Ti;
    double* dep = v->dep + (size_t)p * Td * Td * 2;
    uint8_t* den = v->dep_n + (size_t)p * Td * Td;
    const uint32_t mp = v->n[p] > 8u ? v->n[p] - 8u : 0u;
    const int total = (int)mp + (use_pilots ? 8 : 0);
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)(total + 1));
    const double** rads = (const double**)malloc(sizeof(double*) * (size_t)(total + 1));
    double* deps = (double*)malloc(sizeof(double) * (size_t)(total + 1));
    for (int j = 0; j < total; ++j) {
        float d[3];
        if (use_pilots && j < 8) {
            const float* pd = v->pil_dir + ((size_t)p * 8 + (size_t)j) * 3;
            d[0] = pd[0];
            d[1] = pd[1];
            d[2] = pd[2];
            rads[j] = v->pil_rad + ((size_t)p * 8 + (size_t)j) * 3;
            deps[j] = v->pil_dep[(size_t)p * 8 + (size_t)j];
        } else {
            int i = use_pilots ? j - 8 : j;
            main_dir(v, (int)mp, i, d);
            size_t r = (size_t)v->off[p] + (size_t)i;
            rads[j] = v->m_rad + r * 3;
            deps[j] = v->m_dep[r];
        }
        for (int c = 0; c < 3; ++c) dirs[j * 3 + c] = d[c];
    }
    double* si = (double*)calloc((size_t)Ti * Ti * 3, sizeof(double));
    int* ki = (int*)calloc((size_t)Ti * Ti, sizeof(int));
    double* sd = (double*)calloc((size_t)Td * Td * 2, sizeof(double));
    int* kd = (int*)calloc((size_t)Td * Td, sizeof(int));
    for (int pass = 0; pass < 2; ++pass) {
        const int n = pass ? nd : ni, T = n + 2;
        for (int cy = 0; cy < n; ++cy)
            for (int cx = 0; cx < n; ++cx) {
                const int t = (cy + 1) * T + (cx + 1);
                float nt[3];
                texel_centre_dir(cx, cy, n, nt);
                double sw = 0.0, acc[3] = {0.0, 0.0, 0.0}, cmax = 0.0;
                int k = 0;
                if (pass) /* the depth weights relative to the largest c: the same mean, no underflow */
                    for (int j = 0; j < total; ++j) {
                        const float c32 = (nt[0] * (float)dirs[j * 3] + nt[1] * (float)dirs[j * 3 + 1]) +
                                          nt[2] * (float)dirs[j * 3 + 2];
                        double c = (double)nt[0] * dirs[j * 3] + (double)nt[1] * dirs[j * 3 + 1] +
                                   (double)nt[2] * dirs[j * 3 + 2];
                        if (c32 > 0.0f && c > cmax) cmax = c;
                    }
                for (int j = 0; j < total; ++j) {
                    const float c32 = (nt[0] * (float)dirs[j * 3] + nt[1] * (float)dirs[j * 3 + 1]) +
                                      nt[2] * (float)dirs[j * 3 + 2];
                    if (!(c32 > 0.0f)) continue;
                    ++k;
                    double c = (double)nt[0] * dirs[j * 3] + (double)nt[1] * dirs[j * 3 + 1] + (double)nt[2] * dirs[j * 3 + 2];
                    if (c < 0.0) c = 0.0;
                    if (!pass) {
                        sw += c;
                        for (int q = 0; q < 3; ++q) acc[q] += c * rads[j][q];
                    } else {
                        double wgt = cmax > 0.0 ? pow(c / cmax, COS_DEPTH_SHARPNESS) : 1.0;
                        sw += wgt;
                        acc[0] += wgt * deps[j];
                        acc[1] += wgt * deps[j] * deps[j];
                    }
                }
                if (!k || !(sw > 0.0)) continue;
                /* the weighted mean times k: batch_apply divides the sums by k */
                if (!pass) {
                    for (int q = 0; q < 3; ++q) si[t * 3 + q] = acc[q] / sw * k;
                    ki[t] = k;
                } else {
                    sd[t * 2] = acc[0] / sw * k;
                    sd[t * 2 + 1] = acc[1] / sw * k;
                    kd[t] = k;
                }
            }
    }
    batch_apply(irr, irn, si, ki, Ti * Ti, 3, h);
    batch_apply(dep, den, sd, kd, Td * Td, 2, h);
    if (v->cls[p] == 1) {
        for (int t = 0; t < Ti * Ti; ++t)
            if (irn[t] > 16) irn[t] = 16;
        for (int t = 0; t < Td * Td; ++t)
            if (den[t] > 16) den[t] = 16;
    }
    border_copy(irr, irn, ni, 3);
    border_copy(dep, den, nd, 2);
    free(si);
    free(ki);
    free(sd);
    free(kd);
    free(dirs);
    free(rads);
    free(deps);
}

static void pilot_probe(orc_vol* v, const orc_frame* fr, int p)
{
    if (v->cls[p] == 0) { /* outside V_out: no pilot rays (records: a miss with nothing gathered) */
        for (int k = 0; k < 8; ++k) {
            size_t i = (size_t)p * 8 + (size_t)k;
            orc_pilot_dir(fr->seed, fr->frame, (uint32_t)p, k, v->pil_dir + i * 3);
            v->pil_t[i] = INFINITY;
            v->pil_tri[i] = -1;
            v->pil_lum[i] = 0.0f;
            v->pil_rad[i * 3] = v->pil_rad[i * 3 + 1] = v->pil_rad[i * 3 + 2] = 0.0;
            v->pil_dep[i] = v->depth_max;
        }
        return;
    }
    float o[3];
    probe_pos(v, p, o);
    for (int k = 0; k < 8; ++k) {
        size_t i = (size_t)p * 8 + (size_t)k;
        float* d = v->pil_dir + i * 3;
        orc_pilot_dir(fr->seed, fr->frame, (uint32_t)p, k, d);
        hitrec h = vol_closest(v, o, d, v->tmin, INFINITY);
        v->pil_t[i] = h.tri >= 0 ? h.t : INFINITY;
        v->pil_tri[i] = h.tri;
        shade_ray(v, fr, o, d, h, v->pil_rad + i * 3, v->pil_dep + i, v->pil_lum + i);
    }
}

static void main_probe(orc_vol* v, const orc_frame* fr, int p)
{
    float o[3];
    probe_pos(v, p, o);
    int mp = v->n[p] > 8u ? (int)v->n[p] - 8 : 0;
    for (int i = 0; i < mp; ++i) {
        float d[3];
        main_dir(v, mp, i, d);
        size_t r = (size_t)v->off[p] + (size_t)i;
        hitrec h = vol_closest(v, o, d, v->tmin, INFINITY);
        v->m_t[r] = h.tri >= 0 ? h.t : INFINITY;
        v->m_tri[r] = h.tri;
        shade_ray(v, fr, o, d, h, v->m_rad + r * 3, v->m_dep + r, NULL);
    }
}

static void* worker(void* arg)
{
    job* j = (job*)arg;
    for (int p = j->t0; p < j->t1; ++p) {
        if (j->phase == 3)
            mh_chain(j->v, j->fr, (size_t)p);
        else if (j->phase == 4)
            mh_sample_rays(j->v, j->fr, (size_t)p);
        else if (j->phase == 5)
            mh_blend_probe(j->v, p, (j->fr->frame & 1u) == 0 && j->v->cls[p] >= 1, (double)j->v->d.hyst);
        else if (j->phase == 6)
            dyn_chain(j->v, j->fr, (size_t)p);
        else if (j->phase == 7)
            dyn_ray(j->v, j->fr, (size_t)p);
        else if (j->phase == 0)
            pilot_probe(j->v, j->fr, p);  /* outside V_out: no pilot rays (see pilot_probe) */
        else if (j->phase == 1)
            main_probe(j->v, j->fr, p);
        else
            if (j->v->d.packed)
                blend_probe_packed(j->v, p, (j->fr->frame & 1u) == 0 && j->v->cls[p] >= 1);
            else if (j->v->d.blend_mode == 1)
                blend_probe_cos(j->v, p, (j->fr->frame & 1u) == 0 && j->v->cls[p] >= 1, (double)j->v->d.hyst);
            else
                blend_probe(j->v, p, (j->fr->frame & 1u) == 0 && j->v->cls[p] >= 1, (double)j->v->d.hyst);
    }
    return NULL;
}

/* a phase over items [lo, hi), split evenly over the threads */
static void run_phase_range(orc_vol* v, const orc_frame* fr, int phase, long long lo, long long hi)
{
    const long long N = hi - lo;
    if (N <= 0) return;
    int nt = v->nthreads;
    if (nt > N) nt = (int)N;
    pthread_t th[256];
    job jobs[256];
    if (nt > 256) nt = 256;
    for (int t = 0; t < nt; ++t) {
        jobs[t].v = v;
        jobs[t].fr = fr;
        jobs[t].phase = phase;
        jobs[t].t0 = (int)(lo + N * t / nt);
        jobs[t].t1 = (int)(lo + N * (t + 1) / nt);
    }
    if (nt == 1) {
        worker(&jobs[0]);
        return;
    }
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
}

static void run_phase(orc_vol* v, const orc_frame* fr, int phase)
{
    /* phases 3 and 4 run over chains and samples, 6 and 7 over dynamic
       chains and rays, the others over probes */
    const long long N = phase == 3   ? (long long)v->C
                        : phase == 4 ? (long long)v->B
                        : phase == 6 ? (long long)v->Cd
                        : phase == 7 ? (long long)v->Rdyn
                                     : (long long)v->P;
    run_phase_range(v, fr, phase, 0, N);
}

EXPORT int orc_update(orc_vol* v, const orc_frame* fr)
{
    if (v->bvh_dirty) {
        if (cbvh_build(&v->bvh, v->V, v->nv, v->I, v->nt)) return -1;
        v->bvh_dirty = 0;
    }
    orc_frame_rotation(fr->seed, fr->frame, v->R);
    classify(v, fr);
    run_phase(v, fr, 0);
    change_detect(v, fr);
    if (orc_allocate_masked(v->W, v->cls, v->P, v->d.avg, v->d.rmin, v->d.rmax, v->n, v->off)) return -1;
    if (v->d.sampler == 1) { /* Metropolis chains instead of the per-probe allocation */
        pthread_once(&g_mh_once, mh_tables_init);
        if (!v->chains_live) mh_init(v, fr->seed);
        run_phase(v, fr, 3);
        run_phase(v, fr, 4);
        mh_group(v);
        if (v->d.dyn_ratio > 0) { /* the dynamic chains run after the static ones */
            if (!v->dyn_live) dyn_init(v, fr->seed);
            run_phase(v, fr, 6);
            dyn_marks(v);
            run_phase(v, fr, 7);
        }
        run_phase(v, fr, 5);
        return 0;
    }
    run_phase(v, fr, 1);
    run_phase(v, fr, 2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Probe-slab split of one update over ranks (the multi-GPU form of the     */
/* deterministic mode).  A rank owns probes [p0, p1) and keeps full-size    */
/* arrays; per frame:                                                        */
/*   orc_slab_begin    rotation, clip classes of every probe, the pilot     */
/*                     rays of its probes and their change state (q, Tr);   */
/*   (the ranks exchange Tr of the two planes beside each slab border)      */
/*   orc_slab_weights  W_p of its probes (5x5x5 x octant sum);              */
/*   (the ranks all-gather W)                                               */
/*   orc_slab_finish   the allocation of the whole budget over all W (every */
/*                     rank computes the same integers), the adaptive rays  */
/*                     of its probes (shading reads the previous atlases    */
/*                     wherever a ray hits) and the blend of its tiles;     */
/*   (the ranks all-gather the tiles, so every rank holds the whole atlas   */
/*   that the next frame's shading reads: rays have no length limit).       */
/* Each step is the single-volume step restricted to the rank's probes, so  */
/* the result equals orc_update's.  Deterministic allocation and the FP64   */
/* atlases only (sampler 0, not packed).                                    */
/* ------------------------------------------------------------------------ */
static int slab_ok(const orc_vol* v, int p0, int p1)
{
    return v->d.sampler == 0 && !v->d.packed && p0 >= 0 && p0 <= p1 && p1 <= v->P;
}

EXPORT int orc_slab_begin(orc_vol* v, const orc_frame* fr, int p0, int p1)
{
    if (!slab_ok(v, p0, p1)) return -1;
    if (v->bvh_dirty) {
        if (cbvh_build(&v->bvh, v->V, v->nv, v->I, v->nt)) return -1;
        v->bvh_dirty = 0;
    }
    orc_frame_rotation(fr->seed, fr->frame, v->R);
    classify(v, fr);
    run_phase_range(v, fr, 0, p0, p1);
    change_state(v, fr, p0, p1);
    return 0;
}

EXPORT int orc_slab_weights(orc_vol* v, const orc_frame* fr, int p0, int p1)
{
    if (!slab_ok(v, p0, p1)) return -1;
    change_weights(v, fr, p0, p1);
    return 0;
}

EXPORT int orc_slab_finish(orc_vol* v, const orc_frame* fr, int p0, int p1)
{
    if (!slab_ok(v, p0, p1)) return -1;
    if (orc_allocate_masked(v->W, v->cls, v->P, v->d.avg, v->d.rmin, v->d.rmax, v->n, v->off)) return -1;
    run_phase_range(v, fr, 1, p0, p1);
    run_phase_range(v, fr, 2, p0, p1);
    return 0;
}

/* Copy the part of a per-probe state array that belongs to probes [p0, p1)
   out to buf (into = 0) or in from buf (into = 1).  which: 0 Tr_v, 1 Tr_r
   (uint16[8] a probe), 2 W (uint32), 3 irradiance tiles (double[Ti^2][3]),
   4 irradiance counts (uint8[Ti^2]), 5 depth tiles (double[Td^2][2]),
   6 depth counts (uint8[Td^2]).  Returns the bytes copied, or -1. */
EXPORT long long orc_slab_slice(orc_vol* v, int which, int p0, int p1, void* buf, int into)
{
    if (p0 < 0 || p0 > p1 || p1 > v->P || !buf) return -1;
    size_t per;
    char* base;
    switch (which) {
    case 0: per = 16; base = (char*)v->trv; break;
    case 1: per = 16; base = (char*)v->trr; break;
    case 2: per = 4; base = (char*)v->W; break;
    case 3: per = (size_t)v->Ti * v->Ti * 3 * sizeof(double); base = (char*)v->irr; break;
    case 4: per = (size_t)v->Ti * v->Ti; base = (char*)v->irr_n; break;
    case 5: per = (size_t)v->Td * v->Td * 2 * sizeof(double); base = (char*)v->dep; break;
    case 6: per = (size_t)v->Td * v->Td; base = (char*)v->dep_n; break;
    default: return -1;
    }
    const size_t n = per * (size_t)(p1 - p0);
    if (into)
        memcpy(base + per * (size_t)p0, buf, n);
    else
        memcpy(buf, base + per * (size_t)p0, n);
    return (long long)n;
}

/* Trace + shade the pilot and main rays of a probe subset without blending */
/* (timing sample for the CPU baseline), split over the volume's threads.    */
/* Requires a previous orc_update.                                           */
typedef struct {
    orc_vol* v;
    const orc_frame* fr;
    const int* probes;
    int k0, k1;
    long long rays;
} sample_job;

static void* sample_worker(void* arg)
{
    sample_job* j = (sample_job*)arg;
    for (int k = j->k0; k < j->k1; ++k) {
        const int p = j->probes[k];
        pilot_probe(j->v, j->fr, p);
        main_probe(j->v, j->fr, p);
        j->rays += j->v->n[p];
    }
    return NULL;
}

EXPORT long long orc_trace_shade_probes(orc_vol* v, const orc_frame* fr, const int* probes, int count)
{
    for (int k = 0; k < count; ++k)
        if (probes[k] < 0 || probes[k] >= v->P) return -1;
    int nt = v->nthreads;
    if (nt > count) nt = count;
    if (nt > 256) nt = 256;
    if (nt < 1) return 0;
    pthread_t th[256];
    sample_job jobs[256];
    for (int t = 0; t < nt; ++t) {
        jobs[t].v = v;
        jobs[t].fr = fr;
        jobs[t].probes = probes;
        jobs[t].k0 = (int)((long long)count * t / nt);
        jobs[t].k1 = (int)((long long)count * (t + 1) / nt);
        jobs[t].rays = 0;
    }
    for (int t = 1; t < nt; ++t) pthread_create(&th[t], NULL, sample_worker, &jobs[t]);
    sample_worker(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    long long rays = 0;
    for (int t = 0; t < nt; ++t) rays += jobs[t].rays;
    return rays;
}

/* ------------------------------------------------------------------------ */
/* State readers for the tests.                                              */
/* ------------------------------------------------------------------------ */
/* the number of threads later phases split over (timing only: results do  */
/* not depend on it)                                                        */
EXPORT void orc_set_threads(orc_vol* v, int nthreads) { v->nthreads = nthreads > 0 ? nthreads : 1; }
EXPORT int orc_num_probes(const orc_vol* v) { return v->P; }
EXPORT long long orc_num_main_rays(const orc_vol* v) { return (long long)v->R_main; }
EXPORT const double* orc_irr(const orc_vol* v) { return v->irr; }
EXPORT const uint8_t* orc_irr_n(const orc_vol* v) { return v->irr_n; }
EXPORT const double* orc_dep(const orc_vol* v) { return v->dep; }
EXPORT const uint8_t* orc_dep_n(const orc_vol* v) { return v->dep_n; }
EXPORT const uint32_t* orc_W(const orc_vol* v) { return v->W; }
EXPORT const uint32_t* orc_n(const orc_vol* v) { return v->n; }
EXPORT const uint32_t* orc_off(const orc_vol* v) { return v->off; }
EXPORT const uint16_t* orc_qv(const orc_vol* v) { return v->qv; }
EXPORT const uint16_t* orc_qr(const orc_vol* v) { return v->qr; }
EXPORT const uint16_t* orc_trv(const orc_vol* v) { return v->trv; }
EXPORT const uint16_t* orc_trr(const orc_vol* v) { return v->trr; }
EXPORT const float* orc_pil_t(const orc_vol* v) { return v->pil_t; }
EXPORT const int* orc_pil_tri(const orc_vol* v) { return v->pil_tri; }
EXPORT const float* orc_pil_lum(const orc_vol* v) { return v->pil_lum; }
EXPORT const float* orc_pil_dir(const orc_vol* v) { return v->pil_dir; }
EXPORT const double* orc_pil_rad(const orc_vol* v) { return v->pil_rad; }
EXPORT const double* orc_pil_dep(const orc_vol* v) { return v->pil_dep; }
EXPORT const float* orc_m_t(const orc_vol* v) { return v->m_t; }
EXPORT const int* orc_m_tri(const orc_vol* v) { return v->m_tri; }
EXPORT const double* orc_m_rad(const orc_vol* v) { return v->m_rad; }
EXPORT const double* orc_m_dep(const orc_vol* v) { return v->m_dep; }
EXPORT const float* orc_rot(const orc_vol* v) { return v->R; }
EXPORT void orc_probe_pos(const orc_vol* v, int p, float out[3]) { probe_pos(v, p, out); }
EXPORT void orc_main_dir(const orc_vol* v, int m, int i, float out[3]) { main_dir(v, m, i, out); }
EXPORT double orc_voxel_diag(const orc_vol* v) { return v->s; }
EXPORT float orc_depth_max(const orc_vol* v) { return v->depth_max; }
EXPORT float orc_tmin(const orc_vol* v) { return v->tmin; }

/* Test hooks: overwrite state to set up closed-form cases. */
EXPORT void orc_set_atlas(orc_vol* v, const double* irr, const uint8_t* irr_n, const double* dep, const uint8_t* dep_n)
{
    size_t P = (size_t)v->P;
    if (irr) memcpy(v->irr, irr, P * v->Ti * v->Ti * 3 * sizeof(double));
    if (irr_n) memcpy(v->irr_n, irr_n, P * v->Ti * v->Ti);
    if (dep) memcpy(v->dep, dep, P * v->Td * v->Td * 2 * sizeof(double));
    if (dep_n) memcpy(v->dep_n, dep_n, P * v->Td * v->Td);
}

EXPORT void orc_border_copy(double* tile, uint8_t* cnt, int n, int ch) { border_copy(tile, cnt, n, ch); }

/* Metropolis sampler state and samples (desc.sampler = 1) */
EXPORT long long orc_mh_samples(const orc_vol* v) { return (long long)v->B; }
EXPORT const uint32_t* orc_qd(const orc_vol* v) { return v->qd; }
EXPORT const uint8_t* orc_cls(const orc_vol* v) { return v->cls; }
EXPORT void orc_dyn_sizes(const orc_vol* v, long long out[8])
{
    out[0] = (long long)v->Cd;
    out[1] = (long long)v->Bd;
    out[2] = (long long)v->Rd;
    out[3] = (long long)v->Rdyn;
    out[4] = v->n_marked;
    out[5] = v->n_incl;
    out[6] = v->Pp;
    out[7] = 0;
}
EXPORT const float* orc_dyn_chain_g(const orc_vol* v) { return v->dch_g; }
EXPORT const float* orc_dyn_chain_u(const orc_vol* v) { return v->dch_u; }
EXPORT const int* orc_dyn_proxy(const orc_vol* v) { return v->dsm_q; }
EXPORT const float* orc_dyn_dir(const orc_vol* v) { return v->dsm_dir; }
EXPORT const int* orc_dyn_cell(const orc_vol* v) { return v->dsm_cell; }
EXPORT const int* orc_dyn_marks(const orc_vol* v) { return v->dmark; }
EXPORT const uint32_t* orc_dyn_off(const orc_vol* v) { return v->doff; }
EXPORT const int* orc_dyn_ray_probe(const orc_vol* v) { return v->d_p; }
EXPORT const int* orc_dyn_ray_key(const orc_vol* v) { return v->d_k; }
EXPORT const float* orc_dyn_t(const orc_vol* v) { return v->d_t; }
EXPORT const int* orc_dyn_tri(const orc_vol* v) { return v->d_tri; }
EXPORT const double* orc_dyn_rad(const orc_vol* v) { return v->d_rad; }
EXPORT const double* orc_dyn_dep(const orc_vol* v) { return v->d_dep; }
EXPORT int orc_dyn_ntex(const orc_vol* v, int o) { return v->ntex[o & 7]; }
EXPORT const int* orc_dyn_tex(const orc_vol* v) { return v->tex_t; }
EXPORT const float* orc_dyn_tex_dir(const orc_vol* v) { return v->tex_dir; }
EXPORT void orc_texel_centre_dir(int cx, int cy, int n, float w[3]) { texel_centre_dir(cx, cy, n, w); }
EXPORT long long orc_mh_chains(const orc_vol* v) { return (long long)v->C; }
EXPORT const float* orc_mh_chain_g(const orc_vol* v) { return v->ch_g; }
EXPORT const float* orc_mh_chain_u(const orc_vol* v) { return v->ch_u; }
EXPORT const int* orc_mh_probe(const orc_vol* v) { return v->smp_p; }
EXPORT const float* orc_mh_dir(const orc_vol* v) { return v->smp_dir; }
EXPORT const int* orc_mh_tri(const orc_vol* v) { return v->smp_tri; }
EXPORT const float* orc_mh_t(const orc_vol* v) { return v->smp_t; }
EXPORT const float* orc_mh_t_neg(const orc_vol* v) { return v->smp_tn; }
EXPORT const int* orc_mh_tri_neg(const orc_vol* v) { return v->smp_trin; }
EXPORT const double* orc_mh_rad(const orc_vol* v) { return v->smp_rad; }
EXPORT const double* orc_mh_dep(const orc_vol* v) { return v->smp_dep; }
/* Test hook: h(x) of the volume's current guide (last frame's heuristics and
   atlas) at grid coordinates g and octahedral coordinates u */
EXPORT float orc_mh_guide(const orc_vol* v, const orc_frame* fr, const float g[3], const float u[2])
{
    pthread_once(&g_mh_once, mh_tables_init);
    return mh_guide(v, fr, g, u);
}

/* packed atlases (NULL unless the volume was created packed) */
EXPORT const uint32_t* orc_irr_packed(const orc_vol* v) { return v->irr_pk; }
EXPORT const uint32_t* orc_dep_packed(const orc_vol* v) { return v->dep_pk; }
EXPORT float orc_cage_diag(const orc_vol* v) { return v->s_f; }

/* Test hook: blend given records of probe p into the packed atlases (the
   probe's pilot directions, n_p and offsets from the last update). */
EXPORT void orc_blend_packed_records(orc_vol* v, int p, int use_pilots, const double* pil_rad, const double* pil_dep,
                                     const double* m_rad, const double* m_dep)
{
    size_t r0 = (size_t)v->off[p], m = (size_t)(v->n[p] - 8u);
    if (pil_rad) memcpy(v->pil_rad + (size_t)p * 8 * 3, pil_rad, 8 * 3 * sizeof(double));
    if (pil_dep) memcpy(v->pil_dep + (size_t)p * 8, pil_dep, 8 * sizeof(double));
    if (m_rad) memcpy(v->m_rad + r0 * 3, m_rad, m * 3 * sizeof(double));
    if (m_dep) memcpy(v->m_dep + r0, m_dep, m * sizeof(double));
    blend_probe_packed(v, p, use_pilots);
}

/* Test hook: run the heuristics step (Sec. 4.1-4.2) on given pilot results. */
EXPORT void orc_change_from_pilots(orc_vol* v, const orc_frame* fr, const float* pil_t, const int* pil_tri,
                                   const float* pil_lum)
{
    size_t n = (size_t)v->P * 8;
    memcpy(v->pil_t, pil_t, n * sizeof(float));
    memcpy(v->pil_tri, pil_tri, n * sizeof(int));
    memcpy(v->pil_lum, pil_lum, n * sizeof(float));
    change_detect(v, fr);
}
