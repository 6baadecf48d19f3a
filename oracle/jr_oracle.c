/*
 * jr_oracle.c -- plain, slow, FP64 CPU oracle for Jump Restore light transport
 * (Holl, Singh, Seidel, "Jump Restore Light Transport", arXiv 2409.07148).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg use it.  It shares no code, header, table or constant generator with the
 * CUDA library; the two meet only through the seeded scene arrays.
 *
 * What it computes, in the paper's order and notation:
 *   - Alg. 2 (Jump Restore, Section 7.2): holding time t1 ~ Exp(1), killing time
 *     t2 ~ Exp(k(x)); t1 < t2 -> local move, else regeneration from mu.
 *   - killing rate for pi-invariant local dynamics and state-independent mu
 *     (Section 6.2, "killing-rate-simplified"): k = c~ * u / p.
 *   - local dynamics M^0 = Metropolis-Hastings (Alg. 1, Section 4) with the
 *     Gaussian small-step kernel zeta (Section 5) and the acceptance function
 *     of Section 4 ("optimal-acceptance-function"); zeta is symmetric so the
 *     proposal densities cancel.
 *   - estimator: normalisation-free tour estimator (Section 6.3),
 *     (c~/j) * sum_i dt_i * g(x_{i-1}) / p(x_{i-1}), left-rectangle rule of
 *     Section 7.4 ("approx").
 *   - the MH baseline of Section 8 ("Metropolis"): Alg. 1 with the mixture
 *     proposal of Section 5, l mu + (1 - l) zeta, and its ergodic-average
 *     estimator after a burn-in (Section 9 parameters).
 *   - Langevin local dynamics (MALA, Section 9): the integrand's gradient in
 *     forward mode, the MALA proposal and its MH acceptance, for Jump Restore
 *     ("MALA Restore") and for the MH baseline ("MALA").
 *   - the general Restore of Section 6.1 (local dynamics that need not be
 *     pi-invariant, killing rate ((L* + kappa mu*) p) / p) on 1-D analytic
 *     targets, with the unadjusted Gaussian random walk as local dynamics.
 *   - the integrand: primary-sample-space (Section 2, Kelemen et al.) path
 *     contribution of a unidirectional path tracer with emission collected at
 *     every vertex; p = luminance of the RGB contribution.
 * Readings where the paper is silent (zeta's scale, luminance weights, path
 * sampler, RNG stream layout, tie rules) are fixed identically for the CUDA
 * library and listed in the design notes; they are restated where used below.
 *
 * Precision: every quantity is double.  Uniform variates are (r >> 8) * 2^-24,
 * exactly representable in float and double.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written from its published definition.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11, Section 3.3): 10 rounds of two 32x32->64 multiplies, */
/* key schedule by the Weyl constants.                                        */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_M4x32_0 = 0xD2511F53u;
static const uint32_t PHILOX_M4x32_1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W32_0 = 0x9E3779B9u;
static const uint32_t PHILOX_W32_1 = 0xBB67AE85u;

ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W32_0;
            k1 += PHILOX_W32_1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M4x32_0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M4x32_1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout (a reading: the paper fixes no RNG).                         *
 *   key     = (lo32(seed), hi32(seed))                                       *
 *   counter = (block + 256*tag, chain id, lo32(step), hi32(step))            *
 * tag 0: one Jump Restore step; block 0 -> (U1, U2, Ua, spare), blocks       *
 *        1..ceil(D/4) -> D coordinates (Gaussian pairs for the local move or *
 *        uniforms for regeneration -- the same counters, so the stream never *
 *        depends on the branch taken).                                       *
 * tag 1: the initial state of a chain (blocks 1.., step 0).                  *
 * tag 2: plain path-tracing sample (chain id field = lo32(sample),           *
 *        step field = hi32(sample)).                                         */
enum { ORC_TAG_STEP = 0, ORC_TAG_INIT = 1, ORC_TAG_PT = 2 };

static double u01(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

static void draw_block(uint64_t seed, uint32_t tag, uint32_t block, uint32_t chain, uint64_t step, double u[4])
{
    uint32_t ctr[4] = { block + 256u * tag, chain, (uint32_t)step, (uint32_t)(step >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = u01(r[i]);
}

/* D coordinates from blocks 1..ceil((D+1)/4); one extra value is always there *
 * for odd D so that Gaussian pairs never run short.                          */
#define ORC_MAX_DIM 64
static void draw_coords(uint64_t seed, uint32_t tag, uint32_t chain, uint64_t step, int D, double v[ORC_MAX_DIM + 4])
{
    int nblk = (D + 3) / 4;
    if (D % 2 == 1 && 4 * nblk < D + 1) nblk++;
    for (int b = 0; b < nblk; ++b) draw_block(seed, tag, (uint32_t)(b + 1), chain, step, v + 4 * b);
}

ORC_EXPORT void orc_draw_uniforms(uint64_t seed, uint32_t tag, uint32_t block, uint32_t chain, uint64_t step, double out[4])
{
    draw_block(seed, tag, block, chain, step, out);
}

/* The same block for chains chain_begin .. +n (out: n x 4). */
ORC_EXPORT void orc_draw_uniforms_many(uint64_t seed, uint32_t tag, uint32_t block, uint32_t chain_begin, uint64_t n,
                                       uint64_t step, double* out)
{
    for (uint64_t i = 0; i < n; ++i) draw_block(seed, tag, block, (uint32_t)(chain_begin + i), step, out + 4 * i);
}

/* ------------------------------------------------------------------------- */
/* Small vector helpers                                                       */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = { x, y, z }; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static v3 normalize(v3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }

/* Orthonormal basis around unit n: Duff et al., "Building an Orthonormal     *
 * Basis, Revisited", JCGT 6(1), 2017.                                        */
static void onb(v3 n, v3* t, v3* b)
{
    double sign = copysign(1.0, n.z);
    double a = -1.0 / (sign + n.z);
    double bb = n.x * n.y * a;
    *t = mk(1.0 + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    *b = mk(bb, sign + n.y * n.y * a, -n.y);
}

/* ------------------------------------------------------------------------- */
/* Scene                                                                      */
/* ------------------------------------------------------------------------- */
/* Material record: 12 floats                                                 *
 *  [0] type (0 Lambertian, 1 modified Phong, 2 smooth dielectric)            *
 *  [1..3] albedo rho (RGB)  [4..6] emission L_e (RGB, one-sided, emits on    *
 *  the side the winding normal points to)  [7] Phong exponent  [8] IOR       */
#define ORC_MAT_FLOATS 12
enum { ORC_LAMBERT = 0, ORC_PHONG = 1, ORC_DIELECTRIC = 2 };

typedef struct {
    int type;
    v3 albedo, emission;
    double phong_n, ior;
    int emits;
} orc_material;

typedef struct {
    double lo[3], hi[3];
    int left, right;    /* children, or -1 for a leaf */
    int first, count;   /* leaf triangle range in the permuted index list */
} orc_bvh_node;

typedef struct {
    int n_tris, n_mats;
    v3* v0; v3* v1; v3* v2;
    v3* ng;              /* unit geometric normal (e1 x e2) */
    int* mat;
    orc_material* mats;
    v3 cam_o, cam_f, cam_r, cam_u;
    /* optional median-split BVH (closest hit must equal brute force) */
    int n_nodes;
    orc_bvh_node* nodes;
    int* perm;
} orc_scene;

ORC_EXPORT orc_scene* orc_scene_create(const float* verts, int n_verts, const uint32_t* tris, int n_tris,
                                       const uint32_t* tri_mat, const float* mats, int n_mats, const float* camera12)
{
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    if (!s) return NULL;
    s->n_tris = n_tris;
    s->n_mats = n_mats;
    s->v0 = (v3*)malloc(sizeof(v3) * (size_t)(n_tris > 0 ? n_tris : 1));
    s->v1 = (v3*)malloc(sizeof(v3) * (size_t)(n_tris > 0 ? n_tris : 1));
    s->v2 = (v3*)malloc(sizeof(v3) * (size_t)(n_tris > 0 ? n_tris : 1));
    s->ng = (v3*)malloc(sizeof(v3) * (size_t)(n_tris > 0 ? n_tris : 1));
    s->mat = (int*)malloc(sizeof(int) * (size_t)(n_tris > 0 ? n_tris : 1));
    s->mats = (orc_material*)malloc(sizeof(orc_material) * (size_t)(n_mats > 0 ? n_mats : 1));
    for (int i = 0; i < n_tris; ++i) {
        const uint32_t* t = tris + 3 * i;
        if ((int)t[0] >= n_verts || (int)t[1] >= n_verts || (int)t[2] >= n_verts) { free(s); return NULL; }
        s->v0[i] = mk(verts[3 * t[0]], verts[3 * t[0] + 1], verts[3 * t[0] + 2]);
        s->v1[i] = mk(verts[3 * t[1]], verts[3 * t[1] + 1], verts[3 * t[1] + 2]);
        s->v2[i] = mk(verts[3 * t[2]], verts[3 * t[2] + 1], verts[3 * t[2] + 2]);
        s->ng[i] = normalize(cross(sub(s->v1[i], s->v0[i]), sub(s->v2[i], s->v0[i])));
        s->mat[i] = (int)tri_mat[i];
    }
    for (int m = 0; m < n_mats; ++m) {
        const float* r = mats + ORC_MAT_FLOATS * m;
        orc_material* q = &s->mats[m];
        q->type = (int)r[0];
        q->albedo = mk(r[1], r[2], r[3]);
        q->emission = mk(r[4], r[5], r[6]);
        q->phong_n = r[7];
        q->ior = r[8];
        q->emits = (r[4] != 0.0f || r[5] != 0.0f || r[6] != 0.0f);
    }
    s->cam_o = mk(camera12[0], camera12[1], camera12[2]);
    s->cam_f = mk(camera12[3], camera12[4], camera12[5]);
    s->cam_r = mk(camera12[6], camera12[7], camera12[8]);
    s->cam_u = mk(camera12[9], camera12[10], camera12[11]);
    return s;
}

ORC_EXPORT void orc_scene_destroy(orc_scene* s)
{
    if (!s) return;
    free(s->v0); free(s->v1); free(s->v2); free(s->ng); free(s->mat); free(s->mats);
    free(s->nodes); free(s->perm);
    free(s);
}

/* Moller-Trumbore ray/triangle test (Moller & Trumbore, JGT 1997).  Returns  *
 * t > 0 of the hit, or +inf.  det == 0 (ray in the triangle's plane) misses. */
static double mt_intersect(v3 o, v3 d, v3 v0, v3 v1, v3 v2)
{
    v3 e1 = sub(v1, v0), e2 = sub(v2, v0);
    v3 pv = cross(d, e2);
    double det = dot(e1, pv);
    if (det == 0.0) return INFINITY;
    double inv = 1.0 / det;
    v3 tv = sub(o, v0);
    double u = dot(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return INFINITY;
    v3 qv = cross(tv, e1);
    double v = dot(d, qv) * inv;
    if (v < 0.0 || u + v > 1.0) return INFINITY;
    double t = dot(e2, qv) * inv;
    return t > 0.0 ? t : INFINITY;
}

ORC_EXPORT double orc_intersect_triangle(const double o[3], const double d[3], const double v0[3], const double v1[3],
                                         const double v2[3])
{
    return mt_intersect(mk(o[0], o[1], o[2]), mk(d[0], d[1], d[2]), mk(v0[0], v0[1], v0[2]),
                        mk(v1[0], v1[1], v1[2]), mk(v2[0], v2[1], v2[2]));
}

/* Closest hit by brute force: the definition.  Ties on equal t go to the     *
 * smaller triangle index (strict < over increasing index).                   */
static int closest_brute(const orc_scene* s, v3 o, v3 d, double* t_out)
{
    double best = INFINITY;
    int id = -1;
    for (int i = 0; i < s->n_tris; ++i) {
        double t = mt_intersect(o, d, s->v0[i], s->v1[i], s->v2[i]);
        if (t < best) { best = t; id = i; }
    }
    *t_out = best;
    return id;
}

/* --- optional median-split BVH (only an accelerator; pinned to brute force) */
static int bvh_build_rec(orc_scene* s, int first, int count, int* cap)
{
    if (s->n_nodes >= *cap) {
        *cap *= 2;
        s->nodes = (orc_bvh_node*)realloc(s->nodes, sizeof(orc_bvh_node) * (size_t)*cap);
    }
    int me = s->n_nodes++;
    orc_bvh_node nd;
    for (int k = 0; k < 3; ++k) { nd.lo[k] = INFINITY; nd.hi[k] = -INFINITY; }
    double clo[3] = { INFINITY, INFINITY, INFINITY }, chi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int i = first; i < first + count; ++i) {
        int t = s->perm[i];
        v3 p[3] = { s->v0[t], s->v1[t], s->v2[t] };
        for (int j = 0; j < 3; ++j) {
            double c[3] = { p[j].x, p[j].y, p[j].z };
            for (int k = 0; k < 3; ++k) {
                if (c[k] < nd.lo[k]) nd.lo[k] = c[k];
                if (c[k] > nd.hi[k]) nd.hi[k] = c[k];
            }
        }
        double cen[3] = { (p[0].x + p[1].x + p[2].x) / 3, (p[0].y + p[1].y + p[2].y) / 3, (p[0].z + p[1].z + p[2].z) / 3 };
        for (int k = 0; k < 3; ++k) {
            if (cen[k] < clo[k]) clo[k] = cen[k];
            if (cen[k] > chi[k]) chi[k] = cen[k];
        }
    }
    /* widen by a relative margin so that a slab test never rejects a box      *
     * whose triangle the exact test accepts                                  */
    for (int k = 0; k < 3; ++k) {
        double m = 1e-9 * (1.0 + fabs(nd.lo[k]) + fabs(nd.hi[k]));
        nd.lo[k] -= m; nd.hi[k] += m;
    }
    nd.left = nd.right = -1;
    nd.first = first;
    nd.count = count;
    int axis = 0;
    double ext = chi[0] - clo[0];
    for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > ext) { ext = chi[k] - clo[k]; axis = k; }
    if (count > 4 && ext > 0.0) {
        double mid = 0.5 * (clo[axis] + chi[axis]);
        int i = first, j = first + count - 1;
        while (i <= j) {
            int t = s->perm[i];
            double c = axis == 0 ? s->v0[t].x + s->v1[t].x + s->v2[t].x
                     : axis == 1 ? s->v0[t].y + s->v1[t].y + s->v2[t].y
                                 : s->v0[t].z + s->v1[t].z + s->v2[t].z;
            if (c / 3 < mid) ++i;
            else { int tmp = s->perm[i]; s->perm[i] = s->perm[j]; s->perm[j] = tmp; --j; }
        }
        int nl = i - first;
        if (nl == 0 || nl == count) nl = count / 2;
        s->nodes[me] = nd;
        int l = bvh_build_rec(s, first, nl, cap);
        int r = bvh_build_rec(s, first + nl, count - nl, cap);
        s->nodes[me].left = l;
        s->nodes[me].right = r;
        return me;
    }
    s->nodes[me] = nd;
    return me;
}

ORC_EXPORT int orc_scene_build_bvh(orc_scene* s)
{
    free(s->nodes); free(s->perm);
    s->n_nodes = 0;
    if (s->n_tris == 0) { s->nodes = NULL; s->perm = NULL; return 0; }
    int cap = 2 * s->n_tris + 1;
    s->nodes = (orc_bvh_node*)malloc(sizeof(orc_bvh_node) * (size_t)cap);
    s->perm = (int*)malloc(sizeof(int) * (size_t)s->n_tris);
    for (int i = 0; i < s->n_tris; ++i) s->perm[i] = i;
    bvh_build_rec(s, 0, s->n_tris, &cap);
    return s->n_nodes;
}

static int slab_hits(const orc_bvh_node* n, v3 o, v3 inv, double tmax)
{
    double oo[3] = { o.x, o.y, o.z }, ii[3] = { inv.x, inv.y, inv.z };
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double a = (n->lo[k] - oo[k]) * ii[k], b = (n->hi[k] - oo[k]) * ii[k];
        if (isnan(a) || isnan(b)) { /* origin on a slab plane of a flat axis */
            if (oo[k] < n->lo[k] || oo[k] > n->hi[k]) return 0;
            continue;
        }
        double lo = a < b ? a : b, hi = a < b ? b : a;
        if (lo > t0) t0 = lo;
        if (hi < t1) t1 = hi;
        if (t0 > t1) return 0;
    }
    return 1;
}

static int closest_bvh(const orc_scene* s, v3 o, v3 d, double* t_out)
{
    double best = INFINITY;
    int id = -1;
    if (s->n_nodes == 0) { *t_out = best; return -1; }
    v3 inv = mk(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const orc_bvh_node* n = &s->nodes[stack[--sp]];
        if (!slab_hits(n, o, inv, best)) continue;
        if (n->left < 0) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int t = s->perm[i];
                double th = mt_intersect(o, d, s->v0[t], s->v1[t], s->v2[t]);
                if (th < best || (th == best && th < INFINITY && t < id)) { best = th; id = t; }
            }
        } else {
            if (sp + 2 > 128) abort();
            stack[sp++] = n->right;
            stack[sp++] = n->left;
        }
    }
    *t_out = best;
    return id;
}

static int closest_hit(const orc_scene* s, v3 o, v3 d, double* t)
{
    return s->n_nodes > 0 ? closest_bvh(s, o, d, t) : closest_brute(s, o, d, t);
}

ORC_EXPORT int orc_closest_hit(const orc_scene* s, const double o[3], const double d[3], int use_bvh, double* t)
{
    v3 oo = mk(o[0], o[1], o[2]), dd = mk(d[0], d[1], d[2]);
    return use_bvh ? closest_bvh(s, oo, dd, t) : closest_brute(s, oo, dd, t);
}

/* ------------------------------------------------------------------------- */
/* BSDF sampling (the path sampler; the paper renders with pbrt/lmc and does  */
/* not print one, so this is a reading fixed for both sides).                 */
/* d: incoming ray direction (unit), ng: unit geometric normal.               */
/* Returns 0 if the path terminates (zero weight).                            */
/* ------------------------------------------------------------------------- */
static double lum(v3 c) { return 0.2126 * c.x + 0.7152 * c.y + 0.0722 * c.z; }

/* Exact unpolarised Fresnel reflectance of a smooth dielectric interface.    */
static double fresnel_dielectric(double cos_i, double eta_i, double eta_t, double* cos_t_out)
{
    double e = eta_i / eta_t;
    double sin2_t = e * e * (1.0 - cos_i * cos_i);
    if (sin2_t >= 1.0) { *cos_t_out = 0.0; return 1.0; }
    double cos_t = sqrt(1.0 - sin2_t);
    double rs = (eta_i * cos_i - eta_t * cos_t) / (eta_i * cos_i + eta_t * cos_t);
    double rp = (eta_t * cos_i - eta_i * cos_t) / (eta_t * cos_i + eta_i * cos_t);
    *cos_t_out = cos_t;
    return 0.5 * (rs * rs + rp * rp);
}

ORC_EXPORT double orc_fresnel(double cos_i, double eta_i, double eta_t)
{
    double ct;
    return fresnel_dielectric(cos_i, eta_i, eta_t, &ct);
}

static int scatter(const orc_material* m, v3 d, v3 ng, double u1, double u2, v3* wi, v3* w)
{
    if (m->type == ORC_DIELECTRIC) {
        double cos_i = -dot(d, ng);
        double eta_i = 1.0, eta_t = m->ior;
        v3 nn = ng;
        if (cos_i < 0.0) { cos_i = -cos_i; eta_i = m->ior; eta_t = 1.0; nn = scl(ng, -1.0); }
        double cos_t;
        double R = fresnel_dielectric(cos_i, eta_i, eta_t, &cos_t);
        if (u1 < R) {
            *wi = add(d, scl(nn, 2.0 * cos_i));
        } else {
            double e = eta_i / eta_t;
            *wi = add(scl(d, e), scl(nn, e * cos_i - cos_t));
        }
        *w = mk(1.0, 1.0, 1.0);
        return 1;
    }
    v3 ns = dot(d, ng) < 0.0 ? ng : scl(ng, -1.0); /* two-sided: face the viewer */
    if (m->type == ORC_LAMBERT) {
        /* cosine-weighted hemisphere by Malley's method; weight = albedo */
        double r = sqrt(u1), phi = 2.0 * M_PI * u2;
        double lz = sqrt(1.0 - u1 > 0.0 ? 1.0 - u1 : 0.0);
        v3 t, b;
        onb(ns, &t, &b);
        *wi = add(add(scl(t, r * cos(phi)), scl(b, r * sin(phi))), scl(ns, lz));
        *w = m->albedo;
        return lum(*w) > 0.0 || w->x > 0.0 || w->y > 0.0 || w->z > 0.0;
    }
    /* modified Phong (Lafortune & Willems 1994): sample cos^n lobe about the  *
     * mirror direction, pdf (n+1)/(2pi) cos^n a; weight = f cos_i / pdf       *
     * = rho (n+2)/(n+1) cos_i, zero below the surface                         */
    v3 r = sub(d, scl(ns, 2.0 * dot(d, ns)));
    double n = m->phong_n;
    double cos_a = pow(1.0 - u1, 1.0 / (n + 1.0));
    double sin_a = sqrt(1.0 - cos_a * cos_a > 0.0 ? 1.0 - cos_a * cos_a : 0.0);
    double phi = 2.0 * M_PI * u2;
    v3 t, b;
    onb(r, &t, &b);
    *wi = add(add(scl(t, sin_a * cos(phi)), scl(b, sin_a * sin(phi))), scl(r, cos_a));
    double cos_i = dot(*wi, ns);
    if (cos_i <= 0.0) { *w = mk(0, 0, 0); return 0; }
    *w = scl(m->albedo, (n + 2.0) / (n + 1.0) * cos_i);
    return 1;
}

ORC_EXPORT int orc_scatter(const float* mat12, const double d[3], const double ng[3], double u1, double u2,
                           double wi_out[3], double w_out[3])
{
    orc_material m;
    m.type = (int)mat12[0];
    m.albedo = mk(mat12[1], mat12[2], mat12[3]);
    m.emission = mk(mat12[4], mat12[5], mat12[6]);
    m.phong_n = mat12[7];
    m.ior = mat12[8];
    v3 wi, w;
    int ok = scatter(&m, mk(d[0], d[1], d[2]), mk(ng[0], ng[1], ng[2]), u1, u2, &wi, &w);
    wi_out[0] = wi.x; wi_out[1] = wi.y; wi_out[2] = wi.z;
    w_out[0] = w.x; w_out[1] = w.y; w_out[2] = w.z;
    return ok;
}

/* ------------------------------------------------------------------------- */
/* The integrand: PSS path contribution F(x), x in [0,1)^D, D = 2 + 2*depth.  */
/* (x0, x1): film point; bounce b uses (x_{2+2b}, x_{3+2b}).  Emission is     */
/* added at every vertex v1..v_{depth+1}.  Miss -> stop (black background).   */
/* No Russian roulette, no light sampling.  Returns the number of ray casts.  */
/* hit_ids (optional, depth+1 entries): triangle hit by each cast, -1 = none. */
/* ------------------------------------------------------------------------- */
#define ORC_EPS_OFFSET 1e-4

static int eval_path(const orc_scene* s, int depth, const double* x, v3* F_out, int* hit_ids)
{
    v3 F = mk(0, 0, 0), T = mk(1, 1, 1);
    v3 o = s->cam_o;
    v3 d = normalize(add(s->cam_f, add(scl(s->cam_r, 2.0 * x[0] - 1.0), scl(s->cam_u, 1.0 - 2.0 * x[1]))));
    int casts = 0;
    if (hit_ids) for (int v = 0; v <= depth; ++v) hit_ids[v] = -1;
    for (int v = 0; v <= depth; ++v) {
        double t;
        int id = closest_hit(s, o, d, &t);
        ++casts;
        if (hit_ids) hit_ids[v] = id;
        if (id < 0) break;
        const orc_material* m = &s->mats[s->mat[id]];
        v3 ng = s->ng[id];
        v3 p = add(o, scl(d, t));
        if (m->emits && -dot(d, ng) > 0.0)
            F = add(F, mk(T.x * m->emission.x, T.y * m->emission.y, T.z * m->emission.z));
        if (v == depth) break;
        v3 wi, w;
        if (!scatter(m, d, ng, x[2 + 2 * v], x[3 + 2 * v], &wi, &w)) break;
        T = mk(T.x * w.x, T.y * w.y, T.z * w.z);
        if (T.x == 0.0 && T.y == 0.0 && T.z == 0.0) break;
        v3 off = dot(wi, ng) >= 0.0 ? ng : scl(ng, -1.0);
        double mx = fabs(p.x);
        if (fabs(p.y) > mx) mx = fabs(p.y);
        if (fabs(p.z) > mx) mx = fabs(p.z);
        o = add(p, scl(off, ORC_EPS_OFFSET * (1.0 + mx)));
        d = wi;
    }
    *F_out = F;
    return casts;
}

/* ------------------------------------------------------------------------- */
/* Analytic targets on [0,1)^D for the quadrature pins.                       */
/*   kind 1: sum of isotropic Gaussian bumps in the first two coordinates,    */
/*           zero on a band a <= x0 < b; RGB channels modulated so g != p:    */
/*           F = q * (0.5 + x0, 1, 0.5 + x1) (x1 := 0 when D == 1).           */
/* params: [n_modes, band_a, band_b, (w, m0, m1, s) * n_modes]                */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n_modes;
    double band_a, band_b;
    double w[16], m0[16], m1[16], sd[16];
} orc_analytic;

ORC_EXPORT orc_analytic* orc_analytic_create(const double* params)
{
    orc_analytic* a = (orc_analytic*)calloc(1, sizeof(orc_analytic));
    a->n_modes = (int)params[0];
    if (a->n_modes > 16) a->n_modes = 16;
    a->band_a = params[1];
    a->band_b = params[2];
    for (int i = 0; i < a->n_modes; ++i) {
        a->w[i] = params[3 + 4 * i];
        a->m0[i] = params[4 + 4 * i];
        a->m1[i] = params[5 + 4 * i];
        a->sd[i] = params[6 + 4 * i];
    }
    return a;
}

ORC_EXPORT void orc_analytic_destroy(orc_analytic* a) { free(a); }

static v3 eval_analytic(const orc_analytic* a, int D, const double* x)
{
    double x0 = x[0], x1 = D >= 2 ? x[1] : 0.0;
    if (x0 >= a->band_a && x0 < a->band_b) return mk(0, 0, 0);
    double q = 0.0;
    for (int i = 0; i < a->n_modes; ++i) {
        double dx = x0 - a->m0[i], dy = D >= 2 ? x1 - a->m1[i] : 0.0;
        q += a->w[i] * exp(-(dx * dx + dy * dy) / (2.0 * a->sd[i] * a->sd[i]));
    }
    return mk(q * (0.5 + x0), q, q * (0.5 + x1));
}

ORC_EXPORT void orc_analytic_eval(const orc_analytic* a, int D, int n, const double* x, double* F3)
{
    for (int i = 0; i < n; ++i) {
        v3 F = eval_analytic(a, D, x + (size_t)i * D);
        F3[3 * i] = F.x; F3[3 * i + 1] = F.y; F3[3 * i + 2] = F.z;
    }
}

/* ------------------------------------------------------------------------- */
/* Method parameters and the target                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int target_kind;        /* 0 scene path, 1 analytic */
    const orc_scene* scene;
    const orc_analytic* analytic;
    int D, depth;           /* depth only for the scene target (D = 2+2 depth) */
    int width, height;
    double c_tilde;         /* c~ of the simplified killing rate (Section 6.2) */
    double sigma;           /* std of the Gaussian small-step kernel zeta */
    uint64_t seed;
    int rao_blackwell;      /* 1: holding time replaced by its mean 1/(1+k) */
} orc_params;

/* Target density p = luminance of F (all weights > 0: p = 0 iff F = 0).      */
static void eval_target(const orc_params* P, const double* x, v3* F, double* p, int* hit_ids)
{
    if (P->target_kind == 0) eval_path(P->scene, P->depth, x, F, hit_ids);
    else *F = eval_analytic(P->analytic, P->D, x);
    *p = lum(*F);
}

/* Regeneration density u of mu w.r.t. Lebesgue measure on [0,1)^D: the      *
 * uniform large-step distribution, u = 1 (Section 8: mu is the baseline's    *
 * large-step distribution).                                                  */
static double regen_density(const orc_params* P, const double* x) { (void)P; (void)x; return 1.0; }

/* Killing rate, Section 6.2 ("killing-rate-simplified"): k = c~ u / p, with   *
 * k = +inf where p = 0.                                                       */
ORC_EXPORT double orc_killing_rate(double p, double u, double c_tilde)
{
    return p > 0.0 ? c_tilde * u / p : INFINITY;
}

/* Metropolis-Hastings acceptance probability, Section 4 ("optimal-          *
 * acceptance-function") for a symmetric proposal: min(1, p(y)/p(x)) if       *
 * p(x) > 0, else 1.                                                          */
ORC_EXPORT double orc_mh_accept_prob(double px, double py)
{
    if (!(px > 0.0)) return 1.0;
    double r = py / px;
    return r < 1.0 ? r : 1.0;
}

static void pixel_of(const orc_params* P, const double* x, int* px, int* py)
{
    int i = (int)floor(x[0] * P->width);
    int j = P->D >= 2 ? (int)floor(x[1] * P->height) : 0;
    if (i >= P->width) i = P->width - 1;
    if (j >= P->height) j = P->height - 1;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    *px = i; *py = j;
}

static double wrap01(double y)
{
    double w = y - floor(y);
    return w >= 1.0 ? 0.0 : w;
}

/* ------------------------------------------------------------------------- */
/* Chains                                                                     */
/* State row per chain (doubles): x[0..D), F.rgb, p, u.                       */
/* ------------------------------------------------------------------------- */
ORC_EXPORT int orc_state_stride(int D) { return D + 5; }

static orc_params make_params(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                              int width, int height, double c_tilde, double sigma, uint64_t seed, int rb)
{
    orc_params P;
    P.target_kind = target_kind;
    P.scene = scene;
    P.analytic = an;
    P.D = D;
    P.depth = depth;
    P.width = width;
    P.height = height;
    P.c_tilde = c_tilde;
    P.sigma = sigma;
    P.seed = seed;
    P.rao_blackwell = rb;
    return P;
}

static void eval_into_state(const orc_params* P, const double* x, double* st)
{
    v3 F;
    double p;
    for (int d = 0; d < P->D; ++d) st[d] = x[d];
    eval_target(P, x, &F, &p, NULL);
    st[P->D] = F.x; st[P->D + 1] = F.y; st[P->D + 2] = F.z;
    st[P->D + 3] = p;
    st[P->D + 4] = regen_density(P, x);
}

/* Initial state of each chain: x0 ~ mu (uniform), tag 1. */
static void init_chains(const orc_params* P, uint64_t chain_begin, uint64_t n, double* state)
{
    int S = P->D + 5;
    double v[ORC_MAX_DIM + 8];
    for (uint64_t c = 0; c < n; ++c) {
        draw_coords(P->seed, ORC_TAG_INIT, (uint32_t)(chain_begin + c), 0, P->D, v);
        eval_into_state(P, v, state + c * S);
    }
}

typedef struct {
    const orc_params* P;
    uint64_t chain_begin, c_lo, c_hi;
    uint64_t step_begin, n_steps;
    double* state;
    double* accum;            /* W*H*4: RGB sums and time in the pixel */
    uint64_t J, accepts, locals;
    uint8_t* tr_flags;        /* optional [chain][step] */
    double* tr_dt;
    int32_t* tr_pix;
    double* tr_margin;        /* optional: decision margins (t1 - t2, p_y - Ua p_x) */
} orc_job;

/* One chain advanced n steps by Alg. 2.  Splat (estimator of Section 6.3 with *
 * the left-rectangle rule of Section 7.4): the state x_{i-1} held for dt_i     *
 * contributes c~ dt_i (W H) F(x_{i-1}) / p(x_{i-1}) to its pixel; the factor   *
 * W H is the box filter of a pixel in film coordinates.                        */
static void run_chain(orc_job* jb, uint64_t c)
{
    const orc_params* P = jb->P;
    int D = P->D, S = D + 5;
    double* st = jb->state + c * S;
    uint32_t chain = (uint32_t)(jb->chain_begin + c);
    double v[ORC_MAX_DIM + 8], y[ORC_MAX_DIM];
    double WH = (double)P->width * (double)P->height;
    for (uint64_t i = 0; i < jb->n_steps; ++i) {
        uint64_t step = jb->step_begin + i;
        double U[4];
        draw_block(P->seed, ORC_TAG_STEP, 0, chain, step, U);
        double p = st[D + 3], u = st[D + 4];
        /* line "Sample t1 from Exp(1)" and "Sample t2 from Exp(k(x))" */
        double E1 = -log(1.0 - U[0]);
        double E2 = -log(1.0 - U[1]);
        double t1 = E1;
        double t2 = p > 0.0 ? E2 * p / (P->c_tilde * u) : 0.0; /* Exp(k), k = c~u/p; k = inf -> 0 */
        int local = t1 < t2;                                    /* tie -> termination branch */
        double dt = local ? t1 : t2;
        if (P->rao_blackwell) dt = p > 0.0 ? p / (p + P->c_tilde * u) : 0.0;
        int pix = -1;
        if (dt > 0.0 && p > 0.0) {
            int px, py;
            pixel_of(P, st, &px, &py);
            pix = py * P->width + px;
            double wgt = P->c_tilde * dt * WH / p;
            double* a = jb->accum + 4 * (size_t)pix;
            a[0] += wgt * st[D];
            a[1] += wgt * st[D + 1];
            a[2] += wgt * st[D + 2];
            a[3] += dt;
        }
        draw_coords(P->seed, ORC_TAG_STEP, chain, step, D, v);
        int accepted = 0;
        double margin2 = 0.0;
        if (local) {
            /* local state transition: one MH step of M^0 with zeta = N(x, sigma^2) *
             * wrapped onto the unit torus (symmetric, so alpha = min(1, p(y)/p(x))) */
            for (int k = 0; k < (D + 1) / 2; ++k) {
                double R = sqrt(-2.0 * log(1.0 - v[2 * k]));
                double ang = 2.0 * M_PI * v[2 * k + 1];
                y[2 * k] = wrap01(st[2 * k] + P->sigma * R * cos(ang));
                if (2 * k + 1 < D) y[2 * k + 1] = wrap01(st[2 * k + 1] + P->sigma * R * sin(ang));
            }
            double cand[ORC_MAX_DIM + 5];
            eval_into_state(P, y, cand);
            double py = cand[D + 3];
            /* U < alpha(x, y)  <=>  Ua * p(x) < p(y)  when p(x) > 0 */
            accepted = (p > 0.0) ? (U[2] * p < py) : 1;
            margin2 = py - U[2] * p;
            if (accepted) memcpy(st, cand, sizeof(double) * (size_t)S);
            jb->accepts += (uint64_t)accepted;
            jb->locals += 1;
        } else {
            /* global state transition: regenerate from mu (a new tour) */
            eval_into_state(P, v, st);
            jb->J += 1;
        }
        if (jb->tr_flags) {
            size_t o = (size_t)c * jb->n_steps + i;
            jb->tr_flags[o] = (uint8_t)((local ? 0 : 1) | (accepted ? 2 : 0));
            jb->tr_dt[o] = dt;
            jb->tr_pix[o] = pix;
            if (jb->tr_margin) {
                jb->tr_margin[2 * o] = t1 - t2;
                jb->tr_margin[2 * o + 1] = margin2;
            }
        }
    }
}

static void* run_worker(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    for (uint64_t c = jb->c_lo; c < jb->c_hi; ++c) run_chain(jb, c);
    return NULL;
}

static int resolve_threads(int n_threads, uint64_t n_items)
{
    if (n_threads <= 0) {
        long n = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = n > 0 ? (int)n : 1;
    }
    if ((uint64_t)n_threads > n_items) n_threads = (int)(n_items > 0 ? n_items : 1);
    return n_threads;
}

/* Public: initialise n chains (state rows). */
ORC_EXPORT void orc_chains_init(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                                int width, int height, double c_tilde, double sigma, uint64_t seed,
                                uint64_t chain_begin, uint64_t n, double* state)
{
    orc_params P = make_params(target_kind, scene, an, D, depth, width, height, c_tilde, sigma, seed, 0);
    init_chains(&P, chain_begin, n, state);
}

/* Public: advance n chains by n_steps (global step indices step_begin..).     *
 * accum (W*H*4 doubles) is ADDED to; counters are returned in out3 =          *
 * (J, accepts, local steps).  Trace arrays are optional ([chain][step]).      */
ORC_EXPORT int orc_chains_advance(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                                  int width, int height, double c_tilde, double sigma, uint64_t seed,
                                  int rao_blackwell, uint64_t chain_begin, uint64_t n, uint64_t step_begin,
                                  uint64_t n_steps, double* state, double* accum, uint64_t* out3, uint8_t* tr_flags,
                                  double* tr_dt, int32_t* tr_pix, double* tr_margin, int n_threads)
{
    if (D > ORC_MAX_DIM || D < 1) return -1;
    orc_params P = make_params(target_kind, scene, an, D, depth, width, height, c_tilde, sigma, seed, rao_blackwell);
    int T = resolve_threads(n_threads, n);
    orc_job* jobs = (orc_job*)calloc((size_t)T, sizeof(orc_job));
    pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
    size_t npx = (size_t)width * (size_t)height * 4;
    for (int t = 0; t < T; ++t) {
        orc_job* jb = &jobs[t];
        jb->P = &P;
        jb->chain_begin = chain_begin;
        jb->c_lo = n * (uint64_t)t / (uint64_t)T;
        jb->c_hi = n * (uint64_t)(t + 1) / (uint64_t)T;
        jb->step_begin = step_begin;
        jb->n_steps = n_steps;
        jb->state = state;
        jb->accum = (double*)calloc(npx, sizeof(double));
        jb->tr_flags = tr_flags;
        jb->tr_dt = tr_dt;
        jb->tr_pix = tr_pix;
        jb->tr_margin = tr_margin;
        if (T > 1) pthread_create(&th[t], NULL, run_worker, jb);
    }
    if (T == 1) run_worker(&jobs[0]);
    uint64_t J = 0, A = 0, L = 0;
    for (int t = 0; t < T; ++t) {
        if (T > 1) pthread_join(th[t], NULL);
        for (size_t k = 0; k < npx; ++k) accum[k] += jobs[t].accum[k];
        free(jobs[t].accum);
        J += jobs[t].J;
        A += jobs[t].accepts;
        L += jobs[t].locals;
    }
    out3[0] = J; out3[1] = A; out3[2] = L;
    free(jobs);
    free(th);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The MH baseline "Metropolis" of the paper's practical pairing (Section 8):  */
/* one MH chain per chain id with the mixture proposal of Section 5 (eq.       */
/* "mixture-proposal-kernel"): Q_l(x, .) = l mu + (1 - l) zeta(x, .), with the */
/* large-step distribution mu = uniform on [0,1)^D and the small-step kernel   */
/* zeta = N(x, sigma^2) wrapped onto the torus (both symmetric in x and y, so  */
/* the Hastings ratio of Q_l is 1 and the acceptance of Section 4 is           */
/* min(1, p(y)/p(x))); Alg. 1 takes one step.  Section 9: l = 0.3 and the      */
/* estimate uses only the iterations after the first burn_in.                  */
/*                                                                             */
/* Estimator (the ergodic average of the MH chain, pi = p / b): pixel j =      */
/* b_hat * (1/N) sum_{i >= burn_in} W H 1[pix(x_i) = j] F(x_i) / p(x_i), with  */
/* x_i the state before iteration i, N the number of such iterations, and the  */
/* normalisation b = integral of p estimated by the mean of p over the         */
/* large-step proposals (uniform draws, so an unbiased estimate of b).         */
/*                                                                             */
/* Random numbers (a reading): the Restore step's counters (tag 0).  Block 0   */
/* gives (U_s, -, U_a, -): a large step if U_s < l; U_a decides acceptance.    */
/* Blocks 1.. give the D coordinates: uniforms for a large step, Gaussian      */
/* pairs for a small step, exactly as in the Restore step.                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_params* P;
    double ell;
    uint64_t burn_in;
    uint64_t chain_begin, c_lo, c_hi;
    uint64_t step_begin, n_steps;
    double* state;
    double* accum;            /* W*H*4: RGB sums of W H F / p and the count of splats */
    uint64_t n_large, n_small, accepts, splats;
    double p_sum_large;       /* sum of p(y) over the large-step proposals */
    uint8_t* tr_flags;        /* optional [chain][step]: bit0 large step, bit1 accepted, bit2 splatted */
    int32_t* tr_pix;
    double* tr_margin;        /* optional: U_a p(x) - p(y) */
} orc_mh_job;

static void run_chain_mh(orc_mh_job* jb, uint64_t c)
{
    const orc_params* P = jb->P;
    int D = P->D, S = D + 5;
    double* st = jb->state + c * S;
    uint32_t chain = (uint32_t)(jb->chain_begin + c);
    double v[ORC_MAX_DIM + 8], y[ORC_MAX_DIM], cand[ORC_MAX_DIM + 5];
    double WH = (double)P->width * (double)P->height;
    for (uint64_t i = 0; i < jb->n_steps; ++i) {
        uint64_t step = jb->step_begin + i;
        double U[4];
        draw_block(P->seed, ORC_TAG_STEP, 0, chain, step, U);
        double p = st[D + 3];
        /* the estimator's term for the state x_i held at this iteration */
        int pix = -1, splatted = 0;
        if (step >= jb->burn_in) {
            jb->splats += 1;
            splatted = 1;
            if (p > 0.0) {
                int px, py;
                pixel_of(P, st, &px, &py);
                pix = py * P->width + px;
                double wgt = WH / p;
                double* a = jb->accum + 4 * (size_t)pix;
                a[0] += wgt * st[D];
                a[1] += wgt * st[D + 1];
                a[2] += wgt * st[D + 2];
                a[3] += 1.0;
            }
        }
        /* proposal y ~ Q_l(x, .): large step from mu with probability l */
        int large = U[0] < jb->ell;
        draw_coords(P->seed, ORC_TAG_STEP, chain, step, D, v);
        if (large) {
            for (int d = 0; d < D; ++d) y[d] = v[d];
        } else {
            for (int k = 0; k < (D + 1) / 2; ++k) {
                double R = sqrt(-2.0 * log(1.0 - v[2 * k]));
                double ang = 2.0 * M_PI * v[2 * k + 1];
                y[2 * k] = wrap01(st[2 * k] + P->sigma * R * cos(ang));
                if (2 * k + 1 < D) y[2 * k + 1] = wrap01(st[2 * k + 1] + P->sigma * R * sin(ang));
            }
        }
        eval_into_state(P, y, cand);
        double py = cand[D + 3];
        if (large) {
            jb->n_large += 1;
            jb->p_sum_large += py;
        } else {
            jb->n_small += 1;
        }
        /* Alg. 1: accept with probability alpha = min(1, p(y)/p(x)) (1 if p(x) = 0) */
        int accepted = U[2] < orc_mh_accept_prob(p, py);
        if (accepted) memcpy(st, cand, sizeof(double) * (size_t)S);
        jb->accepts += (uint64_t)accepted;
        if (jb->tr_flags) {
            size_t o = (size_t)c * jb->n_steps + i;
            jb->tr_flags[o] = (uint8_t)((large ? 1 : 0) | (accepted ? 2 : 0) | (splatted ? 4 : 0));
            jb->tr_pix[o] = pix;
            if (jb->tr_margin) jb->tr_margin[o] = U[2] * p - py;
        }
    }
}

static void* run_worker_mh(void* arg)
{
    orc_mh_job* jb = (orc_mh_job*)arg;
    for (uint64_t c = jb->c_lo; c < jb->c_hi; ++c) run_chain_mh(jb, c);
    return NULL;
}

/* Public: advance n MH chains by n_steps (global step indices step_begin..).  *
 * accum (W*H*4) is ADDED to; out4 = (large-step proposals, small-step         *
 * proposals, accepted, splatted iterations); *p_sum_large is ADDED to.        *
 * States are initialised with orc_chains_init (x0 ~ mu).                      */
ORC_EXPORT int orc_mh_advance(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                              int width, int height, double sigma, double ell, uint64_t burn_in, uint64_t seed,
                              uint64_t chain_begin, uint64_t n, uint64_t step_begin, uint64_t n_steps, double* state,
                              double* accum, uint64_t* out4, double* p_sum_large, uint8_t* tr_flags, int32_t* tr_pix,
                              double* tr_margin, int n_threads)
{
    if (D > ORC_MAX_DIM || D < 1 || !(ell >= 0.0 && ell <= 1.0)) return -1;
    orc_params P = make_params(target_kind, scene, an, D, depth, width, height, 1.0, sigma, seed, 0);
    int T = resolve_threads(n_threads, n);
    orc_mh_job* jobs = (orc_mh_job*)calloc((size_t)T, sizeof(orc_mh_job));
    pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
    size_t npx = (size_t)width * (size_t)height * 4;
    for (int t = 0; t < T; ++t) {
        orc_mh_job* jb = &jobs[t];
        jb->P = &P;
        jb->ell = ell;
        jb->burn_in = burn_in;
        jb->chain_begin = chain_begin;
        jb->c_lo = n * (uint64_t)t / (uint64_t)T;
        jb->c_hi = n * (uint64_t)(t + 1) / (uint64_t)T;
        jb->step_begin = step_begin;
        jb->n_steps = n_steps;
        jb->state = state;
        jb->accum = (double*)calloc(npx, sizeof(double));
        jb->tr_flags = tr_flags;
        jb->tr_pix = tr_pix;
        jb->tr_margin = tr_margin;
        if (T > 1) pthread_create(&th[t], NULL, run_worker_mh, jb);
    }
    if (T == 1) run_worker_mh(&jobs[0]);
    uint64_t L = 0, Sm = 0, A = 0, N = 0;
    double ps = 0.0;
    for (int t = 0; t < T; ++t) {
        if (T > 1) pthread_join(th[t], NULL);
        for (size_t k = 0; k < npx; ++k) accum[k] += jobs[t].accum[k];
        free(jobs[t].accum);
        L += jobs[t].n_large;
        Sm += jobs[t].n_small;
        A += jobs[t].accepts;
        N += jobs[t].splats;
        ps += jobs[t].p_sum_large;
    }
    out4[0] = L; out4[1] = Sm; out4[2] = A; out4[3] = N;
    *p_sum_large += ps;
    free(jobs);
    free(th);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient of the integrand w.r.t. the PSS coordinates, for the Langevin     */
/* local dynamics (MALA, Section 9's second family).  Forward mode: every     */
/* quantity that depends continuously on x carries its D partial derivatives. */
/* In this path sampler F depends continuously on x only through the camera   */
/* direction, the scattered directions and the modified Phong weights         */
/* (Lambertian and dielectric weights are constant, and the hit points only   */
/* select triangles, which is piecewise constant); so origins and hit points  */
/* carry no derivatives.  The result is the gradient almost everywhere; at a  */
/* change of the hit triangle, the bounce type or the Fresnel choice it is    */
/* the one-sided gradient of the piece the state lies in.                     */
/* ------------------------------------------------------------------------- */
typedef struct { double v; double g[ORC_MAX_DIM]; } dnum;
typedef struct { dnum x, y, z; } dvec;
static _Thread_local int g_dn_D = 0;   /* the active dimension D, set per evaluation */

static dnum dn_c(double v) { dnum r; r.v = v; memset(r.g, 0, sizeof(r.g)); return r; }
static dnum dn_var(double v, int i) { dnum r = dn_c(v); r.g[i] = 1.0; return r; }
static dnum dn_add(dnum a, dnum b) { dnum r; r.v = a.v + b.v; for (int i = 0; i < g_dn_D; ++i) r.g[i] = a.g[i] + b.g[i]; return r; }
static dnum dn_sub(dnum a, dnum b) { dnum r; r.v = a.v - b.v; for (int i = 0; i < g_dn_D; ++i) r.g[i] = a.g[i] - b.g[i]; return r; }
static dnum dn_mul(dnum a, dnum b)
{
    dnum r; r.v = a.v * b.v;
    for (int i = 0; i < g_dn_D; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
    return r;
}
static dnum dn_scl(dnum a, double s) { dnum r; r.v = a.v * s; for (int i = 0; i < g_dn_D; ++i) r.g[i] = a.g[i] * s; return r; }
static dnum dn_div(dnum a, dnum b)
{
    dnum r; r.v = a.v / b.v;
    for (int i = 0; i < g_dn_D; ++i) r.g[i] = (a.g[i] * b.v - a.v * b.g[i]) / (b.v * b.v);
    return r;
}
static dnum dn_sqrt(dnum a)
{
    dnum r; r.v = sqrt(a.v > 0.0 ? a.v : 0.0);
    for (int i = 0; i < g_dn_D; ++i) r.g[i] = r.v > 0.0 ? 0.5 * a.g[i] / r.v : 0.0;
    return r;
}
static dnum dn_pow(dnum a, double e)   /* a^e, a > 0 */
{
    dnum r; r.v = pow(a.v, e);
    double d = a.v > 0.0 ? e * pow(a.v, e - 1.0) : 0.0;
    for (int i = 0; i < g_dn_D; ++i) r.g[i] = d * a.g[i];
    return r;
}
static dnum dn_cos(dnum a) { dnum r; r.v = cos(a.v); for (int i = 0; i < g_dn_D; ++i) r.g[i] = -sin(a.v) * a.g[i]; return r; }
static dnum dn_sin(dnum a) { dnum r; r.v = sin(a.v); for (int i = 0; i < g_dn_D; ++i) r.g[i] = cos(a.v) * a.g[i]; return r; }
static dvec dv_c(v3 a) { dvec r; r.x = dn_c(a.x); r.y = dn_c(a.y); r.z = dn_c(a.z); return r; }
static v3 dv_val(dvec a) { return mk(a.x.v, a.y.v, a.z.v); }
static dvec dv_add(dvec a, dvec b) { dvec r; r.x = dn_add(a.x, b.x); r.y = dn_add(a.y, b.y); r.z = dn_add(a.z, b.z); return r; }
static dvec dv_sub(dvec a, dvec b) { dvec r; r.x = dn_sub(a.x, b.x); r.y = dn_sub(a.y, b.y); r.z = dn_sub(a.z, b.z); return r; }
static dvec dv_scl(dvec a, dnum s) { dvec r; r.x = dn_mul(a.x, s); r.y = dn_mul(a.y, s); r.z = dn_mul(a.z, s); return r; }
static dvec dv_sclc(dvec a, double s) { dvec r; r.x = dn_scl(a.x, s); r.y = dn_scl(a.y, s); r.z = dn_scl(a.z, s); return r; }
static dvec dv_cmul(dvec a, v3 c) { dvec r; r.x = dn_scl(a.x, c.x); r.y = dn_scl(a.y, c.y); r.z = dn_scl(a.z, c.z); return r; }
static dnum dv_dot(dvec a, dvec b) { return dn_add(dn_add(dn_mul(a.x, b.x), dn_mul(a.y, b.y)), dn_mul(a.z, b.z)); }
static dnum dv_dotc(dvec a, v3 c) { return dn_add(dn_add(dn_scl(a.x, c.x), dn_scl(a.y, c.y)), dn_scl(a.z, c.z)); }
static dvec dv_normalize(dvec a) { dnum l = dn_sqrt(dv_dot(a, a)); dvec r; r.x = dn_div(a.x, l); r.y = dn_div(a.y, l); r.z = dn_div(a.z, l); return r; }

/* Duff et al.'s basis around the unit vector n, with derivatives. */
static void dv_onb(dvec n, dvec* t, dvec* b)
{
    double sign = copysign(1.0, n.z.v);
    dnum a = dn_div(dn_c(-1.0), dn_add(dn_c(sign), n.z));
    dnum bb = dn_mul(dn_mul(n.x, n.y), a);
    t->x = dn_add(dn_c(1.0), dn_scl(dn_mul(dn_mul(n.x, n.x), a), sign));
    t->y = dn_scl(bb, sign);
    t->z = dn_scl(n.x, -sign);
    b->x = bb;
    b->y = dn_add(dn_c(sign), dn_mul(dn_mul(n.y, n.y), a));
    b->z = dn_scl(n.y, -1.0);
}

/* The scatter of the path sampler (same branches as scatter()), on dual      *
 * directions; u1, u2 are the bounce's coordinates (dual).                    */
static int scatter_d(const orc_material* m, dvec d, v3 ng, dnum u1, dnum u2, dvec* wi, dvec* w)
{
    if (m->type == ORC_DIELECTRIC) {
        dnum cos_i = dn_scl(dv_dotc(d, ng), -1.0);
        double eta_i = 1.0, eta_t = m->ior;
        v3 nn = ng;
        if (cos_i.v < 0.0) { cos_i = dn_scl(cos_i, -1.0); eta_i = m->ior; eta_t = 1.0; nn = scl(ng, -1.0); }
        double e = eta_i / eta_t;
        dnum sin2_t = dn_scl(dn_sub(dn_c(1.0), dn_mul(cos_i, cos_i)), e * e);
        double cos_t_v;
        double R = fresnel_dielectric(cos_i.v, eta_i, eta_t, &cos_t_v);
        dvec nnd = dv_c(nn);
        if (u1.v < R) {
            *wi = dv_add(d, dv_scl(nnd, dn_scl(cos_i, 2.0)));
        } else {
            dnum cos_t = dn_sqrt(dn_sub(dn_c(1.0), sin2_t));
            *wi = dv_add(dv_sclc(d, e), dv_scl(nnd, dn_sub(dn_scl(cos_i, e), cos_t)));
        }
        *w = dv_c(mk(1.0, 1.0, 1.0));
        return 1;
    }
    v3 ns = dot(dv_val(d), ng) < 0.0 ? ng : scl(ng, -1.0);
    dvec t, b;
    if (m->type == ORC_LAMBERT) {
        dnum r = dn_sqrt(u1), phi = dn_scl(u2, 2.0 * M_PI);
        dnum lz = dn_sqrt(dn_sub(dn_c(1.0), u1));
        v3 tc, bc;
        onb(ns, &tc, &bc);
        *wi = dv_add(dv_add(dv_scl(dv_c(tc), dn_mul(r, dn_cos(phi))), dv_scl(dv_c(bc), dn_mul(r, dn_sin(phi)))),
                     dv_scl(dv_c(ns), lz));
        *w = dv_c(m->albedo);
        return m->albedo.x > 0.0 || m->albedo.y > 0.0 || m->albedo.z > 0.0;
    }
    dvec nsd = dv_c(ns);
    dvec r = dv_sub(d, dv_scl(nsd, dn_scl(dv_dotc(d, ns), 2.0)));
    double n = m->phong_n;
    dnum cos_a = dn_pow(dn_sub(dn_c(1.0), u1), 1.0 / (n + 1.0));
    dnum sin_a = dn_sqrt(dn_sub(dn_c(1.0), dn_mul(cos_a, cos_a)));
    dnum phi = dn_scl(u2, 2.0 * M_PI);
    dv_onb(r, &t, &b);
    *wi = dv_add(dv_add(dv_scl(t, dn_mul(sin_a, dn_cos(phi))), dv_scl(b, dn_mul(sin_a, dn_sin(phi)))), dv_scl(r, cos_a));
    dnum cos_i = dv_dotc(*wi, ns);
    if (cos_i.v <= 0.0) return 0;
    *w = dv_sclc(dv_c(m->albedo), 0.0);
    w->x = dn_scl(cos_i, m->albedo.x * (n + 2.0) / (n + 1.0));
    w->y = dn_scl(cos_i, m->albedo.y * (n + 2.0) / (n + 1.0));
    w->z = dn_scl(cos_i, m->albedo.z * (n + 2.0) / (n + 1.0));
    return 1;
}

/* F(x) and dF/dx (3 x D, row-major by channel).  Same path as eval_path(). */
static void eval_path_grad(const orc_scene* s, int depth, int D, const double* x, v3* F_out, double* dF)
{
    g_dn_D = D;
    dvec F = dv_c(mk(0, 0, 0)), T = dv_c(mk(1, 1, 1));
    v3 o = s->cam_o;
    dnum x0 = dn_var(x[0], 0), x1 = dn_var(x[1], 1);
    dvec d = dv_add(dv_c(s->cam_f), dv_add(dv_scl(dv_c(s->cam_r), dn_sub(dn_scl(x0, 2.0), dn_c(1.0))),
                                           dv_scl(dv_c(s->cam_u), dn_sub(dn_c(1.0), dn_scl(x1, 2.0)))));
    d = dv_normalize(d);
    for (int v = 0; v <= depth; ++v) {
        double t;
        v3 dv = dv_val(d);
        int id = closest_hit(s, o, dv, &t);
        if (id < 0) break;
        const orc_material* m = &s->mats[s->mat[id]];
        v3 ng = s->ng[id];
        v3 p = add(o, scl(dv, t));
        if (m->emits && -dot(dv, ng) > 0.0) F = dv_add(F, dv_cmul(T, m->emission));
        if (v == depth) break;
        dvec wi, w;
        dnum u1 = dn_var(x[2 + 2 * v], 2 + 2 * v), u2 = dn_var(x[3 + 2 * v], 3 + 2 * v);
        if (!scatter_d(m, d, ng, u1, u2, &wi, &w)) break;
        dvec Tn;
        Tn.x = dn_mul(T.x, w.x); Tn.y = dn_mul(T.y, w.y); Tn.z = dn_mul(T.z, w.z);
        T = Tn;
        if (T.x.v == 0.0 && T.y.v == 0.0 && T.z.v == 0.0) break;
        v3 wv = dv_val(wi);
        v3 off = dot(wv, ng) >= 0.0 ? ng : scl(ng, -1.0);
        double mx = fabs(p.x);
        if (fabs(p.y) > mx) mx = fabs(p.y);
        if (fabs(p.z) > mx) mx = fabs(p.z);
        o = add(p, scl(off, ORC_EPS_OFFSET * (1.0 + mx)));
        d = wi;
    }
    *F_out = dv_val(F);
    for (int i = 0; i < D; ++i) {
        dF[i] = F.x.g[i];
        dF[D + i] = F.y.g[i];
        dF[2 * D + i] = F.z.g[i];
    }
}

/* F and dF/dx of the analytic target (the definition differentiated by hand: *
 * q = sum_i w_i exp(-r_i^2 / (2 s_i^2)), F = q (0.5 + x0, 1, 0.5 + x1), zero  *
 * inside the band a <= x0 < b; the band edges are jumps, where the gradient  *
 * of the piece the state lies in is taken).                                  */
static void eval_analytic_grad(const orc_analytic* a, int D, const double* x, v3* F_out, double* dF)
{
    for (int i = 0; i < 3 * D; ++i) dF[i] = 0.0;
    double x0 = x[0], x1 = D >= 2 ? x[1] : 0.0;
    if (x0 >= a->band_a && x0 < a->band_b) { *F_out = mk(0, 0, 0); return; }
    double q = 0.0, dq0 = 0.0, dq1 = 0.0;
    for (int i = 0; i < a->n_modes; ++i) {
        double dx = x0 - a->m0[i], dy = D >= 2 ? x1 - a->m1[i] : 0.0;
        double s2 = a->sd[i] * a->sd[i];
        double e = a->w[i] * exp(-(dx * dx + dy * dy) / (2.0 * s2));
        q += e;
        dq0 += -dx / s2 * e;
        dq1 += -dy / s2 * e;
    }
    *F_out = mk(q * (0.5 + x0), q, q * (0.5 + x1));
    dF[0] = dq0 * (0.5 + x0) + q;       /* dF_r / dx0 */
    dF[D] = dq0;                        /* dF_g / dx0 */
    dF[2 * D] = dq0 * (0.5 + x1);       /* dF_b / dx0 */
    if (D >= 2) {
        dF[1] = dq1 * (0.5 + x0);
        dF[D + 1] = dq1;
        dF[2 * D + 1] = dq1 * (0.5 + x1) + q;
    }
}

ORC_EXPORT void orc_analytic_grad(const orc_analytic* a, int D, uint64_t n, const double* x, double* F3, double* dF)
{
    for (uint64_t i = 0; i < n; ++i) {
        v3 F;
        eval_analytic_grad(a, D, x + i * (uint64_t)D, &F, dF + i * 3 * (uint64_t)D);
        F3[3 * i] = F.x; F3[3 * i + 1] = F.y; F3[3 * i + 2] = F.z;
    }
}

/* Public: F and dF/dx (n x 3 x D) for states x (row-major n x D). */
ORC_EXPORT void orc_eval_grad(const orc_scene* s, int D, int depth, uint64_t n, const double* x, double* F3, double* dF)
{
    for (uint64_t i = 0; i < n; ++i) {
        v3 F;
        eval_path_grad(s, depth, D, x + i * (uint64_t)D, &F, dF + i * 3 * (uint64_t)D);
        F3[3 * i] = F.x; F3[3 * i + 1] = F.y; F3[3 * i + 2] = F.z;
    }
}

/* ------------------------------------------------------------------------- */
/* Langevin local dynamics (MALA): one MH step (Alg. 1) with the proposal     */
/* y = (x + m(x) + sigma N) mod 1, m(x) = clamp(sigma^2/2 grad log p(x),      */
/* -2 sigma, 2 sigma) per coordinate (the clamp keeps the drift of a sharp    */
/* Phong lobe from throwing the proposal across the torus; any deterministic  */
/* drift gives a valid proposal), and acceptance                              */
/* min(1, p(y) q(x|y) / (p(x) q(y|x))), q(y|x) = prod_d phi_sigma(y_d - x_d - */
/* m_d(x)) on the signed torus difference (the nearest image; the others are */
/* below exp(-50) for sigma <= 0.05).  MALA leaves pi invariant, so          */
/* "MALA Restore" keeps the killing rate c~ u / p of Section 6.2; the MALA    */
/* baseline is the mixture of a large step (prob. l, uniform, acceptance      */
/* min(1, p(y)/p(x))) and a MALA step, each with its own MH acceptance.        */
/* State row: x[D], F.rgb, p, u, m[D] (the drift at x).                        */
/* ------------------------------------------------------------------------- */
static void mala_eval(const orc_params* P, const double* x, double* row, double sigma)
{
    int D = P->D;
    v3 F;
    double dF[3 * ORC_MAX_DIM];
    if (P->target_kind == 0) eval_path_grad(P->scene, P->depth, D, x, &F, dF);
    else eval_analytic_grad(P->analytic, D, x, &F, dF);
    for (int d = 0; d < D; ++d) row[d] = x[d];
    row[D] = F.x; row[D + 1] = F.y; row[D + 2] = F.z;
    double p = lum(F);
    row[D + 3] = p;
    row[D + 4] = 1.0;
    for (int d = 0; d < D; ++d) {
        double g = p > 0.0 ? (0.2126 * dF[d] + 0.7152 * dF[D + d] + 0.0722 * dF[2 * D + d]) / p : 0.0;
        double m = isfinite(g) ? 0.5 * sigma * sigma * g : 0.0;
        if (m > 2.0 * sigma) m = 2.0 * sigma;
        if (m < -2.0 * sigma) m = -2.0 * sigma;
        row[D + 5 + d] = m;
    }
}

static double torus_delta(double to, double from)
{
    double d = to - from;
    return d - floor(d + 0.5);
}

/* log q(y | x) up to the constant, from x's drift m */
static double mala_log_q(const double* y, const double* x, const double* m, int D, double sigma)
{
    double s = 0.0;
    for (int d = 0; d < D; ++d) {
        double e = torus_delta(y[d], x[d]) - m[d];
        s += e * e;
    }
    return -s / (2.0 * sigma * sigma);
}

typedef struct {
    const orc_params* P;
    int method;           /* 0: Jump Restore with MALA local moves; 1: MH baseline with MALA small steps;
                             2: as 1 but with the Hastings ratio dropped -- a deliberately wrong kernel that
                                only the tests' negative control runs */
    double ell;
    uint64_t burn_in, chain_begin, c_lo, c_hi, step_begin, n_steps;
    double* state;        /* stride 2 D + 5 */
    double* accum;
    uint64_t J, locals, accepts, splats;
    double p_sum_large;
    uint8_t* tr_flags;
    int32_t* tr_pix;
    double* tr_margin;    /* log of the acceptance ratio minus log U_a (local / small steps), else 0 */
} orc_mala_job;

static void* mala_worker(void* arg)
{
    orc_mala_job* jb = (orc_mala_job*)arg;
    const orc_params* P = jb->P;
    int D = P->D, S = 2 * D + 5;
    double WH = (double)P->width * (double)P->height;
    double v[ORC_MAX_DIM + 8], y[ORC_MAX_DIM], cand[2 * ORC_MAX_DIM + 5];
    for (uint64_t c = jb->c_lo; c < jb->c_hi; ++c) {
        double* st = jb->state + c * S;
        uint32_t chain = (uint32_t)(jb->chain_begin + c);
        for (uint64_t i = 0; i < jb->n_steps; ++i) {
            uint64_t step = jb->step_begin + i;
            double U[4];
            draw_block(P->seed, ORC_TAG_STEP, 0, chain, step, U);
            double p = st[D + 3], u = st[D + 4];
            int local;
            double dt = 0.0, wgt = 0.0;
            if (jb->method == 0) {   /* Alg. 2 clocks, killing rate c~ u / p */
                double t1 = -log(1.0 - U[0]);
                double t2 = p > 0.0 ? -log(1.0 - U[1]) * p / (P->c_tilde * u) : 0.0;
                local = t1 < t2;
                dt = local ? t1 : t2;
                wgt = P->c_tilde * dt * WH / (p > 0.0 ? p : 1.0);
            } else {                 /* MH baseline: large step with probability l */
                local = !(U[0] < jb->ell);
                if (step >= jb->burn_in) { dt = 1.0; jb->splats += 1; }
                wgt = WH / (p > 0.0 ? p : 1.0);
            }
            int pix = -1;
            if (dt > 0.0 && p > 0.0) {
                int px, py;
                pixel_of(P, st, &px, &py);
                pix = py * P->width + px;
                double* a = jb->accum + 4 * (size_t)pix;
                a[0] += wgt * st[D]; a[1] += wgt * st[D + 1]; a[2] += wgt * st[D + 2]; a[3] += dt;
            }
            draw_coords(P->seed, ORC_TAG_STEP, chain, step, D, v);
            int accepted = 0;
            double margin = 0.0;
            if (local) {   /* MALA proposal from the drift cached with the state */
                const double* m = st + D + 5;
                for (int k = 0; k < (D + 1) / 2; ++k) {
                    double R = sqrt(-2.0 * log(1.0 - v[2 * k]));
                    double ang = 2.0 * M_PI * v[2 * k + 1];
                    y[2 * k] = wrap01(st[2 * k] + m[2 * k] + P->sigma * R * cos(ang));
                    if (2 * k + 1 < D) y[2 * k + 1] = wrap01(st[2 * k + 1] + m[2 * k + 1] + P->sigma * R * sin(ang));
                }
                mala_eval(P, y, cand, P->sigma);
                double py = cand[D + 3];
                if (!(p > 0.0)) {
                    accepted = 1;
                } else if (py > 0.0) {
                    double la = log(py) - log(p);
                    if (jb->method != 2)
                        la += mala_log_q(st, y, cand + D + 5, D, P->sigma) - mala_log_q(y, st, m, D, P->sigma);
                    margin = la - log(U[2]);
                    accepted = U[2] > 0.0 ? margin > 0.0 : 1;
                }
                if (accepted) memcpy(st, cand, sizeof(double) * (size_t)S);
                jb->locals += 1;
                jb->accepts += (uint64_t)accepted;
            } else if (jb->method == 0) {   /* regeneration from mu */
                mala_eval(P, v, st, P->sigma);
                jb->J += 1;
            } else {                        /* MH large step: uniform, symmetric */
                mala_eval(P, v, cand, P->sigma);
                double py = cand[D + 3];
                jb->J += 1;
                jb->p_sum_large += py;
                accepted = U[2] < orc_mh_accept_prob(p, py);
                margin = U[2] * p - py;
                if (accepted) memcpy(st, cand, sizeof(double) * (size_t)S);
                jb->accepts += (uint64_t)accepted;
            }
            if (jb->tr_flags) {
                size_t o = (size_t)c * jb->n_steps + i;
                jb->tr_flags[o] = (uint8_t)((local ? 0 : 1) | (accepted ? 2 : 0));
                jb->tr_pix[o] = pix;
                if (jb->tr_margin) jb->tr_margin[o] = margin;
            }
        }
    }
    return NULL;
}

/* Public: initial states (x0 ~ mu, tag 1) with F, p, u and the drift. */
ORC_EXPORT void orc_mala_init(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                              double sigma, uint64_t seed, uint64_t chain_begin, uint64_t n, double* state)
{
    orc_params P = make_params(target_kind, scene, an, D, depth, 1, 1, 1.0, sigma, seed, 0);
    double v[ORC_MAX_DIM + 8];
    for (uint64_t c = 0; c < n; ++c) {
        draw_coords(seed, ORC_TAG_INIT, (uint32_t)(chain_begin + c), 0, D, v);
        mala_eval(&P, v, state + c * (uint64_t)(2 * D + 5), sigma);
    }
}

/* Public: advance MALA chains.  method 0 = Jump Restore (J = regenerations,   *
 * out4 = (J, local steps, accepted, 0)); method 1 = MH baseline (out4 =       *
 * (large steps, small steps, accepted, splatted iterations), p_sum_large).    */
ORC_EXPORT int orc_mala_advance(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                                int width, int height, double sigma, double c_tilde, int method, double ell,
                                uint64_t burn_in, uint64_t seed, uint64_t chain_begin, uint64_t n,
                                uint64_t step_begin, uint64_t n_steps, double* state, double* accum, uint64_t* out4,
                                double* p_sum_large, uint8_t* tr_flags, int32_t* tr_pix, double* tr_margin,
                                int n_threads)
{
    if (D > ORC_MAX_DIM || D < 2) return -1;
    orc_params P = make_params(target_kind, scene, an, D, depth, width, height, c_tilde, sigma, seed, 0);
    int T = resolve_threads(n_threads, n);
    orc_mala_job* jobs = (orc_mala_job*)calloc((size_t)T, sizeof(orc_mala_job));
    pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
    size_t npx = (size_t)width * (size_t)height * 4;
    for (int t = 0; t < T; ++t) {
        orc_mala_job* jb = &jobs[t];
        jb->P = &P; jb->method = method; jb->ell = ell; jb->burn_in = burn_in;
        jb->chain_begin = chain_begin;
        jb->c_lo = n * (uint64_t)t / (uint64_t)T;
        jb->c_hi = n * (uint64_t)(t + 1) / (uint64_t)T;
        jb->step_begin = step_begin; jb->n_steps = n_steps; jb->state = state;
        jb->accum = (double*)calloc(npx, sizeof(double));
        jb->tr_flags = tr_flags; jb->tr_pix = tr_pix; jb->tr_margin = tr_margin;
        if (T > 1) pthread_create(&th[t], NULL, mala_worker, jb);
    }
    if (T == 1) mala_worker(&jobs[0]);
    uint64_t J = 0, L = 0, A = 0, N = 0;
    double ps = 0.0;
    for (int t = 0; t < T; ++t) {
        if (T > 1) pthread_join(th[t], NULL);
        for (size_t k = 0; k < npx; ++k) accum[k] += jobs[t].accum[k];
        free(jobs[t].accum);
        J += jobs[t].J; L += jobs[t].locals; A += jobs[t].accepts; N += jobs[t].splats; ps += jobs[t].p_sum_large;
    }
    out4[0] = J; out4[1] = L; out4[2] = A; out4[3] = N;
    *p_sum_large += ps;
    free(jobs);
    free(th);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* General Restore (Section 6.1, eq. "killing-rate"; supplement, Theorem A):  */
/* local dynamics that need not leave pi invariant, so the killing rate keeps */
/* the adjoint term: k = ((L* + kappa mu*) p) / p.  With state-independent mu */
/* of density u, kappa mu* p = c~ u with c~ = kappa p_lambda, and             */
/* k = (L* p + c~ u) / p.                                                     */
/* ------------------------------------------------------------------------- */
ORC_EXPORT double orc_killing_rate_general(double p, double lstar_p, double kappa_mustar_p)
{
    return p > 0.0 ? (lstar_p + kappa_mustar_p) / p : INFINITY;
}

/* Local dynamics of the continuous general Restore below: the unadjusted     *
 * Gaussian random walk on the unit torus, y = (x + sigma N) mod 1, always    *
 * taken (no MH correction), run as the jump process of Section 7.1 (holding  *
 * times Exp(1)).  Its generator is L f = zeta f - f, so                       *
 * (L* p)(x) = integral over [0,1) of p(y) zeta(y, x) dy - p(x), with          *
 * zeta(y, x) the wrapped normal density sum_k phi_sigma(x - y + k).  The     *
 * integral is a midpoint rule on n_quad points (1-D analytic targets).       */
static double wrapped_normal(double d, double sigma)
{
    double s = 0.0;
    for (int k = -3; k <= 3; ++k) {
        double z = (d + k) / sigma;
        s += exp(-0.5 * z * z);
    }
    return s / (sigma * sqrt(2.0 * M_PI));
}

static double lstar_p_1d(const orc_analytic* an, double x, double sigma, int n_quad)
{
    double acc = 0.0, h = 1.0 / n_quad;
    for (int q = 0; q < n_quad; ++q) {
        double y = (q + 0.5) * h;
        v3 F = eval_analytic(an, 1, &y);
        acc += lum(F) * wrapped_normal(x - y, sigma);
    }
    v3 Fx = eval_analytic(an, 1, &x);
    return acc * h - lum(Fx);
}

ORC_EXPORT void orc_lstar_p_1d(const orc_analytic* an, int n, const double* x, double sigma, int n_quad, double* out)
{
    for (int i = 0; i < n; ++i) out[i] = lstar_p_1d(an, x[i], sigma, n_quad);
}

typedef struct {
    const orc_analytic* an;
    double sigma, c_tilde;
    int n_quad, W, simplified;
    uint64_t seed, chain_begin, c_lo, c_hi, step_begin, n_steps;
    double* state;    /* per chain: x, p, k */
    double* accum;    /* W*4 */
    uint64_t J;
} orc_gen_job;

static void gen_eval(const orc_gen_job* jb, double x, double* p, double* k)
{
    v3 F = eval_analytic(jb->an, 1, &x);
    *p = lum(F);
    double ls = jb->simplified ? 0.0 : lstar_p_1d(jb->an, x, jb->sigma, jb->n_quad);
    *k = orc_killing_rate_general(*p, ls, jb->c_tilde * 1.0 /* u = 1 */);
}

static void* gen_worker(void* arg)
{
    orc_gen_job* jb = (orc_gen_job*)arg;
    for (uint64_t c = jb->c_lo; c < jb->c_hi; ++c) {
        double* st = jb->state + 3 * c;
        uint32_t chain = (uint32_t)(jb->chain_begin + c);
        for (uint64_t i = 0; i < jb->n_steps; ++i) {
            uint64_t step = jb->step_begin + i;
            double U[4], V[4];
            draw_block(jb->seed, ORC_TAG_STEP, 0, chain, step, U);
            draw_block(jb->seed, ORC_TAG_STEP, 1, chain, step, V);
            double x = st[0], p = st[1], k = st[2];
            /* Alg. 2 clocks with the general killing rate */
            double t1 = -log(1.0 - U[0]);
            double t2 = isinf(k) ? 0.0 : -log(1.0 - U[1]) / k;
            int local = t1 < t2;
            double dt = local ? t1 : t2;
            if (dt > 0.0 && p > 0.0) {
                int px = (int)floor(x * jb->W);
                if (px >= jb->W) px = jb->W - 1;
                v3 F = eval_analytic(jb->an, 1, &x);
                double wgt = jb->c_tilde * dt * jb->W / p;
                double* a = jb->accum + 4 * (size_t)px;
                a[0] += wgt * F.x; a[1] += wgt * F.y; a[2] += wgt * F.z; a[3] += dt;
            }
            double y;
            if (local) { /* the unadjusted random walk: always moves */
                double R = sqrt(-2.0 * log(1.0 - V[0]));
                y = wrap01(x + jb->sigma * R * cos(2.0 * M_PI * V[1]));
            } else {     /* regeneration from mu = uniform */
                y = V[0];
                jb->J += 1;
            }
            st[0] = y;
            gen_eval(jb, y, &st[1], &st[2]);
        }
    }
    return NULL;
}

/* Public: n chains of the general Restore process on a 1-D analytic target   *
 * (state rows x, p, k; initialise with orc_general_init).  simplified = 1    *
 * drops the L* p term (the killing rate of pi-invariant dynamics: a          *
 * deliberately wrong choice for this local dynamics, the negative control).  */
ORC_EXPORT void orc_general_init(const orc_analytic* an, double sigma, double c_tilde, int n_quad, int simplified,
                                 uint64_t seed, uint64_t chain_begin, uint64_t n, double* state)
{
    orc_gen_job jb;
    memset(&jb, 0, sizeof(jb));
    jb.an = an; jb.sigma = sigma; jb.c_tilde = c_tilde; jb.n_quad = n_quad; jb.simplified = simplified;
    for (uint64_t c = 0; c < n; ++c) {
        double v[ORC_MAX_DIM + 8];
        draw_coords(seed, ORC_TAG_INIT, (uint32_t)(chain_begin + c), 0, 1, v);
        state[3 * c] = v[0];
        gen_eval(&jb, v[0], &state[3 * c + 1], &state[3 * c + 2]);
    }
}

ORC_EXPORT uint64_t orc_general_advance(const orc_analytic* an, int width, double sigma, double c_tilde, int n_quad,
                                        int simplified, uint64_t seed, uint64_t chain_begin, uint64_t n,
                                        uint64_t step_begin, uint64_t n_steps, double* state, double* accum,
                                        int n_threads)
{
    int T = resolve_threads(n_threads, n);
    orc_gen_job* jobs = (orc_gen_job*)calloc((size_t)T, sizeof(orc_gen_job));
    pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
    size_t npx = (size_t)width * 4;
    for (int t = 0; t < T; ++t) {
        orc_gen_job* jb = &jobs[t];
        jb->an = an; jb->sigma = sigma; jb->c_tilde = c_tilde; jb->n_quad = n_quad; jb->W = width;
        jb->simplified = simplified; jb->seed = seed; jb->chain_begin = chain_begin;
        jb->c_lo = n * (uint64_t)t / (uint64_t)T;
        jb->c_hi = n * (uint64_t)(t + 1) / (uint64_t)T;
        jb->step_begin = step_begin; jb->n_steps = n_steps; jb->state = state;
        jb->accum = (double*)calloc(npx, sizeof(double));
        if (T > 1) pthread_create(&th[t], NULL, gen_worker, jb);
    }
    if (T == 1) gen_worker(&jobs[0]);
    uint64_t J = 0;
    for (int t = 0; t < T; ++t) {
        if (T > 1) pthread_join(th[t], NULL);
        for (size_t k = 0; k < npx; ++k) accum[k] += jobs[t].accum[k];
        free(jobs[t].accum);
        J += jobs[t].J;
    }
    free(jobs);
    free(th);
    return J;
}

/* Public: F, p, u, k for given states (row-major n x D).  hit_ids optional,   *
 * n x (depth+1).                                                             */
ORC_EXPORT void orc_eval_states(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                                double c_tilde, uint64_t n, const double* x, double* F3, double* p, double* u,
                                double* k, int32_t* hit_ids)
{
    orc_params P = make_params(target_kind, scene, an, D, depth, 1, 1, c_tilde, 0.0, 0, 0);
    for (uint64_t i = 0; i < n; ++i) {
        const double* xi = x + i * (uint64_t)D;
        v3 F;
        double pp;
        int ids[ORC_MAX_DIM];
        eval_target(&P, xi, &F, &pp, hit_ids ? ids : NULL);
        if (hit_ids) for (int v = 0; v <= depth; ++v) hit_ids[i * (uint64_t)(depth + 1) + (uint64_t)v] = ids[v];
        F3[3 * i] = F.x; F3[3 * i + 1] = F.y; F3[3 * i + 2] = F.z;
        p[i] = pp;
        u[i] = regen_density(&P, xi);
        k[i] = orc_killing_rate(pp, u[i], c_tilde);
    }
}

/* ------------------------------------------------------------------------- */
/* Plain Monte Carlo path tracing (the regeneration-only estimator; converged */
/* references).  Sample s uses tag 2.  accum (W*H*4) gets W H F(x) per sample */
/* (channel 3 counts samples); the pixel estimate is accum / n_samples.       */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_params* P;
    uint64_t s_lo, s_hi;
    double* accum;
} orc_pt_job;

static void* pt_worker(void* arg)
{
    orc_pt_job* jb = (orc_pt_job*)arg;
    const orc_params* P = jb->P;
    double v[ORC_MAX_DIM + 8];
    double WH = (double)P->width * (double)P->height;
    for (uint64_t s = jb->s_lo; s < jb->s_hi; ++s) {
        draw_coords(P->seed, ORC_TAG_PT, (uint32_t)s, s >> 32, P->D, v);
        v3 F;
        double p;
        eval_target(P, v, &F, &p, NULL);
        int px, py;
        pixel_of(P, v, &px, &py);
        double* a = jb->accum + 4 * ((size_t)py * P->width + px);
        a[0] += WH * F.x; a[1] += WH * F.y; a[2] += WH * F.z; a[3] += 1.0;
    }
    return NULL;
}

ORC_EXPORT void orc_render_pt(int target_kind, const orc_scene* scene, const orc_analytic* an, int D, int depth,
                              int width, int height, uint64_t seed, uint64_t sample_begin, uint64_t n_samples,
                              double* accum, int n_threads)
{
    orc_params P = make_params(target_kind, scene, an, D, depth, width, height, 1.0, 0.0, seed, 0);
    int T = resolve_threads(n_threads, n_samples);
    orc_pt_job* jobs = (orc_pt_job*)calloc((size_t)T, sizeof(orc_pt_job));
    pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
    size_t npx = (size_t)width * (size_t)height * 4;
    for (int t = 0; t < T; ++t) {
        jobs[t].P = &P;
        jobs[t].s_lo = sample_begin + n_samples * (uint64_t)t / (uint64_t)T;
        jobs[t].s_hi = sample_begin + n_samples * (uint64_t)(t + 1) / (uint64_t)T;
        jobs[t].accum = (double*)calloc(npx, sizeof(double));
        if (T > 1) pthread_create(&th[t], NULL, pt_worker, &jobs[t]);
    }
    if (T == 1) pt_worker(&jobs[0]);
    for (int t = 0; t < T; ++t) {
        if (T > 1) pthread_join(th[t], NULL);
        for (size_t k = 0; k < npx; ++k) accum[k] += jobs[t].accum[k];
        free(jobs[t].accum);
    }
    free(jobs);
    free(th);
}

ORC_EXPORT int orc_threads_default(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}
