// Device functions shared by the megakernel (jr_kernels.cu) and the
// wavefront pipeline (jr_wavefront.cu): Philox, vector helpers, BVH
// traversal, BSDF sampling, the PSS path integrand.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/jr.h"
#include "jr_internal.h"

namespace jr {
namespace {

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t tag, uint32_t block, uint32_t chain, uint64_t step) {
    return philox4x32_10(make_uint4(block + 256u * tag, chain, (uint32_t)step, (uint32_t)(step >> 32)),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// (r >> 8) * 2^-24: exact in float, in [0, 1).
__device__ __forceinline__ float u01(uint32_t r) { return (float)(r >> 8) * 5.9604644775390625e-8f; }

// ------------------------------------------------------------------ vectors
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float lum(float3 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }

// Orthonormal basis around unit n (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
    const float sign = copysignf(1.0f, n.z);
    const float a = -1.0f / (sign + n.z);
    const float bb = n.x * n.y * a;
    t = f3(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    b = f3(bb, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float wrap01(float y) {
    const float w = y - floorf(y);
    return w >= 1.0f ? 0.0f : w;
}

// ------------------------------------------------------------------ traversal
constexpr int kSentinel = INT32_MIN;

// Work counters of the instrumented kernel variant (compiled out otherwise).
struct Work {
    uint32_t rays = 0, nodes = 0, tris = 0;
};

// Three-input float min/max (PTX min/max with three sources, sm_100+): one
// instruction where two-input chains take two.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// A ray prepared for slab tests, plus the resumable state of its traversal.
// The stack lives with the caller (per-thread local memory).
struct Trav {
    float3 o, d;
    float ix, iy, iz, ox, oy, oz;
    float tb;          // closest hit so far
    int best, best_id;  // its leaf-order record and original triangle index
    int ref, sp;        // node/leaf ref being visited, stack depth
    uint32_t visits;
    int oct;            // ray octant: bit a set when the direction's axis-a component is negative
};

__device__ __forceinline__ void trav_begin_at(Trav& r, float3 o, float3 d, int root) {
    r.o = o;
    r.d = d;
    const float dx = fabsf(d.x) < 1e-20f ? copysignf(1e-20f, d.x) : d.x;
    const float dy = fabsf(d.y) < 1e-20f ? copysignf(1e-20f, d.y) : d.y;
    const float dz = fabsf(d.z) < 1e-20f ? copysignf(1e-20f, d.z) : d.z;
    r.ix = 1.0f / dx;
    r.iy = 1.0f / dy;
    r.iz = 1.0f / dz;
    r.ox = o.x * r.ix;
    r.oy = o.y * r.iy;
    r.oz = o.z * r.iz;
    r.oct = (r.ix < 0.0f ? 1 : 0) | (r.iy < 0.0f ? 2 : 0) | (r.iz < 0.0f ? 4 : 0);
    r.tb = INFINITY;
    r.best = -1;
    r.best_id = INT32_MAX;
    r.ref = root;
    r.sp = 0;
    r.visits = 0;
}
__device__ __forceinline__ void trav_begin(const SceneView& s, Trav& r, float3 o, float3 d) {
    trav_begin_at(r, o, d, s.root);
}

// Order two (distance, ref) pairs so that the nearer comes first.
__device__ __forceinline__ void cswap(float& ta, int& ra, float& tb, int& rb) {
    const bool sw = tb < ta;
    const float t = sw ? tb : ta;
    tb = sw ? ta : tb;
    ta = t;
    const int q = sw ? rb : ra;
    rb = sw ? ra : rb;
    ra = q;
}

// Slab test of one child box against [0, tb], given its near and far plane
// per axis (picked by the ray's octant, see trav_node): entry distance, or
// +inf for a miss.  The far distance is scaled up by 2 ulp so that a ray
// grazing a face of a (conservatively widened) box still enters it.
__device__ __forceinline__ float slab(const Trav& r, float nx, float fx, float ny, float fy, float nz, float fz) {
    const float tn = fmax3(fmaf(nx, r.ix, -r.ox), fmaf(ny, r.iy, -r.oy), fmaxf(fmaf(nz, r.iz, -r.oz), 0.0f));
    const float tf = fmin3(fmaf(fx, r.ix, -r.ox), fmaf(fy, r.iy, -r.oy), fminf(fmaf(fz, r.iz, -r.oz), r.tb));
    return tn <= tf * 1.00000024f ? tn : INFINITY;
}

// Visit inner node r.ref of the 4-wide BVH: slab-test its children against
// [0, tb], descend to the nearest hit child and push the other hit children
// farthest first (front-to-back order), or pop.  Returns false (and sets a
// status bit) if the visit budget or the stack ran out: the ray then counts
// as a miss.
template <bool kCount>
__device__ __forceinline__ bool trav_node(const SceneView& s, Trav& r, int* stack, unsigned& status, Work& work) {
    if (++r.visits > s.visit_budget) {
        status |= JR_STATUS_TRAVERSAL;
        return false;
    }
    if constexpr (kCount) work.nodes++;
    const Bvh4Node* n = s.nodes + r.ref;
    // The planes are stored lo, hi per axis.  For a positive direction
    // component the lo plane is met first, for a negative one the hi plane:
    // (lo * i - o) <= (hi * i - o) for i > 0 and the reverse for i < 0, and
    // both sides round monotonically, so for finite ray data the octant picks
    // exactly the values min and max would pick (with a NaN in the ray the two
    // forms differ, and such a ray carries no contribution either way).
    const float4* pl = &n->lox;
    const int sx = r.oct & 1, sy = (r.oct >> 1) & 1, sz = (r.oct >> 2) & 1;
    const float4 nx = __ldg(pl + sx), fx = __ldg(pl + (sx ^ 1));
    const float4 ny = __ldg(pl + 2 + sy), fy = __ldg(pl + 2 + (sy ^ 1));
    const float4 nz = __ldg(pl + 4 + sz), fz = __ldg(pl + 4 + (sz ^ 1));
    int4 rf = __ldg(&n->refs);
    float t0 = slab(r, nx.x, fx.x, ny.x, fy.x, nz.x, fz.x);
    float t1 = slab(r, nx.y, fx.y, ny.y, fy.y, nz.y, fz.y);
    float t2 = slab(r, nx.z, fx.z, ny.z, fy.z, nz.z, fz.z);
    float t3 = slab(r, nx.w, fx.w, ny.w, fy.w, nz.w, fz.w);  // an empty slot's box misses (+inf)
    // 5-comparator sorting network on (distance, ref)
    cswap(t0, rf.x, t1, rf.y);
    cswap(t2, rf.z, t3, rf.w);
    cswap(t0, rf.x, t2, rf.z);
    cswap(t1, rf.y, t3, rf.w);
    cswap(t1, rf.y, t2, rf.z);
    const int pushes = (t1 < INFINITY) + (t2 < INFINITY) + (t3 < INFINITY);
    if (r.sp + pushes > s.stack_limit) {
        status |= JR_STATUS_STACK;
        return false;
    }
    if (t3 < INFINITY) stack[r.sp++] = rf.w;
    if (t2 < INFINITY) stack[r.sp++] = rf.z;
    if (t1 < INFINITY) stack[r.sp++] = rf.y;
    if (t0 < INFINITY) r.ref = rf.x;
    else r.ref = r.sp > 0 ? stack[--r.sp] : kSentinel;
    return true;
}

// Test the triangles of leaf `leaf` (Moller-Trumbore, JGT 1997; ties on equal
// t to the smaller original index) against the ray, updating the closest hit.
// Branch-free: every quantity is computed and one predicate takes the hit (the
// early-out form diverged per triangle; measured +0.5 % on the path kernel).
template <bool kCount>
__device__ __forceinline__ void trav_test_leaf(const SceneView& s, Trav& r, int leaf, Work& work) {
    const int enc = ~leaf;
    const int first = enc >> 3, cnt = (enc & 7) + 1;
    if constexpr (kCount) work.tris += (uint32_t)cnt;
    for (int k = first; k < first + cnt; ++k) {
        const TriRecord* tr = s.tris + k;
        const float4 q0 = __ldg(&tr->v0_id), q1 = __ldg(&tr->e1_mat), q2 = __ldg(&tr->e2);
        const float3 e1 = f3(q1.x, q1.y, q1.z), e2 = f3(q2.x, q2.y, q2.z);
        const float3 pv = cross(r.d, e2);
        const float det = dot(e1, pv);
        const float inv = 1.0f / det;
        const float3 tv = r.o - f3(q0.x, q0.y, q0.z);
        const float u = dot(tv, pv) * inv;
        const float3 qv = cross(tv, e1);
        const float v = dot(r.d, qv) * inv;
        const float t = dot(e2, qv) * inv;
        const int id = __float_as_int(q0.w);
        const bool hit = det != 0.0f && !(u < 0.0f || u > 1.0f) && !(v < 0.0f || u + v > 1.0f) && t > 0.0f &&
                         (t < r.tb || (t == r.tb && id < r.best_id));
        r.tb = hit ? t : r.tb;
        r.best = hit ? k : r.best;
        r.best_id = hit ? id : r.best_id;
    }
}

// Test the triangles of leaf r.ref, then pop.  Returns false when the ray is done.
template <bool kCount>
__device__ __forceinline__ bool trav_leaf(const SceneView& s, Trav& r, const int* stack, Work& work) {
    trav_test_leaf<kCount>(s, r, r.ref, work);
    r.ref = r.sp > 0 ? stack[--r.sp] : kSentinel;
    return r.ref != kSentinel;
}

// The inner-node loop of a warp-synchronous traversal round ends once at most
// kSearchExit lanes are still on their way to a leaf (after at least one node
// visit), instead of when none is: the few lanes with the longest way no
// longer hold the warp's other lanes, which test their leaves and go on; the
// rest carry on in the next round.  Measured on the 512^2 Cornell + spheres
// workload (wavefront): 1.04 (exit at 0), 1.17 (4), 1.19 (6 and 8), 1.14 (16)
// x 10^9 chain steps/s.  The exit waits while the searching lanes outnumber
// the others (a sparse warp, late in a drain, has nobody to release and would
// only pay an extra round per node visit).
constexpr int kSearchExit = 6;
__device__ __forceinline__ bool search_done(unsigned searching, unsigned tracing) {
    const int ns = __popc(searching);
    return ns <= kSearchExit && 2 * ns <= __popc(tracing);
}

// Closest hit for the lanes in `mask`, which must all call together (lanes
// without a ray pass want = false).  Warp-synchronous while-while traversal
// (Aila & Laine, HPG 2009): each inner-node round and each leaf round ends in
// a __any_sync over `mask`, so the lanes reconverge every iteration instead of
// drifting apart under independent thread scheduling.  Returns the leaf-order
// record index or -1; t_out gets the hit distance.
template <bool kCount>
__device__ __forceinline__ int closest_hit(const SceneView& s, unsigned mask, bool want, float3 o, float3 d,
                                           float& t_out, unsigned& status, Work& work) {
    Trav r;
    trav_begin(s, r, o, d);
    bool active = want && s.root != kSentinel;
    if constexpr (kCount) work.rays += want ? 1u : 0u;
    int stack[kStackSize];
    while (__any_sync(mask, active)) {
        const unsigned tracing = __ballot_sync(mask, active);
        while (__any_sync(mask, active && r.ref >= 0)) {
            if (active && r.ref >= 0 && !trav_node<kCount>(s, r, stack, status, work)) {
                active = false;
                r.best = -1;
            }
            if (search_done(__ballot_sync(mask, active && r.ref >= 0), tracing)) break;
        }
        if (active && r.ref < 0) active = r.ref != kSentinel && trav_leaf<kCount>(s, r, stack, work);
    }
    t_out = r.best >= 0 ? r.tb : INFINITY;
    return r.best;
}

// ------------------------------------------------------------------ BSDFs
// Exact unpolarised Fresnel reflectance of a smooth dielectric interface.
__device__ __forceinline__ float fresnel(float cos_i, float eta_i, float eta_t, float& cos_t) {
    const float e = eta_i / eta_t;
    const float sin2_t = e * e * (1.0f - cos_i * cos_i);
    if (sin2_t >= 1.0f) {
        cos_t = 0.0f;
        return 1.0f;
    }
    cos_t = sqrtf(1.0f - sin2_t);
    const float rs = (eta_i * cos_i - eta_t * cos_t) / (eta_i * cos_i + eta_t * cos_t);
    const float rp = (eta_t * cos_i - eta_i * cos_t) / (eta_t * cos_i + eta_i * cos_t);
    return 0.5f * (rs * rs + rp * rp);
}

// Sample the continuation direction; returns false when the path ends.
__device__ __forceinline__ bool scatter(const Material& m, float3 d, float3 ng, float u1, float u2, float3& wi,
                                        float3& w) {
    if (m.type == JR_MAT_DIELECTRIC) {
        float cos_i = -dot(d, ng);
        float eta_i = 1.0f, eta_t = m.ior;
        float3 nn = ng;
        if (cos_i < 0.0f) {
            cos_i = -cos_i;
            eta_i = m.ior;
            eta_t = 1.0f;
            nn = ng * -1.0f;
        }
        float cos_t;
        const float R = fresnel(cos_i, eta_i, eta_t, cos_t);
        if (u1 < R) {
            wi = d + nn * (2.0f * cos_i);
        } else {
            const float e = eta_i / eta_t;
            wi = d * e + nn * (e * cos_i - cos_t);
        }
        w = f3(1.0f, 1.0f, 1.0f);
        return true;
    }
    const float3 ns = dot(d, ng) < 0.0f ? ng : ng * -1.0f;
    float3 t, b;
    if (m.type == JR_MAT_LAMBERT) {
        // cosine-weighted hemisphere (Malley's method); weight = albedo
        const float r = sqrtf(u1);
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        const float lz = sqrtf(fmaxf(1.0f - u1, 0.0f));
        onb(ns, t, b);
        wi = t * (r * cs) + b * (r * sn) + ns * lz;
        w = m.albedo;
        return m.albedo.x > 0.0f || m.albedo.y > 0.0f || m.albedo.z > 0.0f;
    }
    // modified Phong lobe about the mirror direction; weight rho (n+2)/(n+1) cos_i
    const float3 r = d - ns * (2.0f * dot(d, ns));
    const float cos_a = powf(1.0f - u1, m.phong_inv_n1);
    const float sin_a = sqrtf(fmaxf(1.0f - cos_a * cos_a, 0.0f));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    onb(r, t, b);
    wi = t * (sin_a * cs) + b * (sin_a * sn) + r * cos_a;
    const float cos_i = dot(wi, ns);
    if (cos_i <= 0.0f) return false;
    w = m.albedo * (m.phong_scale * cos_i);
    return true;
}

// ------------------------------------------------------------------ integrand
// PSS path contribution F(y) (the target of Section 4 is p = lum(F)).  y[d] is
// read at y[d * ys]: film point (y0, y1), bounce b uses (y_{2+2b}, y_{3+2b}).
// Emission (one-sided) is collected at every vertex; a miss ends the path.
// Camera ray through film point (y0, y1).
__device__ __forceinline__ void camera_ray(const SceneView& s, float y0, float y1, float3& o, float3& d) {
    const float3 cf = f3(s.cam[3], s.cam[4], s.cam[5]);
    const float3 cr = f3(s.cam[6], s.cam[7], s.cam[8]);
    const float3 cu = f3(s.cam[9], s.cam[10], s.cam[11]);
    o = f3(s.cam[0], s.cam[1], s.cam[2]);
    d = normalize(cf + cr * (2.0f * y0 - 1.0f) + cu * (1.0f - 2.0f * y1));
}

// One path vertex: the ray (o, d) hit record k at distance t.  Adds the
// one-sided emission T * L_e to F, and unless v == depth samples the
// continuation with (u1, u2) = (y_{2+2v}, y_{3+2v}).  Returns true if the path
// continues, with (o, d, T) updated to the next ray.
__device__ __forceinline__ bool shade_vertex(const SceneView& s, int k, float t, int v, int depth, float u1,
                                             float u2, float3& o, float3& d, float3& T, float3& F) {
    const TriRecord* tr = s.tris + k;
    const float4 q1 = __ldg(&tr->e1_mat), q2 = __ldg(&tr->e2);
    const Material m = s.mats[__float_as_int(q1.w)];
    const float3 ng = normalize(cross(f3(q1.x, q1.y, q1.z), f3(q2.x, q2.y, q2.z)));
    const float3 p = o + d * t;
    if (m.emits && -dot(d, ng) > 0.0f) F = F + mul(T, m.emission);
    if (v == depth) return false;
    float3 wi, w;
    if (!scatter(m, d, ng, u1, u2, wi, w)) return false;
    T = mul(T, w);
    if (T.x == 0.0f && T.y == 0.0f && T.z == 0.0f) return false;
    const float3 off = dot(wi, ng) >= 0.0f ? ng : ng * -1.0f;
    const float mx = fmaxf(fmaxf(fabsf(p.x), fabsf(p.y)), fabsf(p.z));
    o = p + off * (1e-4f * (1.0f + mx));
    d = wi;
    return true;
}

__device__ __forceinline__ float3 finite_or_zero(float3 F, unsigned& status) {
    if (!isfinite(F.x) || !isfinite(F.y) || !isfinite(F.z)) {
        status |= JR_STATUS_NONFINITE;
        return f3(0.f, 0.f, 0.f);
    }
    return F;
}

// The integrand for the lanes in `mask` (all of which must call together;
// lanes with want = false only keep the warp in step).  The bounce loop runs
// until no lane in the warp has a live path.
template <bool kCount>
__device__ __forceinline__ float3 eval_path_w(const SceneView& s, unsigned mask, bool want, int depth, const float* y,
                                              uint32_t ys, int32_t* ids, uint64_t id_stride, unsigned& status,
                                              Work& work) {
    float3 F = f3(0.f, 0.f, 0.f), T = f3(1.f, 1.f, 1.f);
    float3 o = f3(0.f, 0.f, 1.f), d = f3(0.f, 0.f, 1.f);
    if (want) camera_ray(s, y[0], y[ys], o, d);
    if (want && ids)
        for (int v = 0; v <= depth; ++v) ids[v * id_stride] = -1;
    bool alive = want;
    for (int v = 0; v <= depth; ++v) {
        if (!__any_sync(mask, alive)) break;
        float t;
        const int k = closest_hit<kCount>(s, mask, alive, o, d, t, status, work);
        if (alive) {
            if (k < 0) {
                alive = false;
            } else {
                if (ids) ids[v * id_stride] = __float_as_int(__ldg(&s.tris[k].v0_id.w));
                const float u1 = v < depth ? y[(2 + 2 * v) * ys] : 0.0f;
                const float u2 = v < depth ? y[(3 + 2 * v) * ys] : 0.0f;
                alive = shade_vertex(s, k, t, v, depth, u1, u2, o, d, T, F);
            }
        }
    }
    return want ? finite_or_zero(F, status) : F;
}

__device__ __forceinline__ float3 eval_path(const SceneView& s, unsigned mask, bool want, int depth, const float* y,
                                            uint32_t ys, int32_t* ids, uint64_t id_stride, unsigned& status) {
    Work w;
    return eval_path_w<false>(s, mask, want, depth, y, ys, ids, id_stride, status, w);
}

// ------------------------------------------------------------------ gradient
// dF/dx for the Langevin local dynamics (MALA), forward mode.  F depends on x
// continuously only through the directions (camera, scattered) and the modified
// Phong weights (Lambertian and dielectric weights are constant; hit points only
// select triangles), so a lane carries the Jacobians of the current direction,
// of the throughput and of F, 3 x D each: column c is d/dx_c.  A Lambertian
// bounce's direction depends only on its own two coordinates, so its Jacobian
// restarts there.  At a change of hit triangle, bounce type or Fresnel choice the
// result is the gradient of the piece the state lies in.
struct Jac3 {
    float c[3][kMaxDim];
};

// J_out = d(normalize(v))/dx from J_v (v unnormalised, n = v / |v|).
__device__ inline void jac_normalize(float3 n, float inv_len, const Jac3& Jv, Jac3& Jn, int D) {
    for (int k = 0; k < D; ++k) {
        const float dvx = Jv.c[0][k], dvy = Jv.c[1][k], dvz = Jv.c[2][k];
        const float proj = n.x * dvx + n.y * dvy + n.z * dvz;
        Jn.c[0][k] = (dvx - n.x * proj) * inv_len;
        Jn.c[1][k] = (dvy - n.y * proj) * inv_len;
        Jn.c[2][k] = (dvz - n.z * proj) * inv_len;
    }
}

// The scatter of `scatter` with the Jacobian of the outgoing direction (Jwi) and
// the weight's log-derivative contribution: dw[ch][k] = d(weight_ch)/dx_k.
// Jd: Jacobian of the incoming direction d; (u1, u2) are coordinates i1, i1+1.
__device__ inline bool scatter_grad(const Material& m, float3 d, float3 ng, float u1, float u2, int i1, const Jac3& Jd,
                                    float3& wi, float3& w, Jac3& Jwi, Jac3& Jw, int D) {
    for (int q = 0; q < 3; ++q)
        for (int k = 0; k < D; ++k) Jw.c[q][k] = 0.f;
    if (m.type == JR_MAT_DIELECTRIC) {
        float cos_i = -dot(d, ng);
        float eta_i = 1.0f, eta_t = m.ior;
        float3 nn = ng;
        if (cos_i < 0.0f) {
            cos_i = -cos_i;
            eta_i = m.ior;
            eta_t = 1.0f;
            nn = ng * -1.0f;
        }
        float cos_t;
        const float R = fresnel(cos_i, eta_i, eta_t, cos_t);
        const float e = eta_i / eta_t;
        const bool refl = u1 < R;
        if (refl) wi = d + nn * (2.0f * cos_i);
        else wi = d * e + nn * (e * cos_i - cos_t);
        for (int k = 0; k < D; ++k) {
            const float dci = -(nn.x * Jd.c[0][k] + nn.y * Jd.c[1][k] + nn.z * Jd.c[2][k]);
            if (refl) {
                Jwi.c[0][k] = Jd.c[0][k] + 2.0f * nn.x * dci;
                Jwi.c[1][k] = Jd.c[1][k] + 2.0f * nn.y * dci;
                Jwi.c[2][k] = Jd.c[2][k] + 2.0f * nn.z * dci;
            } else {
                const float dct = cos_t > 0.0f ? e * e * cos_i * dci / cos_t : 0.0f;
                const float g = e * dci - dct;
                Jwi.c[0][k] = e * Jd.c[0][k] + nn.x * g;
                Jwi.c[1][k] = e * Jd.c[1][k] + nn.y * g;
                Jwi.c[2][k] = e * Jd.c[2][k] + nn.z * g;
            }
        }
        w = f3(1.0f, 1.0f, 1.0f);
        return true;
    }
    const float3 ns = dot(d, ng) < 0.0f ? ng : ng * -1.0f;
    float3 t, b;
    for (int q = 0; q < 3; ++q)
        for (int k = 0; k < D; ++k) Jwi.c[q][k] = 0.f;
    if (m.type == JR_MAT_LAMBERT) {
        const float r = sqrtf(u1);
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        const float lz = sqrtf(fmaxf(1.0f - u1, 0.0f));
        onb(ns, t, b);
        wi = t * (r * cs) + b * (r * sn) + ns * lz;
        // d/du1 and d/du2 only
        const float dr = r > 0.0f ? 0.5f / r : 0.0f, dlz = lz > 0.0f ? -0.5f / lz : 0.0f;
        const float tw = 2.0f * 3.14159265358979f;
        const float3 d1 = t * (dr * cs) + b * (dr * sn) + ns * dlz;
        const float3 d2 = t * (-r * sn * tw) + b * (r * cs * tw);
        Jwi.c[0][i1] = d1.x; Jwi.c[1][i1] = d1.y; Jwi.c[2][i1] = d1.z;
        Jwi.c[0][i1 + 1] = d2.x; Jwi.c[1][i1 + 1] = d2.y; Jwi.c[2][i1 + 1] = d2.z;
        w = m.albedo;
        return m.albedo.x > 0.0f || m.albedo.y > 0.0f || m.albedo.z > 0.0f;
    }
    // modified Phong: r = d - 2 (d.ns) ns, basis around r, lobe angle from u1, azimuth from u2
    const float3 r = d - ns * (2.0f * dot(d, ns));
    const float cos_a = powf(1.0f - u1, m.phong_inv_n1);
    const float sin_a = sqrtf(fmaxf(1.0f - cos_a * cos_a, 0.0f));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    onb(r, t, b);
    wi = t * (sin_a * cs) + b * (sin_a * sn) + r * cos_a;
    const float cos_i = dot(wi, ns);
    if (cos_i <= 0.0f) return false;
    const float sign = copysignf(1.0f, r.z);
    const float a = -1.0f / (sign + r.z);  // the basis's a; its bb term is differentiated in the loop
    // d cos_a / d u1 and d sin_a / d u1
    const float dca = 1.0f - u1 > 0.0f ? -m.phong_inv_n1 * cos_a / (1.0f - u1) : 0.0f;
    const float dsa = sin_a > 0.0f ? -cos_a * dca / sin_a : 0.0f;
    const float tw = 2.0f * 3.14159265358979f;
    for (int k = 0; k < D; ++k) {
        const float ddx = Jd.c[0][k], ddy = Jd.c[1][k], ddz = Jd.c[2][k];
        const float dn = ns.x * ddx + ns.y * ddy + ns.z * ddz;
        const float drx = ddx - 2.0f * ns.x * dn, dry = ddy - 2.0f * ns.y * dn, drz = ddz - 2.0f * ns.z * dn;
        const float da = a * a * drz;
        const float dbb = r.y * a * drx + r.x * a * dry + r.x * r.y * da;
        const float dtx = sign * (2.0f * r.x * a * drx + r.x * r.x * da), dty = sign * dbb, dtz = -sign * drx;
        const float dbx = dbb, dby = 2.0f * r.y * a * dry + r.y * r.y * da, dbz = -dry;
        float gx = dtx * (sin_a * cs) + dbx * (sin_a * sn) + drx * cos_a;
        float gy = dty * (sin_a * cs) + dby * (sin_a * sn) + dry * cos_a;
        float gz = dtz * (sin_a * cs) + dbz * (sin_a * sn) + drz * cos_a;
        if (k == i1) {
            gx += t.x * (dsa * cs) + b.x * (dsa * sn) + r.x * dca;
            gy += t.y * (dsa * cs) + b.y * (dsa * sn) + r.y * dca;
            gz += t.z * (dsa * cs) + b.z * (dsa * sn) + r.z * dca;
        } else if (k == i1 + 1) {
            gx += sin_a * tw * (-t.x * sn + b.x * cs);
            gy += sin_a * tw * (-t.y * sn + b.y * cs);
            gz += sin_a * tw * (-t.z * sn + b.z * cs);
        }
        Jwi.c[0][k] = gx;
        Jwi.c[1][k] = gy;
        Jwi.c[2][k] = gz;
        const float dci = ns.x * gx + ns.y * gy + ns.z * gz;
        Jw.c[0][k] = m.albedo.x * m.phong_scale * dci;
        Jw.c[1][k] = m.albedo.y * m.phong_scale * dci;
        Jw.c[2][k] = m.albedo.z * m.phong_scale * dci;
    }
    w = m.albedo * (m.phong_scale * cos_i);
    return true;
}

// F(y) and dF/dy (dF->c[ch][k]) for one lane (no warp cooperation: the
// megakernel's lanes call it together, each with its own state).
template <bool kCount>
__device__ inline float3 eval_path_grad(const SceneView& s, unsigned mask, bool want, int depth, const float* y,
                                        uint32_t ys, Jac3& JF, unsigned& status, Work& work) {
    const int D = 2 + 2 * depth;
    Jac3 Jd, JT, Jtmp, Jw;
    for (int q = 0; q < 3; ++q)
        for (int k = 0; k < D; ++k) {
            JF.c[q][k] = 0.f;
            JT.c[q][k] = 0.f;
            Jd.c[q][k] = 0.f;
        }
    float3 F = f3(0.f, 0.f, 0.f), T = f3(1.f, 1.f, 1.f);
    float3 o = f3(0.f, 0.f, 1.f), d = f3(0.f, 0.f, 1.f);
    if (want) {
        const float3 cf = f3(s.cam[3], s.cam[4], s.cam[5]);
        const float3 cr = f3(s.cam[6], s.cam[7], s.cam[8]);
        const float3 cu = f3(s.cam[9], s.cam[10], s.cam[11]);
        o = f3(s.cam[0], s.cam[1], s.cam[2]);
        const float3 c = cf + cr * (2.0f * y[0] - 1.0f) + cu * (1.0f - 2.0f * y[ys]);
        const float il = 1.0f / sqrtf(dot(c, c));
        d = c * il;
        Jtmp.c[0][0] = 2.0f * cr.x; Jtmp.c[1][0] = 2.0f * cr.y; Jtmp.c[2][0] = 2.0f * cr.z;
        Jtmp.c[0][1] = -2.0f * cu.x; Jtmp.c[1][1] = -2.0f * cu.y; Jtmp.c[2][1] = -2.0f * cu.z;
        for (int q = 0; q < 3; ++q)
            for (int k = 2; k < D; ++k) Jtmp.c[q][k] = 0.f;
        jac_normalize(d, il, Jtmp, Jd, D);
    }
    bool alive = want;
    for (int v = 0; v <= depth; ++v) {
        if (!__any_sync(mask, alive)) break;
        float t;
        const int k = closest_hit<kCount>(s, mask, alive, o, d, t, status, work);
        if (!alive) continue;
        if (k < 0) {
            alive = false;
            continue;
        }
        const TriRecord* tr = s.tris + k;
        const float4 q1 = __ldg(&tr->e1_mat), q2 = __ldg(&tr->e2);
        const Material m = s.mats[__float_as_int(q1.w)];
        const float3 ng = normalize(cross(f3(q1.x, q1.y, q1.z), f3(q2.x, q2.y, q2.z)));
        const float3 p = o + d * t;
        if (m.emits && -dot(d, ng) > 0.0f) {
            F = F + mul(T, m.emission);
            for (int kk = 0; kk < D; ++kk) {
                JF.c[0][kk] += JT.c[0][kk] * m.emission.x;
                JF.c[1][kk] += JT.c[1][kk] * m.emission.y;
                JF.c[2][kk] += JT.c[2][kk] * m.emission.z;
            }
        }
        if (v == depth) {
            alive = false;
            continue;
        }
        float3 wi, w;
        const float u1 = y[(2 + 2 * v) * ys], u2 = y[(3 + 2 * v) * ys];
        if (!scatter_grad(m, d, ng, u1, u2, 2 + 2 * v, Jd, wi, w, Jtmp, Jw, D)) {
            alive = false;
            continue;
        }
        for (int kk = 0; kk < D; ++kk) {  // d(T w) = dT w + T dw
            JT.c[0][kk] = JT.c[0][kk] * w.x + T.x * Jw.c[0][kk];
            JT.c[1][kk] = JT.c[1][kk] * w.y + T.y * Jw.c[1][kk];
            JT.c[2][kk] = JT.c[2][kk] * w.z + T.z * Jw.c[2][kk];
        }
        T = mul(T, w);
        if (T.x == 0.0f && T.y == 0.0f && T.z == 0.0f) {
            alive = false;
            continue;
        }
        for (int q = 0; q < 3; ++q)
            for (int kk = 0; kk < D; ++kk) Jd.c[q][kk] = Jtmp.c[q][kk];
        const float3 off = dot(wi, ng) >= 0.0f ? ng : ng * -1.0f;
        const float mx = fmaxf(fmaxf(fabsf(p.x), fabsf(p.y)), fabsf(p.z));
        o = p + off * (1e-4f * (1.0f + mx));
        d = wi;
    }
    if (want) {
        if (!isfinite(F.x) || !isfinite(F.y) || !isfinite(F.z)) {
            status |= JR_STATUS_NONFINITE;
            F = f3(0.f, 0.f, 0.f);
        }
    }
    return F;
}

// The MALA drift m = clamp(sigma^2 / 2 grad log p, -2 sigma, 2 sigma) per
// coordinate from F and dF/dx (grad log p = grad lum(F) / lum(F); 0 where p = 0
// or the gradient is not finite).
__device__ inline float mala_drift(float3 F, const Jac3& JF, int k, float sigma) {
    const float p = lum(F);
    if (!(p > 0.0f)) return 0.0f;
    const float g = (0.2126f * JF.c[0][k] + 0.7152f * JF.c[1][k] + 0.0722f * JF.c[2][k]) / p;
    if (!isfinite(g)) return 0.0f;
    return fminf(fmaxf(0.5f * sigma * sigma * g, -2.0f * sigma), 2.0f * sigma);
}

__device__ __forceinline__ void flush_status(unsigned status, unsigned int* word) {
    if (status) atomicOr(word, status);
}

// Sum of a double over the 32 lanes of a warp (all lanes call; every lane gets the sum).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace
}  // namespace jr
