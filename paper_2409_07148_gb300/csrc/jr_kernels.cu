// Device code of the Jump Restore light-transport library (sm_103a).
//
// One thread owns one chain for a whole launch (persistent over n_steps).  The
// current state x and the candidate y live in dynamic shared memory, [buf][d]
// [thread] (bank-conflict free), so the accepted move is a buffer flip; F, p
// and u of the current state stay in registers.  Each step runs Alg. 2
// (Section 7.2) of Holl, Singh, Seidel, "Jump Restore Light Transport":
//   t1 ~ Exp(1), t2 ~ Exp(k(x)) with k = c~ u / p (Section 6.2),
//   splat (dt, x) into the framebuffer (Section 6.3 / 7.4 estimator),
//   t1 < t2: local MH move with the Gaussian small-step kernel (Alg. 1),
//   else   : regenerate x ~ mu (uniform) and count a tour.
// Both branches end in exactly one evaluation of the integrand, so the only
// divergence between them is the few instructions that build y.
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

// Closest hit, ties on equal t to the smaller original triangle index.
// Returns the leaf-order record index or -1; t_out gets the hit distance.
template <bool kCount>
__device__ __forceinline__ int closest_hit(const SceneView& s, float3 o, float3 d, float& t_out, unsigned& status,
                                           Work& work) {
    if constexpr (kCount) work.rays++;
    t_out = INFINITY;
    if (s.root == kSentinel) return -1;
    const float dx = fabsf(d.x) < 1e-20f ? copysignf(1e-20f, d.x) : d.x;
    const float dy = fabsf(d.y) < 1e-20f ? copysignf(1e-20f, d.y) : d.y;
    const float dz = fabsf(d.z) < 1e-20f ? copysignf(1e-20f, d.z) : d.z;
    const float ix = 1.0f / dx, iy = 1.0f / dy, iz = 1.0f / dz;
    const float ox = o.x * ix, oy = o.y * iy, oz = o.z * iz;
    float tb = INFINITY;
    int best = -1, best_id = INT32_MAX;
    int stack[kStackSize];
    int sp = 0;
    int ref = s.root;
    uint32_t visits = 0;
    while (true) {
        while (ref >= 0) {
            if (++visits > kNodeVisitBudget) {
                status |= JR_STATUS_TRAVERSAL;
                return -1;
            }
            if constexpr (kCount) work.nodes++;
            const BvhNode* n = s.nodes + ref;
            const float4 a = __ldg(&n->a), b = __ldg(&n->b), c = __ldg(&n->c);
            const int4 rf = __ldg(&n->refs);
            const float l0x = fmaf(a.x, ix, -ox), h0x = fmaf(a.y, ix, -ox);
            const float l0y = fmaf(a.z, iy, -oy), h0y = fmaf(a.w, iy, -oy);
            const float l0z = fmaf(c.x, iz, -oz), h0z = fmaf(c.y, iz, -oz);
            const float l1x = fmaf(b.x, ix, -ox), h1x = fmaf(b.y, ix, -ox);
            const float l1y = fmaf(b.z, iy, -oy), h1y = fmaf(b.w, iy, -oy);
            const float l1z = fmaf(c.z, iz, -oz), h1z = fmaf(c.w, iz, -oz);
            const float tn0 = fmaxf(fmaxf(fminf(l0x, h0x), fminf(l0y, h0y)), fmaxf(fminf(l0z, h0z), 0.0f));
            const float tf0 = fminf(fminf(fmaxf(l0x, h0x), fmaxf(l0y, h0y)), fminf(fmaxf(l0z, h0z), tb));
            const float tn1 = fmaxf(fmaxf(fminf(l1x, h1x), fminf(l1y, h1y)), fmaxf(fminf(l1z, h1z), 0.0f));
            const float tf1 = fminf(fminf(fmaxf(l1x, h1x), fmaxf(l1y, h1y)), fminf(fmaxf(l1z, h1z), tb));
            const bool h0 = tn0 <= tf0 * 1.00000024f;
            const bool h1 = tn1 <= tf1 * 1.00000024f;
            if (h0 && h1) {
                const bool first0 = tn0 <= tn1;
                if (sp >= kStackSize) {
                    status |= JR_STATUS_STACK;
                    return -1;
                }
                stack[sp++] = first0 ? rf.y : rf.x;
                ref = first0 ? rf.x : rf.y;
            } else if (h0) {
                ref = rf.x;
            } else if (h1) {
                ref = rf.y;
            } else {
                ref = sp > 0 ? stack[--sp] : kSentinel;
            }
        }
        if (ref == kSentinel) break;
        const int enc = ~ref;
        const int first = enc >> 3, cnt = (enc & 7) + 1;
        if constexpr (kCount) work.tris += (uint32_t)cnt;
        for (int k = first; k < first + cnt; ++k) {
            const TriRecord* tr = s.tris + k;
            const float4 q0 = __ldg(&tr->v0_id), q1 = __ldg(&tr->e1_mat), q2 = __ldg(&tr->e2);
            // Moller-Trumbore (JGT 1997), same algebra as the reference definition.
            const float3 e1 = f3(q1.x, q1.y, q1.z), e2 = f3(q2.x, q2.y, q2.z);
            const float3 pv = cross(d, e2);
            const float det = dot(e1, pv);
            if (det == 0.0f) continue;
            const float inv = 1.0f / det;
            const float3 tv = o - f3(q0.x, q0.y, q0.z);
            const float u = dot(tv, pv) * inv;
            if (u < 0.0f || u > 1.0f) continue;
            const float3 qv = cross(tv, e1);
            const float v = dot(d, qv) * inv;
            if (v < 0.0f || u + v > 1.0f) continue;
            const float t = dot(e2, qv) * inv;
            const int id = __float_as_int(q0.w);
            if (t > 0.0f && (t < tb || (t == tb && id < best_id))) {
                tb = t;
                best = k;
                best_id = id;
            }
        }
        ref = sp > 0 ? stack[--sp] : kSentinel;
    }
    t_out = tb;
    return best;
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
template <bool kCount>
__device__ __forceinline__ float3 eval_path_w(const SceneView& s, int depth, const float* y, uint32_t ys,
                                              int32_t* ids, uint64_t id_stride, unsigned& status, Work& work) {
    float3 F = f3(0.f, 0.f, 0.f), T = f3(1.f, 1.f, 1.f);
    const float3 co = f3(s.cam[0], s.cam[1], s.cam[2]);
    const float3 cf = f3(s.cam[3], s.cam[4], s.cam[5]);
    const float3 cr = f3(s.cam[6], s.cam[7], s.cam[8]);
    const float3 cu = f3(s.cam[9], s.cam[10], s.cam[11]);
    float3 o = co;
    float3 d = normalize(cf + cr * (2.0f * y[0] - 1.0f) + cu * (1.0f - 2.0f * y[ys]));
    if (ids)
        for (int v = 0; v <= depth; ++v) ids[v * id_stride] = -1;
    for (int v = 0; v <= depth; ++v) {
        float t;
        const int k = closest_hit<kCount>(s, o, d, t, status, work);
        if (k < 0) break;
        const TriRecord* tr = s.tris + k;
        const float4 q1 = __ldg(&tr->e1_mat), q2 = __ldg(&tr->e2);
        if (ids) ids[v * id_stride] = __float_as_int(__ldg(&tr->v0_id.w));
        const Material m = s.mats[__float_as_int(q1.w)];
        const float3 ng = normalize(cross(f3(q1.x, q1.y, q1.z), f3(q2.x, q2.y, q2.z)));
        const float3 p = o + d * t;
        if (m.emits && -dot(d, ng) > 0.0f) F = F + mul(T, m.emission);
        if (v == depth) break;
        float3 wi, w;
        if (!scatter(m, d, ng, y[(2 + 2 * v) * ys], y[(3 + 2 * v) * ys], wi, w)) break;
        T = mul(T, w);
        if (T.x == 0.0f && T.y == 0.0f && T.z == 0.0f) break;
        const float3 off = dot(wi, ng) >= 0.0f ? ng : ng * -1.0f;
        const float mx = fmaxf(fmaxf(fabsf(p.x), fabsf(p.y)), fabsf(p.z));
        o = p + off * (1e-4f * (1.0f + mx));
        d = wi;
    }
    if (!isfinite(F.x) || !isfinite(F.y) || !isfinite(F.z)) {
        status |= JR_STATUS_NONFINITE;
        F = f3(0.f, 0.f, 0.f);
    }
    return F;
}

__device__ __forceinline__ float3 eval_path(const SceneView& s, int depth, const float* y, uint32_t ys, int32_t* ids,
                                            uint64_t id_stride, unsigned& status) {
    Work w;
    return eval_path_w<false>(s, depth, y, ys, ids, id_stride, status, w);
}

__device__ __forceinline__ void flush_status(unsigned status, unsigned int* word) {
    if (status) atomicOr(word, status);
}

// ------------------------------------------------------------------ kernels
// x0 ~ mu (tag 1); y built in shared memory, then written to the SoA state.
__global__ void init_kernel(SceneView s, ChainView c) {
    extern __shared__ float sh[];
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const uint64_t i = blockIdx.x * (uint64_t)B + tid;
    if (i >= c.n) return;
    const int D = (int)c.dim;
    float* y = sh + tid;
    const uint32_t chain = c.chain_offset + (uint32_t)i;
    for (int b = 0; 4 * b < D; ++b) {
        const uint4 r = draw(c.seed, kTagInit, (uint32_t)(b + 1), chain, 0);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * b + q < D) y[(4 * b + q) * B] = u01(rr[q]);
    }
    unsigned status = 0;
    const float3 F = eval_path(s, (int)c.depth, y, B, nullptr, 0, status);
    for (int d = 0; d < D; ++d) c.x[d * c.n + i] = y[d * B];
    c.fpu[0 * c.n + i] = F.x;
    c.fpu[1 * c.n + i] = F.y;
    c.fpu[2 * c.n + i] = F.z;
    c.fpu[3 * c.n + i] = lum(F);
    c.fpu[4 * c.n + i] = 1.0f;  // u of uniform mu
    flush_status(status, c.status);
}

// Re-evaluate F, p, u of the stored states (after jr_set_state).
__global__ void reeval_kernel(SceneView s, ChainView c) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    unsigned status = 0;
    const float3 F = eval_path(s, (int)c.depth, c.x + i, (uint32_t)c.n, nullptr, 0, status);
    c.fpu[0 * c.n + i] = F.x;
    c.fpu[1 * c.n + i] = F.y;
    c.fpu[2 * c.n + i] = F.z;
    c.fpu[3 * c.n + i] = lum(F);
    c.fpu[4 * c.n + i] = 1.0f;
    flush_status(status, c.status);
}

template <bool kTrace, bool kCount>
__global__ void __launch_bounds__(256) step_kernel(SceneView s, ChainView c, uint64_t step_begin, uint32_t n_steps,
                                                   uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix,
                                                   unsigned long long* work_out) {
    extern __shared__ float sh[];
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const uint64_t i = blockIdx.x * (uint64_t)B + tid;
    const bool active = i < c.n;
    const int D = (int)c.dim;
    float* buf0 = sh + tid;
    float* buf1 = sh + (size_t)D * B + tid;
    uint32_t nJ = 0, nL = 0, nA = 0;
    unsigned status = 0;
    Work work;
    if (active) {
        for (int d = 0; d < D; ++d) buf0[d * B] = c.x[d * c.n + i];
        float Fr = c.fpu[0 * c.n + i], Fg = c.fpu[1 * c.n + i], Fb = c.fpu[2 * c.n + i];
        float p = c.fpu[3 * c.n + i], u = c.fpu[4 * c.n + i];
        float* cur = buf0;
        float* cand = buf1;
        const uint32_t chain = c.chain_offset + (uint32_t)i;
        const float c_tilde = c.c_tilde, sigma = c.sigma;
        const float WH = (float)c.width * (float)c.height;
        const bool rb = (c.flags & JR_FLAG_RAO_BLACKWELL) != 0;
        for (uint32_t st = 0; st < n_steps; ++st) {
            const uint64_t step = step_begin + st;
            const uint4 r0 = draw(c.seed, kTagStep, 0, chain, step);
            // Alg. 2: holding time t1 ~ Exp(1); killing time t2 ~ Exp(k), k = c~ u / p.
            const float E1 = -logf(1.0f - u01(r0.x));
            const float E2 = -logf(1.0f - u01(r0.y));
            const float Ua = u01(r0.z);
            const float t2 = p > 0.0f ? E2 * p / (c_tilde * u) : 0.0f;
            const bool local = E1 < t2;  // a tie goes to the killing branch
            float dt = local ? E1 : t2;
            if (rb) dt = p > 0.0f ? p / (p + c_tilde * u) : 0.0f;
            int32_t pix = -1;
            if (dt > 0.0f && p > 0.0f) {
                // left-rectangle estimator: x_{i-1} weighted by dt_i (Section 7.4)
                uint32_t px = (uint32_t)((double)cur[0] * (double)c.width);
                uint32_t py = (uint32_t)((double)cur[B] * (double)c.height);
                px = min(px, c.width - 1);
                py = min(py, c.height - 1);
                pix = (int32_t)(py * c.width + px);
                const float wgt = c_tilde * dt * WH / p;
                atomicAdd(c.fb + pix, make_float4(wgt * Fr, wgt * Fg, wgt * Fb, dt));
            }
            // candidate y: Gaussian small step (local) or a fresh draw from mu
            for (int b = 0; 4 * b < D; ++b) {
                const uint4 r = draw(c.seed, kTagStep, (uint32_t)(b + 1), chain, step);
                const int d0 = 4 * b;
                if (local) {
                    float sn, cs;
                    float R = sqrtf(-2.0f * logf(1.0f - u01(r.x)));
                    sincospif(2.0f * u01(r.y), &sn, &cs);
                    cand[d0 * B] = wrap01(cur[d0 * B] + sigma * R * cs);
                    cand[(d0 + 1) * B] = wrap01(cur[(d0 + 1) * B] + sigma * R * sn);
                    if (d0 + 2 < D) {
                        R = sqrtf(-2.0f * logf(1.0f - u01(r.z)));
                        sincospif(2.0f * u01(r.w), &sn, &cs);
                        cand[(d0 + 2) * B] = wrap01(cur[(d0 + 2) * B] + sigma * R * cs);
                        cand[(d0 + 3) * B] = wrap01(cur[(d0 + 3) * B] + sigma * R * sn);
                    }
                } else {
                    cand[d0 * B] = u01(r.x);
                    cand[(d0 + 1) * B] = u01(r.y);
                    if (d0 + 2 < D) {
                        cand[(d0 + 2) * B] = u01(r.z);
                        cand[(d0 + 3) * B] = u01(r.w);
                    }
                }
            }
            const float3 Fy = eval_path_w<kCount>(s, (int)c.depth, cand, B, nullptr, 0, status, work);
            const float py_ = lum(Fy);
            bool accept;
            if (local) {
                accept = Ua * p < py_;  // U < min(1, p(y)/p(x)), p(x) > 0 on this branch
                nL++;
                nA += accept;
            } else {
                accept = true;
                nJ++;
            }
            if (accept) {
                float* tmp = cur;
                cur = cand;
                cand = tmp;
                Fr = Fy.x;
                Fg = Fy.y;
                Fb = Fy.z;
                p = py_;
                u = 1.0f;
            }
            if (kTrace) {
                const uint64_t o = i * n_steps + st;
                if (tr_flags) tr_flags[o] = (uint8_t)((local ? 0 : 1) | (local && accept ? 2 : 0));
                if (tr_dt) tr_dt[o] = pix >= 0 ? dt : 0.0f;
                if (tr_pix) tr_pix[o] = pix;
            }
        }
        for (int d = 0; d < D; ++d) c.x[d * c.n + i] = cur[d * B];
        c.fpu[0 * c.n + i] = Fr;
        c.fpu[1 * c.n + i] = Fg;
        c.fpu[2 * c.n + i] = Fb;
        c.fpu[3 * c.n + i] = p;
        c.fpu[4 * c.n + i] = u;
    }
    // warp-aggregated counters: one 64-bit atomic per warp and counter
    nJ = __reduce_add_sync(0xffffffffu, nJ);
    nL = __reduce_add_sync(0xffffffffu, nL);
    nA = __reduce_add_sync(0xffffffffu, nA);
    status = __reduce_or_sync(0xffffffffu, status);
    if constexpr (kCount) {
        const uint32_t r = __reduce_add_sync(0xffffffffu, work.rays);
        const uint32_t nd = __reduce_add_sync(0xffffffffu, work.nodes);
        const uint32_t tr = __reduce_add_sync(0xffffffffu, work.tris);
        if ((tid & 31) == 0) {
            atomicAdd(work_out + 0, (unsigned long long)r);
            atomicAdd(work_out + 1, (unsigned long long)nd);
            atomicAdd(work_out + 2, (unsigned long long)tr);
        }
    }
    if ((tid & 31) == 0) {
        if (nJ) atomicAdd(c.counters + 0, (unsigned long long)nJ);
        if (nL) atomicAdd(c.counters + 1, (unsigned long long)nL);
        if (nA) atomicAdd(c.counters + 2, (unsigned long long)nA);
        flush_status(status, c.status);
    }
}

// FP32 framebuffer -> FP64 accumulator, then clear (keeps long runs exact to
// FP64 while the hot loop does single 16-byte vector atomics).
__global__ void fold_kernel(float4* fb, double4_32a* acc, uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float4 v = fb[j];
    if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
        double4_32a a = acc[j];
        a.x += v.x;
        a.y += v.y;
        a.z += v.z;
        a.w += v.w;
        acc[j] = a;
        fb[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// image = accumulator / J (Section 6.3, normalisation-free estimator).
__global__ void resolve_kernel(const double4_32a* acc, const unsigned long long* counters, float* rgb, uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const unsigned long long J = counters[0];
    const double4_32a a = acc[j];
    const double inv = J > 0 ? 1.0 / (double)J : 0.0;
    rgb[3 * j] = (float)(a.x * inv);
    rgb[3 * j + 1] = (float)(a.y * inv);
    rgb[3 * j + 2] = (float)(a.z * inv);
}

__global__ void eval_states_kernel(SceneView s, uint32_t depth, float c_tilde, const float* x, uint64_t n, float* F,
                                   float* p, float* u, float* k, int32_t* ids, unsigned int* status_word) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned status = 0;
    const float3 f = eval_path(s, (int)depth, x + i, (uint32_t)n, ids ? ids + i : nullptr, n, status);
    const float pp = lum(f);
    const float uu = 1.0f;
    if (F) {
        F[i] = f.x;
        F[n + i] = f.y;
        F[2 * n + i] = f.z;
    }
    if (p) p[i] = pp;
    if (u) u[i] = uu;
    if (k) k[i] = pp > 0.0f ? c_tilde * uu / pp : INFINITY;  // Section 6.2
    if (status && status_word) atomicOr(status_word, status);
}

__global__ void render_pt_kernel(SceneView s, uint32_t W, uint32_t H, uint32_t depth, uint64_t seed,
                                 uint64_t sample_begin, uint64_t n, double* accum) {
    extern __shared__ float sh[];
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const uint64_t i = blockIdx.x * (uint64_t)B + tid;
    if (i >= n) return;
    const int D = 2 + 2 * (int)depth;
    float* y = sh + tid;
    const uint64_t smp = sample_begin + i;
    for (int b = 0; 4 * b < D; ++b) {
        const uint4 r = draw(seed, kTagPt, (uint32_t)(b + 1), (uint32_t)smp, smp >> 32);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * b + q < D) y[(4 * b + q) * B] = u01(rr[q]);
    }
    unsigned status = 0;
    const float3 F = eval_path(s, (int)depth, y, B, nullptr, 0, status);
    uint32_t px = min((uint32_t)((double)y[0] * (double)W), W - 1);
    uint32_t py = min((uint32_t)((double)y[B] * (double)H), H - 1);
    const double WH = (double)W * (double)H;
    double* a = accum + 4 * ((size_t)py * W + px);
    if (F.x != 0.f) atomicAdd(a, WH * F.x);
    if (F.y != 0.f) atomicAdd(a + 1, WH * F.y);
    if (F.z != 0.f) atomicAdd(a + 2, WH * F.z);
    // channel 3 is left to the caller: the sample count is n, known on the host
}

__global__ void philox_kernel(uint64_t seed, uint32_t tag, uint32_t block, uint64_t chain_begin, uint64_t step,
                              uint64_t n, uint32_t* out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = draw(seed, tag, block, (uint32_t)(chain_begin + i), step);
    reinterpret_cast<uint4*>(out)[i] = r;
}

inline unsigned grid_for(uint64_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_init(const SceneView& s, const ChainView& c, cudaStream_t st) {
    const unsigned B = 128;
    init_kernel<<<grid_for(c.n, B), B, sizeof(float) * c.dim * B, st>>>(s, c);
    return cudaGetLastError();
}

cudaError_t launch_reeval(const SceneView& s, const ChainView& c, cudaStream_t st) {
    const unsigned B = 128;
    reeval_kernel<<<grid_for(c.n, B), B, 0, st>>>(s, c);
    return cudaGetLastError();
}

cudaError_t launch_step(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                        uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix, unsigned long long* work_out, int block,
                        cudaStream_t st) {
    const unsigned B = (unsigned)block;
    const size_t shm = sizeof(float) * 2 * c.dim * B;  // <= 2 * 32 * 256 * 4 = 64 KB
    const unsigned G = grid_for(c.n, B);
    static bool attr_set = false;  // opt in to > 48 KB of dynamic shared memory once
    if (!attr_set) {
        const int lim = (int)(sizeof(float) * 2 * kMaxDim * 256);
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(step_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(step_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(step_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
                cudaSuccess)
            return e;
        attr_set = true;
    }
    if (work_out)
        step_kernel<false, true><<<G, B, shm, st>>>(s, c, step_begin, n_steps, nullptr, nullptr, nullptr, work_out);
    else if (tr_flags || tr_dt || tr_pix)
        step_kernel<true, false><<<G, B, shm, st>>>(s, c, step_begin, n_steps, tr_flags, tr_dt, tr_pix, nullptr);
    else
        step_kernel<false, false><<<G, B, shm, st>>>(s, c, step_begin, n_steps, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_fold(const ChainView& c, cudaStream_t st) {
    const uint32_t n = c.width * c.height;
    fold_kernel<<<grid_for(n, 256), 256, 0, st>>>(c.fb, c.acc64, n);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const ChainView& c, float* rgb, cudaStream_t st) {
    const uint32_t n = c.width * c.height;
    resolve_kernel<<<grid_for(n, 256), 256, 0, st>>>(c.acc64, c.counters, rgb, n);
    return cudaGetLastError();
}

cudaError_t launch_eval_states(const SceneView& s, uint32_t depth, float c_tilde, const float* x, uint64_t n,
                               float* F, float* p, float* u, float* k, int32_t* ids, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    eval_states_kernel<<<grid_for(n, 128), 128, 0, st>>>(s, depth, c_tilde, x, n, F, p, u, k, ids, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_render_pt(const SceneView& s, uint32_t width, uint32_t height, uint32_t depth, uint64_t seed,
                             uint64_t sample_begin, uint64_t n, double* accum, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned B = 128;
    const size_t shm = sizeof(float) * (2 + 2 * depth) * B;
    render_pt_kernel<<<grid_for(n, B), B, shm, st>>>(s, width, height, depth, seed, sample_begin, n, accum);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t seed, uint32_t tag, uint32_t block, uint64_t chain_begin, uint64_t step,
                          uint64_t n, uint32_t* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    philox_kernel<<<grid_for(n, 256), 256, 0, st>>>(seed, tag, block, chain_begin, step, n, out);
    return cudaGetLastError();
}

}  // namespace jr
