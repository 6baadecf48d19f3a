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

#include <algorithm>

#include "../../include/jr.h"
#include "jr_device.cuh"
#include "jr_internal.h"

namespace jr {
namespace {

// ------------------------------------------------------------------ kernels
// x0 ~ mu (tag 1); y built in shared memory, then written to the SoA state.
__global__ void init_kernel(SceneView s, ChainView c) {
    extern __shared__ float sh[];
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const uint64_t i = blockIdx.x * (uint64_t)B + tid;
    const unsigned mask = __ballot_sync(0xffffffffu, i < c.n);  // lanes that trace together
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
    const float3 F = eval_path(s, mask, true, (int)c.depth, y, B, nullptr, 0, status);
    float2* x2 = reinterpret_cast<float2*>(c.x);
    for (int k = 0; 2 * k < D; ++k) x2[(uint64_t)k * c.n + i] = make_float2(y[2 * k * B], y[(2 * k + 1) * B]);
    c.fpu[0 * c.n + i] = F.x;
    c.fpu[1 * c.n + i] = F.y;
    c.fpu[2 * c.n + i] = F.z;
    c.fpu[3 * c.n + i] = lum(F);
    c.fpu[4 * c.n + i] = 1.0f;  // u of uniform mu
    flush_status(status, c.status);
}

// Load chain i's coordinates (pair layout) into shared memory y[d * B].
__device__ __forceinline__ void load_coords(const ChainView& c, uint64_t i, float* y, uint32_t B) {
    const float2* x2 = reinterpret_cast<const float2*>(c.x);
    for (int k = 0; 2 * k < (int)c.dim; ++k) {
        const float2 v = x2[(uint64_t)k * c.n + i];
        y[2 * k * B] = v.x;
        y[(2 * k + 1) * B] = v.y;
    }
}

// Re-evaluate F, p, u of the stored states (after jr_set_state).
__global__ void reeval_kernel(SceneView s, ChainView c) {
    extern __shared__ float sh[];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const unsigned mask = __ballot_sync(0xffffffffu, i < c.n);
    if (i >= c.n) return;
    unsigned status = 0;
    load_coords(c, i, sh + threadIdx.x, blockDim.x);
    const float3 F = eval_path(s, mask, true, (int)c.depth, sh + threadIdx.x, blockDim.x, nullptr, 0, status);
    c.fpu[0 * c.n + i] = F.x;
    c.fpu[1 * c.n + i] = F.y;
    c.fpu[2 * c.n + i] = F.z;
    c.fpu[3 * c.n + i] = lum(F);
    c.fpu[4 * c.n + i] = 1.0f;
    flush_status(status, c.status);
}

// n_steps of Alg. 2 for chain i of set c (thread tid of the block; `active`
// false for threads without a chain).  Every thread of the block calls it;
// sh holds [2][D][blockDim] floats.
template <bool kTrace, bool kCount>
__device__ __forceinline__ void chain_steps(const SceneView& s, const ChainView& c, uint64_t i, bool active, float* sh,
                                            uint64_t step_begin, uint32_t n_steps, uint8_t* tr_flags, float* tr_dt,
                                            int32_t* tr_pix, unsigned long long* work_out) {
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const unsigned mask = __ballot_sync(0xffffffffu, active);  // lanes that trace together
    const int D = (int)c.dim;
    float* buf0 = sh + tid;
    float* buf1 = sh + (size_t)D * B + tid;
    uint32_t nJ = 0, nL = 0, nA = 0;
    unsigned status = 0;
    Work work;
    const bool mh = (c.flags & JR_FLAG_MH) != 0;
    double psum = 0.0;  // MH: sum of p over this chain's large-step proposals
    if (active) {
        load_coords(c, i, buf0, B);
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
            const float Ua = u01(r0.z);
            bool local;
            float dt;
            if (mh) {
                // the MH baseline: a large step (from mu) with probability l, else
                // a small step; the state before the iteration enters the
                // estimator once the burn-in is over (dt = 1 counts it)
                local = !(u01(r0.x) < c.large_step);
                dt = step >= c.burn_in ? 1.0f : 0.0f;
            } else {
                // Alg. 2: holding time t1 ~ Exp(1); killing time t2 ~ Exp(k), k = c~ u / p.
                const float E1 = -logf(1.0f - u01(r0.x));
                const float E2 = -logf(1.0f - u01(r0.y));
                const float t2 = p > 0.0f ? E2 * p / (c_tilde * u) : 0.0f;
                local = E1 < t2;  // a tie goes to the killing branch
                dt = local ? E1 : t2;
                if (rb) dt = p > 0.0f ? p / (p + c_tilde * u) : 0.0f;
            }
            int32_t pix = -1;
            if (dt > 0.0f && p > 0.0f) {
                // left-rectangle estimator: x_{i-1} weighted by dt_i (Section 7.4);
                // MH: the ergodic average's term W H F / p of the held state
                uint32_t px = (uint32_t)((double)cur[0] * (double)c.width);
                uint32_t py = (uint32_t)((double)cur[B] * (double)c.height);
                px = min(px, c.width - 1);
                py = min(py, c.height - 1);
                pix = (int32_t)(py * c.width + px);
                const float wgt = mh ? WH / p : c_tilde * dt * WH / p;
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
            const float3 Fy = eval_path_w<kCount>(s, mask, true, (int)c.depth, cand, B, nullptr, 0, status, work);
            const float py_ = lum(Fy);
            bool accept;
            if (mh) {  // Alg. 1: U < min(1, p(y)/p(x)), 1 if p(x) = 0
                accept = !(p > 0.0f) || Ua * p < py_;
                if (local) {
                    nL++;
                } else {
                    nJ++;
                    psum += (double)py_;
                }
                nA += accept;
            } else if (local) {
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
                if (tr_flags) tr_flags[o] = (uint8_t)((local ? 0 : 1) | ((mh || local) && accept ? 2 : 0));
                if (tr_dt) tr_dt[o] = pix >= 0 ? dt : 0.0f;
                if (tr_pix) tr_pix[o] = pix;
            }
        }
        float2* x2 = reinterpret_cast<float2*>(c.x);
        for (int k = 0; 2 * k < D; ++k) x2[(uint64_t)k * c.n + i] = make_float2(cur[2 * k * B], cur[(2 * k + 1) * B]);
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
    if (mh) psum = warp_sum(psum);
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
        if (psum != 0.0) atomicAdd(reinterpret_cast<double*>(c.counters + kCounterPSum), psum);
        flush_status(status, c.status);
    }
}

// Both persistent kernels are capped at 64 registers (4 blocks of 256 threads
// per SM): the 4-wide traversal would take 108, and the occupancy the cap buys
// outweighs its small spill (measured: 5.0 -> 5.9e8 chain steps/s for the
// megakernel, 5.9 -> 6.1e8 for the 64-scene batch).
template <bool kTrace, bool kCount>
__global__ void __launch_bounds__(256, 4) step_kernel(SceneView s, ChainView c, uint64_t step_begin, uint32_t n_steps,
                                                   uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix,
                                                   unsigned long long* work_out) {
    extern __shared__ float sh[];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    chain_steps<kTrace, kCount>(s, c, i, i < c.n, sh, step_begin, n_steps, tr_flags, tr_dt, tr_pix, work_out);
}

// ------------------------------------------------------------------ one chain per warp
// For scenes of at most kWarpChainMaxTris triangles with few chains (the
// megakernel's case), one warp carries one chain: lane d holds coordinate d,
// draws its own Philox block and Box-Muller pair, and a ray tests every
// triangle, triangle k in lane k mod 32, before a butterfly reduction picks the
// closest hit.  A step's latency then shrinks to a few triangle tests and one
// shading per vertex, and a few hundred chains spread over as many SMs as
// their warps fill.  The per-chain arithmetic is chain_steps': the same draws,
// the same Box-Muller expressions and acceptance, the same camera_ray and
// shade_vertex; the closest hit is the least (t, original index) over all
// triangles with t > 0, which is what the BVH traversal returns too.

// Closest hit of the ray (o, d) over all n triangle records, for the whole
// warp (every lane calls with the same ray).  Returns the record index or -1.
__device__ __forceinline__ int closest_hit_warp(const SceneView& s, float3 o, float3 d, float& t_out) {
    const int lane = threadIdx.x & 31;
    float tb = INFINITY;
    int best = -1, bid = INT32_MAX;
    for (uint32_t k = lane; k < s.n_tris; k += 32) {
        const TriRecord* tr = s.tris + k;
        const float4 q0 = __ldg(&tr->v0_id), q1 = __ldg(&tr->e1_mat), q2 = __ldg(&tr->e2);
        const float3 e1 = f3(q1.x, q1.y, q1.z), e2 = f3(q2.x, q2.y, q2.z);
        const float3 pv = cross(d, e2);
        const float det = dot(e1, pv);
        const float inv = 1.0f / det;
        const float3 tv = o - f3(q0.x, q0.y, q0.z);
        const float u = dot(tv, pv) * inv;
        const float3 qv = cross(tv, e1);
        const float v = dot(d, qv) * inv;
        const float t = dot(e2, qv) * inv;
        const int id = __float_as_int(q0.w);
        const bool hit = det != 0.0f && !(u < 0.0f || u > 1.0f) && !(v < 0.0f || u + v > 1.0f) && t > 0.0f &&
                         (t < tb || (t == tb && id < bid));
        tb = hit ? t : tb;
        best = hit ? (int)k : best;
        bid = hit ? id : bid;
    }
    // The warp's closest hit, ties to the smaller original index.  Every tb is
    // a hit distance t > 0 or +inf, and for such floats the bit patterns order
    // as the values do, so two warp-wide integer minima find it: the nearest
    // distance, then the smallest index among the lanes at that distance (the
    // indices are distinct); the lane holding it hands over its record.
    const unsigned tbits = __float_as_uint(tb);
    const unsigned tmin = __reduce_min_sync(0xffffffffu, tbits);
    if (tmin == __float_as_uint(INFINITY)) {  // no lane has a hit
        t_out = INFINITY;
        return -1;
    }
    const unsigned imin = __reduce_min_sync(0xffffffffu, tbits == tmin ? (unsigned)bid : 0xffffffffu);
    const int src = __ffs(__ballot_sync(0xffffffffu, tbits == tmin && (unsigned)bid == imin)) - 1;
    best = __shfl_sync(0xffffffffu, best, src);
    t_out = __uint_as_float(tmin);
    return best;
}

// The integrand F(y) for the warp's chain, y[d] in lane d (eval_path_w's steps).
__device__ __forceinline__ float3 eval_path_warp(const SceneView& s, int depth, float yd, unsigned& status) {
    float3 F = f3(0.f, 0.f, 0.f), T = f3(1.f, 1.f, 1.f);
    float3 o, d;
    camera_ray(s, __shfl_sync(0xffffffffu, yd, 0), __shfl_sync(0xffffffffu, yd, 1), o, d);
    for (int v = 0; v <= depth; ++v) {
        float t;
        const int k = closest_hit_warp(s, o, d, t);
        if (k < 0) break;
        const float u1 = __shfl_sync(0xffffffffu, yd, (2 + 2 * v) & 31);
        const float u2 = __shfl_sync(0xffffffffu, yd, (3 + 2 * v) & 31);
        if (!shade_vertex(s, k, t, v, depth, v < depth ? u1 : 0.0f, v < depth ? u2 : 0.0f, o, d, T, F)) break;
    }
    return finite_or_zero(F, status);
}

constexpr int kWarpChainThreads = 128;  // four chains per block

__global__ void __launch_bounds__(kWarpChainThreads) step_kernel_warp(SceneView s, ChainView c, uint64_t step_begin,
                                                                      uint32_t n_steps) {
    const uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= c.n) return;  // a whole warp
    const int lane = threadIdx.x & 31;
    const int D = (int)c.dim;
    const bool mine = lane < D;  // this lane holds coordinate `lane`
    const uint32_t chain = c.chain_offset + (uint32_t)i;
    const bool mh = (c.flags & JR_FLAG_MH) != 0, rb = (c.flags & JR_FLAG_RAO_BLACKWELL) != 0;
    const float c_tilde = c.c_tilde, sigma = c.sigma;
    const float WH = (float)c.width * (float)c.height;
    uint32_t nJ = 0, nL = 0, nA = 0;
    unsigned status = 0;
    double psum = 0.0;
    float xd = mine ? c.x[xidx((uint32_t)lane, i, c.n)] : 0.0f;
    float Fr = c.fpu[0 * c.n + i], Fg = c.fpu[1 * c.n + i], Fb = c.fpu[2 * c.n + i];
    float p = c.fpu[3 * c.n + i], u = c.fpu[4 * c.n + i];
    for (uint32_t st = 0; st < n_steps; ++st) {
        const uint64_t step = step_begin + st;
        const uint4 r0 = draw(c.seed, kTagStep, 0, chain, step);
        const float Ua = u01(r0.z);
        bool local;
        float dt;
        if (mh) {
            local = !(u01(r0.x) < c.large_step);
            dt = step >= c.burn_in ? 1.0f : 0.0f;
        } else {
            const float E1 = -logf(1.0f - u01(r0.x));
            const float E2 = -logf(1.0f - u01(r0.y));
            const float t2 = p > 0.0f ? E2 * p / (c_tilde * u) : 0.0f;
            local = E1 < t2;  // a tie goes to the killing branch
            dt = local ? E1 : t2;
            if (rb) dt = p > 0.0f ? p / (p + c_tilde * u) : 0.0f;
        }
        const float x0 = __shfl_sync(0xffffffffu, xd, 0), x1 = __shfl_sync(0xffffffffu, xd, 1);
        if (lane == 0 && dt > 0.0f && p > 0.0f) {
            uint32_t px = (uint32_t)((double)x0 * (double)c.width);
            uint32_t py = (uint32_t)((double)x1 * (double)c.height);
            px = min(px, c.width - 1);
            py = min(py, c.height - 1);
            const float wgt = mh ? WH / p : c_tilde * dt * WH / p;
            atomicAdd(c.fb + (py * c.width + px), make_float4(wgt * Fr, wgt * Fg, wgt * Fb, dt));
        }
        // candidate coordinate `lane`: Philox block lane / 4 + 1; a local move's
        // Box-Muller pair is (r.x, r.y) for the block's first two coordinates
        // and (r.z, r.w) for the last two
        float yd = 0.0f;
        if (mine) {
            const uint4 r = draw(c.seed, kTagStep, (uint32_t)(lane >> 2) + 1u, chain, step);
            const bool second = (lane & 2) != 0;
            if (local) {
                float sn, cs;
                const float R = sqrtf(-2.0f * logf(1.0f - u01(second ? r.z : r.x)));
                sincospif(2.0f * u01(second ? r.w : r.y), &sn, &cs);
                yd = wrap01(xd + sigma * R * ((lane & 1) ? sn : cs));
            } else {
                yd = u01(second ? ((lane & 1) ? r.w : r.z) : ((lane & 1) ? r.y : r.x));
            }
        }
        const float3 Fy = eval_path_warp(s, (int)c.depth, yd, status);
        const float py_ = lum(Fy);
        bool accept;
        if (mh) {
            accept = !(p > 0.0f) || Ua * p < py_;
            if (local) {
                nL++;
            } else {
                nJ++;
                psum += (double)py_;
            }
            nA += accept;
        } else if (local) {
            accept = Ua * p < py_;
            nL++;
            nA += accept;
        } else {
            accept = true;
            nJ++;
        }
        if (accept) {
            xd = yd;
            Fr = Fy.x;
            Fg = Fy.y;
            Fb = Fy.z;
            p = py_;
            u = 1.0f;
        }
    }
    if (mine) c.x[xidx((uint32_t)lane, i, c.n)] = xd;
    if (lane == 0) {
        c.fpu[0 * c.n + i] = Fr;
        c.fpu[1 * c.n + i] = Fg;
        c.fpu[2 * c.n + i] = Fb;
        c.fpu[3 * c.n + i] = p;
        c.fpu[4 * c.n + i] = u;
        if (nJ) atomicAdd(c.counters + 0, (unsigned long long)nJ);
        if (nL) atomicAdd(c.counters + 1, (unsigned long long)nL);
        if (nA) atomicAdd(c.counters + 2, (unsigned long long)nA);
        if (psum != 0.0) atomicAdd(reinterpret_cast<double*>(c.counters + kCounterPSum), psum);
        flush_status(status, c.status);
    }
}

// ------------------------------------------------------------------ MALA
// Langevin local dynamics (JR_FLAG_MALA), one chain per thread for the whole
// launch.  The state's drift m(x) = clamp(sigma^2/2 grad log p(x), -2 sigma,
// 2 sigma) lives beside it (shared memory during the launch, c.drift between
// launches).  A MALA move proposes y = (x + m(x) + sigma N) mod 1 and accepts
// with min(1, p(y) q(x|y) / (p(x) q(y|x))), q(b|a) = prod_d phi_sigma(b_d - a_d
// - m_d(a)) on the signed torus difference.  With JR_FLAG_MH the chain is the
// MALA baseline (large steps from mu with probability l, MALA small steps);
// otherwise MALA Restore (Alg. 2, local move = the MALA step, k = c~ u / p).
__device__ __forceinline__ float torus_delta(float to, float from) {
    const float d = to - from;
    return d - floorf(d + 0.5f);
}

// log q(b | a) up to the constant, from a's drift ma (all [D] with stride B).
__device__ __forceinline__ float mala_log_q(const float* b, const float* a, const float* ma, int D, uint32_t B,
                                            float sigma) {
    float s = 0.f;
    for (int d = 0; d < D; ++d) {
        const float e = torus_delta(b[d * B], a[d * B]) - ma[d * B];
        s += e * e;
    }
    return -s / (2.0f * sigma * sigma);
}

template <bool kTrace>
__device__ __forceinline__ void chain_steps_mala(const SceneView& s, const ChainView& c, uint64_t i, bool active,
                                                 float* sh, uint64_t step_begin, uint32_t n_steps, uint8_t* tr_flags,
                                                 float* tr_dt, int32_t* tr_pix) {
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    const int D = (int)c.dim;
    float* x0 = sh + tid;                            // [4][D][B]: x, y, m(x), m(y)
    float* x1 = sh + (size_t)D * B + tid;
    float* m0 = sh + (size_t)2 * D * B + tid;
    float* m1 = sh + (size_t)3 * D * B + tid;
    const bool mh = (c.flags & JR_FLAG_MH) != 0;
    uint32_t nJ = 0, nL = 0, nA = 0;
    unsigned status = 0;
    double psum = 0.0;
    Work work;
    Jac3 JF;
    if (active) {
        load_coords(c, i, x0, B);
        for (int d = 0; d < D; ++d) m0[d * B] = c.drift[d * c.n + i];
    }
    float Fr = 0.f, Fg = 0.f, Fb = 0.f, p = 0.f, u = 1.f;
    if (active) {
        Fr = c.fpu[0 * c.n + i];
        Fg = c.fpu[1 * c.n + i];
        Fb = c.fpu[2 * c.n + i];
        p = c.fpu[3 * c.n + i];
        u = c.fpu[4 * c.n + i];
    }
    float *cur = x0, *cand = x1, *mc = m0, *my = m1;
    const uint32_t chain = c.chain_offset + (uint32_t)i;
    const float WH = (float)c.width * (float)c.height;
    for (uint32_t st = 0; st < n_steps; ++st) {
        const uint64_t step = step_begin + st;
        const uint4 r0 = active ? draw(c.seed, kTagStep, 0, chain, step) : make_uint4(0, 0, 0, 0);
        const float Ua = u01(r0.z);
        bool local = false;
        float dt = 0.f;
        if (mh) {
            local = !(u01(r0.x) < c.large_step);
            dt = step >= c.burn_in ? 1.0f : 0.0f;
        } else {
            const float E1 = -logf(1.0f - u01(r0.x));
            const float E2 = -logf(1.0f - u01(r0.y));
            const float t2 = p > 0.0f ? E2 * p / (c.c_tilde * u) : 0.0f;
            local = E1 < t2;
            dt = local ? E1 : t2;
        }
        int32_t pix = -1;
        if (active && dt > 0.0f && p > 0.0f) {
            uint32_t px = min((uint32_t)((double)cur[0] * (double)c.width), c.width - 1);
            uint32_t py = min((uint32_t)((double)cur[B] * (double)c.height), c.height - 1);
            pix = (int32_t)(py * c.width + px);
            const float wgt = mh ? WH / p : c.c_tilde * dt * WH / p;
            atomicAdd(c.fb + pix, make_float4(wgt * Fr, wgt * Fg, wgt * Fb, dt));
        }
        if (active) {
            for (int b = 0; 4 * b < D; ++b) {
                const uint4 r = draw(c.seed, kTagStep, (uint32_t)(b + 1), chain, step);
                const int d0 = 4 * b;
                if (local) {  // the MALA proposal: drift plus Gaussian pairs
                    float sn, cs;
                    float R = sqrtf(-2.0f * logf(1.0f - u01(r.x)));
                    sincospif(2.0f * u01(r.y), &sn, &cs);
                    cand[d0 * B] = wrap01(cur[d0 * B] + mc[d0 * B] + c.sigma * R * cs);
                    cand[(d0 + 1) * B] = wrap01(cur[(d0 + 1) * B] + mc[(d0 + 1) * B] + c.sigma * R * sn);
                    if (d0 + 2 < D) {
                        R = sqrtf(-2.0f * logf(1.0f - u01(r.z)));
                        sincospif(2.0f * u01(r.w), &sn, &cs);
                        cand[(d0 + 2) * B] = wrap01(cur[(d0 + 2) * B] + mc[(d0 + 2) * B] + c.sigma * R * cs);
                        cand[(d0 + 3) * B] = wrap01(cur[(d0 + 3) * B] + mc[(d0 + 3) * B] + c.sigma * R * sn);
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
        }
        const float3 Fy = eval_path_grad<false>(s, mask, active, (int)c.depth, cand, B, JF, status, work);
        bool accept = false;
        if (active) {
            for (int d = 0; d < D; ++d) my[d * B] = mala_drift(Fy, JF, d, c.sigma);
            const float py_ = lum(Fy);
            if (local) {
                if (!(p > 0.0f)) {
                    accept = true;
                } else if (py_ > 0.0f) {
                    const float la = logf(py_) - logf(p) + mala_log_q(cur, cand, my, D, B, c.sigma) -
                                     mala_log_q(cand, cur, mc, D, B, c.sigma);
                    accept = Ua > 0.0f ? logf(Ua) < la : true;
                }
                nL++;
                nA += accept;
            } else if (mh) {  // a large step: uniform and symmetric
                accept = !(p > 0.0f) || Ua * p < py_;
                nJ++;
                psum += (double)py_;
                nA += accept;
            } else {          // regeneration from mu
                accept = true;
                nJ++;
            }
            if (accept) {
                float* t0 = cur;
                cur = cand;
                cand = t0;
                float* t1 = mc;
                mc = my;
                my = t1;
                Fr = Fy.x;
                Fg = Fy.y;
                Fb = Fy.z;
                p = py_;
                u = 1.0f;
            }
            if (kTrace) {
                const uint64_t o = i * n_steps + st;
                if (tr_flags) tr_flags[o] = (uint8_t)((local ? 0 : 1) | ((mh || local) && accept ? 2 : 0));
                if (tr_dt) tr_dt[o] = pix >= 0 ? dt : 0.0f;
                if (tr_pix) tr_pix[o] = pix;
            }
        }
    }
    if (active) {
        float2* x2 = reinterpret_cast<float2*>(c.x);
        for (int k = 0; 2 * k < D; ++k) x2[(uint64_t)k * c.n + i] = make_float2(cur[2 * k * B], cur[(2 * k + 1) * B]);
        for (int d = 0; d < D; ++d) c.drift[d * c.n + i] = mc[d * B];
        c.fpu[0 * c.n + i] = Fr;
        c.fpu[1 * c.n + i] = Fg;
        c.fpu[2 * c.n + i] = Fb;
        c.fpu[3 * c.n + i] = p;
        c.fpu[4 * c.n + i] = u;
    }
    nJ = __reduce_add_sync(0xffffffffu, nJ);
    nL = __reduce_add_sync(0xffffffffu, nL);
    nA = __reduce_add_sync(0xffffffffu, nA);
    status = __reduce_or_sync(0xffffffffu, status);
    if (mh) psum = warp_sum(psum);
    if ((tid & 31) == 0) {
        if (nJ) atomicAdd(c.counters + 0, (unsigned long long)nJ);
        if (nL) atomicAdd(c.counters + 1, (unsigned long long)nL);
        if (nA) atomicAdd(c.counters + 2, (unsigned long long)nA);
        if (psum != 0.0) atomicAdd(reinterpret_cast<double*>(c.counters + kCounterPSum), psum);
        flush_status(status, c.status);
    }
}

template <bool kTrace>
__global__ void __launch_bounds__(128) step_kernel_mala(SceneView s, ChainView c, uint64_t step_begin,
                                                        uint32_t n_steps, uint8_t* tr_flags, float* tr_dt,
                                                        int32_t* tr_pix) {
    extern __shared__ float sh[];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    chain_steps_mala<kTrace>(s, c, i, i < c.n, sh, step_begin, n_steps, tr_flags, tr_dt, tr_pix);
}

// F, p and the drift of the stored states (chain creation and jr_set_state).
__global__ void __launch_bounds__(128) mala_reeval_kernel(SceneView s, ChainView c) {
    extern __shared__ float sh[];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const unsigned mask = __ballot_sync(0xffffffffu, i < c.n);
    if (i >= c.n) return;
    unsigned status = 0;
    Work w;
    Jac3 JF;
    load_coords(c, i, sh + threadIdx.x, blockDim.x);
    const float3 F =
        eval_path_grad<false>(s, mask, true, (int)c.depth, sh + threadIdx.x, blockDim.x, JF, status, w);
    c.fpu[0 * c.n + i] = F.x;
    c.fpu[1 * c.n + i] = F.y;
    c.fpu[2 * c.n + i] = F.z;
    c.fpu[3 * c.n + i] = lum(F);
    c.fpu[4 * c.n + i] = 1.0f;
    for (int d = 0; d < (int)c.dim; ++d) c.drift[d * c.n + i] = mala_drift(F, JF, d, c.sigma);
    flush_status(status, c.status);
}

// F and dF/dx for given states: x [D][n], F [3][n], dF [3][D][n].
__global__ void __launch_bounds__(128) eval_grad_kernel(SceneView s, uint32_t depth, const float* x, uint64_t n,
                                                        float* F, float* dF) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const unsigned mask = __ballot_sync(0xffffffffu, i < n);
    if (i >= n) return;
    unsigned status = 0;
    Work w;
    Jac3 JF;
    const float3 f = eval_path_grad<false>(s, mask, true, (int)depth, x + i, (uint32_t)n, JF, status, w);
    const int D = 2 + 2 * (int)depth;
    if (F) {
        F[i] = f.x;
        F[n + i] = f.y;
        F[2 * n + i] = f.z;
    }
    if (dF)
        for (int q = 0; q < 3; ++q)
            for (int d = 0; d < D; ++d) dF[((uint64_t)q * D + d) * n + i] = JF.c[q][d];
}

// One persistent launch over a batch of chain sets (scenes with different
// triangle counts, images and depths).  Blocks take work items -- a block of
// chains of one set -- from a global cursor; the host orders the items by
// estimated cost, so the longest items start first.  Every item runs all
// n_steps of Alg. 2 for its chains with the same code as step_kernel.
__global__ void __launch_bounds__(256, 4) batch_step_kernel(const BatchEntry* entries, const BatchItem* items,
                                                         uint32_t n_items, unsigned int* cursor, uint32_t n_steps) {
    extern __shared__ float sh[];
    __shared__ unsigned int item_s;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(cursor, 1u);
        __syncthreads();
        const unsigned it = item_s;
        __syncthreads();  // every thread has read item_s before it is overwritten
        if (it >= n_items) break;
        const BatchItem wi = items[it];
        const BatchEntry& e = entries[wi.set];  // descriptor fields are read where used
        const uint64_t i = wi.begin + threadIdx.x;
        chain_steps<false, false>(e.s, e.c, i, i < wi.end, sh, e.step, n_steps, nullptr, nullptr, nullptr, nullptr);
        __syncthreads();  // the shared state buffers are reused by the next item
    }
}

// Fold every set's framebuffer into its accumulator; advance every set's step
// index by n_steps; reset the work cursor for the next launch.
__global__ void batch_fold_kernel(BatchEntry* entries, const uint64_t* px_off, uint32_t n_sets, uint64_t total_px,
                                  unsigned int* cursor, uint32_t n_steps) {
    const uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (j == 0) *cursor = 0u;
    if (j < n_sets) entries[j].step += n_steps;
    if (j >= total_px) return;
    uint32_t lo = 0, hi = n_sets;  // the set whose pixel range holds j
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (px_off[mid] <= j) lo = mid;
        else hi = mid;
    }
    const uint64_t p = j - px_off[lo];
    float4* fb = entries[lo].c.fb;
    const float4 v = fb[p];
    if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
        double4_32a* acc = entries[lo].c.acc64;
        double4_32a a = acc[p];
        a.x += v.x;
        a.y += v.y;
        a.z += v.z;
        a.w += v.w;
        acc[p] = a;
        fb[p] = make_float4(0.f, 0.f, 0.f, 0.f);
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

// image = accumulator / J (Section 6.3, normalisation-free estimator); MH
// (mh_samples > 0): image = b_hat accumulator / N, the ergodic average over the
// N post-burn-in iterations scaled by b_hat = mean p of the large-step proposals.
__global__ void resolve_kernel(const double4_32a* acc, const unsigned long long* counters, float* rgb, uint32_t n,
                               int mh, uint64_t mh_samples) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const unsigned long long J = counters[0];
    const double4_32a a = acc[j];
    double inv = J > 0 ? 1.0 / (double)J : 0.0;
    if (mh) {
        const double psum = __longlong_as_double((long long)counters[kCounterPSum]);
        inv = J > 0 && mh_samples > 0 ? psum / (double)J / (double)mh_samples : 0.0;
    }
    rgb[3 * j] = (float)(a.x * inv);
    rgb[3 * j + 1] = (float)(a.y * inv);
    rgb[3 * j + 2] = (float)(a.z * inv);
}

__global__ void eval_states_kernel(SceneView s, uint32_t depth, float c_tilde, const float* x, uint64_t n, float* F,
                                   float* p, float* u, float* k, int32_t* ids, unsigned int* status_word) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const unsigned mask = __ballot_sync(0xffffffffu, i < n);
    if (i >= n) return;
    unsigned status = 0;
    const float3 f = eval_path(s, mask, true, (int)depth, x + i, (uint32_t)n, ids ? ids + i : nullptr, n, status);
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
    const unsigned mask = __ballot_sync(0xffffffffu, i < n);
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
    const float3 F = eval_path(s, mask, true, (int)depth, y, B, nullptr, 0, status);
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

// FP32 peak: every thread runs kChainsFma independent FMA chains for `iters`
// rounds (2 FLOP per FMA), so the FMA pipes never wait on a dependency; the
// values stay finite (a contraction towards 1) and are written out only if a
// condition that never holds is met, so nothing is optimised away.
constexpr int kChainsFma = 8;
__global__ void __launch_bounds__(256) fma_peak_kernel(uint32_t iters, float* sink) {
    float a[kChainsFma];
    const float m = 0.999f, c = 1e-3f * (float)(threadIdx.x & 7);
#pragma unroll
    for (int k = 0; k < kChainsFma; ++k) a[k] = 1.0f + 1e-3f * (float)k;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChainsFma; ++k) a[k] = fmaf(a[k], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChainsFma; ++k) s += a[k];
    if (s == -1.0f && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

inline unsigned grid_for(uint64_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t measure_fma_peak(double* tflops, double* ms_out, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel, 256, 0)) != cudaSuccess)
        return e;
    const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    const uint32_t iters = 1u << 14;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        fma_peak_kernel<<<grid, 256, 0, st>>>(iters, nullptr);
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
        fma_peak_kernel<<<grid, 256, 0, st>>>(iters, nullptr);
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
        if (rep == 0 || t < best) best = t;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flop = 2.0 * (double)grid * 256.0 * (double)iters * 16.0 * kChainsFma;
    *tflops = flop / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return cudaSuccess;
}

cudaError_t launch_init(const SceneView& s, const ChainView& c, cudaStream_t st) {
    const unsigned B = 128;
    init_kernel<<<grid_for(c.n, B), B, sizeof(float) * c.dim * B, st>>>(s, c);
    return cudaGetLastError();
}

cudaError_t launch_reeval(const SceneView& s, const ChainView& c, cudaStream_t st) {
    const unsigned B = 128;
    reeval_kernel<<<grid_for(c.n, B), B, sizeof(float) * c.dim * B, st>>>(s, c);
    return cudaGetLastError();
}

cudaError_t launch_step_warp(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                             cudaStream_t st) {
    if (c.n == 0 || n_steps == 0) return cudaSuccess;
    const uint64_t threads = 32 * c.n;
    step_kernel_warp<<<grid_for(threads, kWarpChainThreads), kWarpChainThreads, 0, st>>>(s, c, step_begin, n_steps);
    return cudaGetLastError();
}

cudaError_t launch_step(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                        uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix, unsigned long long* work_out, int block,
                        cudaStream_t st) {
    const unsigned B = (unsigned)block;
    const size_t shm = sizeof(float) * 2 * c.dim * B;  // <= 2 * 32 * 256 * 4 = 64 KB
    const unsigned G = grid_for(c.n, B);
    static DeviceOnce once;  // per device: opt in to > 48 KB of dynamic shared memory
    cudaError_t e0 = once.get(
        [](int, long long*) {
            const int lim = (int)(sizeof(float) * 2 * kMaxDim * 256);
            cudaError_t e;
            if ((e = cudaFuncSetAttribute(step_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          lim)) != cudaSuccess ||
                (e = cudaFuncSetAttribute(step_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          lim)) != cudaSuccess ||
                (e = cudaFuncSetAttribute(step_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          lim)) != cudaSuccess)
                return e;
            return cudaSuccess;
        },
        nullptr);
    if (e0 != cudaSuccess) return e0;
    if (work_out)
        step_kernel<false, true><<<G, B, shm, st>>>(s, c, step_begin, n_steps, nullptr, nullptr, nullptr, work_out);
    else if (tr_flags || tr_dt || tr_pix)
        step_kernel<true, false><<<G, B, shm, st>>>(s, c, step_begin, n_steps, tr_flags, tr_dt, tr_pix, nullptr);
    else
        step_kernel<false, false><<<G, B, shm, st>>>(s, c, step_begin, n_steps, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_step_mala(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                             uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix, cudaStream_t st) {
    const unsigned B = 128;
    const size_t shm = sizeof(float) * 4 * c.dim * B;  // <= 4 * 32 * 128 * 4 = 64 KB
    static DeviceOnce once;
    cudaError_t e0 = once.get(
        [](int, long long*) {
            const int lim = (int)(sizeof(float) * 4 * kMaxDim * 128);
            cudaError_t e;
            if ((e = cudaFuncSetAttribute(step_kernel_mala<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          lim)) != cudaSuccess ||
                (e = cudaFuncSetAttribute(step_kernel_mala<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
                    cudaSuccess)
                return e;
            return cudaSuccess;
        },
        nullptr);
    if (e0 != cudaSuccess) return e0;
    const unsigned G = grid_for(c.n, B);
    if (tr_flags || tr_dt || tr_pix)
        step_kernel_mala<true><<<G, B, shm, st>>>(s, c, step_begin, n_steps, tr_flags, tr_dt, tr_pix);
    else
        step_kernel_mala<false><<<G, B, shm, st>>>(s, c, step_begin, n_steps, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_mala_reeval(const SceneView& s, const ChainView& c, cudaStream_t st) {
    mala_reeval_kernel<<<grid_for(c.n, 128), 128, sizeof(float) * c.dim * 128, st>>>(s, c);
    return cudaGetLastError();
}

cudaError_t launch_eval_grad(const SceneView& s, uint32_t depth, const float* x, uint64_t n, float* F, float* dF,
                             cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    eval_grad_kernel<<<grid_for(n, 128), 128, 0, st>>>(s, depth, x, n, F, dF);
    return cudaGetLastError();
}

cudaError_t launch_fold(const ChainView& c, cudaStream_t st) {
    const uint32_t n = c.width * c.height;
    fold_kernel<<<grid_for(n, 256), 256, 0, st>>>(c.fb, c.acc64, n);
    return cudaGetLastError();
}

cudaError_t launch_batch(BatchEntry* entries, const BatchItem* items, uint32_t n_items, const uint64_t* px_off,
                         uint32_t n_sets, uint64_t total_px, unsigned int* cursor, uint32_t max_dim, int block,
                         uint32_t n_steps, cudaStream_t st) {
    static DeviceOnce once;  // per device: the SM count, after the shared-memory opt-in
    const size_t shm = sizeof(float) * 2 * max_dim * (size_t)block;
    long long sms = 0;
    cudaError_t e = once.get(
        [](int dev, long long* v) {
            int n = 0;
            cudaError_t r;
            if ((r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
                (r = cudaFuncSetAttribute(batch_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(float) * 2 * kMaxDim * 256))) != cudaSuccess)
                return r;
            *v = n;
            return cudaSuccess;
        },
        &sms);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel, block, shm)) != cudaSuccess)
        return e;
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)sms * (per_sm > 0 ? per_sm : 1), n_items);
    if (n_steps > 0 && n_items > 0)
        batch_step_kernel<<<grid, block, shm, st>>>(entries, items, n_items, cursor, n_steps);
    const uint64_t total = total_px > n_sets ? total_px : n_sets;
    batch_fold_kernel<<<grid_for(total, 256), 256, 0, st>>>(entries, px_off, n_sets, total_px, cursor, n_steps);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const ChainView& c, float* rgb, uint64_t mh_samples, cudaStream_t st) {
    const uint32_t n = c.width * c.height;
    resolve_kernel<<<grid_for(n, 256), 256, 0, st>>>(c.acc64, c.counters, rgb, n, (c.flags & JR_FLAG_MH) != 0,
                                                     mh_samples);
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
