// Wavefront execution of the Jump Restore step (sm_103a).
//
// The megakernel (jr_kernels.cu) keeps one chain per thread for a whole
// launch; its warps idle while their longest path and their longest ray finish.
// Here a step of Alg. 2 (Section 7.2) is split in two launches:
//
//   step kernel (all chains, converged): finish the previous step (MH
//     acceptance or regeneration), draw the new step's clocks t1 ~ Exp(1),
//     t2 ~ Exp(k), k = c~ u / p (Section 6.2), splat (dt, x) (Sections 6.3/7.4),
//     build the candidate y (Gaussian small step or a draw from mu); every
//     chain joins the path queue.
//   path kernel (persistent warps): the whole path of every queued candidate,
//     vertex after vertex, in registers: warp-synchronous BVH traversal, batched
//     shading, and dynamic fetch of new paths into idle lanes, so that a warp
//     idles neither for its longest ray nor for its longest path.
//
// Per-chain arithmetic is the megakernel's, through the same device functions,
// so both modes give the same chains for the same Philox streams.  The state
// lives in two buffers (x, y) with a per-chain parity byte, so an accepted
// move is a flip; the final finish launch copies states back into x.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/jr.h"
#include "jr_device.cuh"
#include "jr_internal.h"

namespace jr {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRefill = 4;  // refill a warp once this many lanes are idle

// Append chain i to a queue if `live`; one atomic per warp.  All 32 lanes call.
__device__ __forceinline__ void enqueue(bool live, uint32_t i, uint32_t* q, unsigned int* count) {
    const unsigned m = __ballot_sync(kFull, live);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (live) q[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// The splat of a step, aggregated per warp: the lanes that splat into the same
// pixel (pix >= 0) are grouped with __match_any_sync and one lane of each group
// adds the group's sum with one vector atomic.  All 32 lanes call.
__device__ __forceinline__ void splat_warp(float4* fb, int32_t pix, float4 v) {
    const unsigned want = __ballot_sync(kFull, pix >= 0);
    if (!want) return;
    const unsigned peers = __match_any_sync(kFull, pix);
    if (pix < 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    if (peers != (1u << lane)) {  // more than one lane in the pixel: the leader gathers
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        for (unsigned m = peers; m; m &= m - 1) {
            const int j = __ffs(m) - 1;
            sum.x += __shfl_sync(peers, v.x, j);
            sum.y += __shfl_sync(peers, v.y, j);
            sum.z += __shfl_sync(peers, v.z, j);
            sum.w += __shfl_sync(peers, v.w, j);
        }
        v = sum;
    }
    if (lane == leader) atomicAdd(fb + pix, v);
}

// The step kernels' counters (J, local steps, acceptances, status, and with
// JR_FLAG_MH the sum of p over large steps), flushed once per block: each warp
// adds its counts into the block's shared totals, and the block's last warp to
// arrive issues the global atomics, so no warp waits at a closing barrier for
// the others (measured: the step kernel about 6 % faster than with one) and the
// three counter addresses see one atomic per block.  The totals are zeroed
// behind the block's first barrier.  All 32 lanes of every warp call.
struct BlockCounts {
    unsigned J, L, A, status, arrived;
    double ps;
};
__device__ __forceinline__ void block_counts_init(BlockCounts& b) {
    if (threadIdx.x == 0) {
        b.J = b.L = b.A = b.status = b.arrived = 0;
        b.ps = 0.0;
    }
    __syncthreads();
}
__device__ __forceinline__ void count_and_flush_last(BlockCounts& b, uint32_t nJ, uint32_t nL, uint32_t nA,
                                                     unsigned status, double ps, const ChainView& c) {
    const bool mh = (c.flags & JR_FLAG_MH) != 0;
    nJ = __reduce_add_sync(kFull, nJ);
    nL = __reduce_add_sync(kFull, nL);
    nA = __reduce_add_sync(kFull, nA);
    status = __reduce_or_sync(kFull, status);
    if (mh) ps = warp_sum(ps);
    if ((threadIdx.x & 31) == 0) {
        if (nJ) atomicAdd(&b.J, nJ);
        if (nL) atomicAdd(&b.L, nL);
        if (nA) atomicAdd(&b.A, nA);
        if (status) atomicOr(&b.status, status);
        if (mh && ps != 0.0) atomicAdd(&b.ps, ps);
        __threadfence_block();
        if (atomicAdd(&b.arrived, 1u) == (blockDim.x >> 5) - 1) {
            __threadfence_block();
            const unsigned sJ = *(volatile unsigned*)&b.J, sL = *(volatile unsigned*)&b.L,
                           sA = *(volatile unsigned*)&b.A, st = *(volatile unsigned*)&b.status;
            const double sp = *(volatile double*)&b.ps;
            if (sJ) atomicAdd(c.counters + 0, (unsigned long long)sJ);
            if (sL) atomicAdd(c.counters + 1, (unsigned long long)sL);
            if (sA) atomicAdd(c.counters + 2, (unsigned long long)sA);
            if (st) atomicOr(c.status, st);
            if (mh && sp != 0.0) atomicAdd(reinterpret_cast<double*>(c.counters + kCounterPSum), sp);
        }
    }
}

// finish = 1: complete step `step - 1` of every chain.  begin = 1: start step
// `step`.  With begin = 0 the launch also moves every state back into x.
// restart = 1: the step is a restart of every chain from mu (a new tour that is
// not a regeneration of Alg. 2: no clocks, no splat, J unchanged); `step` is
// then the restart epoch and the stream tag is kTagRestart.
// With a flow attached (c.flow.D > 0), a regeneration draws from the flow when
// Ub < beta (Ub = fourth value of block 0), else uniformly.  Flow draws go to
// the sampling queue, whose kernel fills in y and u(y) before the path kernel
// (ua = -3 marks them).  u(y) of the other candidates is needed only where the
// candidate becomes a state with p > 0 (k = c~ u / p is +inf at p = 0 whatever
// u is; a rejected local candidate never becomes a state), so the path kernel
// queues exactly those rows for the density pass after it; a state with p = 0
// keeps u = 1 as a placeholder.
// mode = kModeDrain: a kill ends the chain's tour (counted in J) and the chain
// (done = 1); done chains do nothing; no regeneration starts a new tour.
// Chains still in a tour after the step are counted in qcount[kQActive].
// Outside a drain every chain is traced, so the path queue is the identity
// (chain j is entry j) and is not written; a drain step writes it.
//
// step_chain is one chain's part (the body of the step kernel and of the
// batched step kernel).  traced: the candidate is traced this step;
// to_sample: it is a flow draw; active: in a drain, the tour goes on.
// With JR_FLAG_MH the chain runs the MH baseline (Alg. 1 with the mixture
// proposal of Section 5): the candidate is a large step (a draw from mu, as a
// regeneration's) with probability l, else a small step (as a local move's);
// every candidate goes through the MH acceptance; the held state is splatted
// (weight W H F / p, count 1) once the step index reaches the burn-in.  The
// stored Ua carries the large-step flag in its sign bit (-Ua, -0 included), so
// the acceptance sees the exact Ua.  ps collects p of the large-step proposals.
// The splat is returned (splat_pix >= 0, splat_val), not added: the caller adds
// it for the whole warp (splat_warp).
__device__ __forceinline__ void step_chain(const ChainView& c, uint64_t i, uint64_t step, bool finish, bool begin,
                                           int mode, uint32_t& nJ, uint32_t& nL, uint32_t& nA, unsigned& status,
                                           double& ps, bool& traced, bool& to_sample, bool& active,
                                           int32_t& splat_pix, float4& splat_val) {
    const int D = (int)c.dim;
    const uint64_t n = c.n;
    const WaveView& w = c.wf;
    const bool has_flow = c.flow.D != 0;
    const bool mh = (c.flags & JR_FLAG_MH) != 0;
    const bool restart = mode == kModeRestart, drain = mode == kModeDrain;
    // A chain whose tour ended earlier in a drain has nothing to finish and
    // nothing to begin: it leaves after one byte (late in a drain nearly every
    // chain is such a chain, and the full loads below cost the drain's steps
    // most of their time).  The closing launch (begin = 0) still visits it, to
    // move its state back into x.
    if (drain && begin && w.done[i]) {
        traced = false;
        return;
    }
    // Every load the step needs is issued here, before any store: the film
    // point of the current state is read from both buffers, so that no
    // load waits for the parity byte.
    uint8_t par = w.par[i];
    float Fr = c.fpu[0 * n + i], Fg = c.fpu[1 * n + i], Fb = c.fpu[2 * n + i];
    float p = c.fpu[3 * n + i], u = c.fpu[4 * n + i];
    const float ua = finish ? w.ua[i] : 0.0f;
    const float4 pf = finish ? w.fy[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 xs = make_float2(0.f, 0.f), ys = make_float2(0.f, 0.f);
    if (begin) {  // coordinate pair 0 (the film point) of both buffers
        xs = reinterpret_cast<const float2*>(c.x)[i];
        ys = reinterpret_cast<const float2*>(w.y)[i];
    }
    const bool was_done = drain && w.done[i];
    if (finish && !(drain && ua == -2.0f)) {
        const float3 Fy = finite_or_zero(f3(pf.x, pf.y, pf.z), status);
        const float py = lum(Fy);
        bool accept;
        if (restart) {     // a restart: the new tour's start, not a regeneration
            accept = true;
            w.done[i] = 0;
        } else if (mh) {   // MH baseline: U < min(1, p(y)/p(x)), 1 if p(x) = 0
            const bool large = signbit(ua);
            accept = !(p > 0.0f) || fabsf(ua) * p < py;
            if (large) {
                nJ++;
                ps += (double)py;
            } else {
                nL++;
            }
            nA += accept;
        } else if (ua >= 0.0f) {  // local branch: MH acceptance, U < min(1, p(y)/p(x))
            accept = ua * p < py;
            nL++;
            nA += accept;
        } else {           // regeneration: the candidate is the new tour's start
            accept = true;
            nJ++;
        }
        if (accept) {
            par ^= 1;
            Fr = Fy.x;
            Fg = Fy.y;
            Fb = Fy.z;
            p = py;
            u = has_flow && py > 0.0f ? w.uy[i] : 1.0f;
            c.fpu[0 * n + i] = Fr;
            c.fpu[1 * n + i] = Fg;
            c.fpu[2 * n + i] = Fb;
            c.fpu[3 * n + i] = p;
            c.fpu[4 * n + i] = u;
        }
    }
    float2* cur = reinterpret_cast<float2*>(par ? w.y : c.x);  // pair layout: pair k of chain i at k n + i
    float2* cand = reinterpret_cast<float2*>(par ? c.x : w.y);
    if (begin && was_done) {  // finished its tour during this drain
        w.ua[i] = -2.0f;
        traced = false;
    } else if (begin) {
        const uint32_t chain = c.chain_offset + (uint32_t)i;
        const uint32_t tag = restart ? kTagRestart : kTagStep;
        const uint4 r0 = draw(c.seed, tag, 0, chain, step);
        const float Ua = u01(r0.z);
        bool local;
        float dt;
        if (mh) {
            local = !(u01(r0.x) < c.large_step);
            dt = step >= c.burn_in ? 1.0f : 0.0f;
        } else {
            const float E1 = -logf(1.0f - u01(r0.x));
            const float E2 = -logf(1.0f - u01(r0.y));
            const float t2 = p > 0.0f ? E2 * p / (c.c_tilde * u) : 0.0f;
            local = !restart && E1 < t2;  // a tie goes to the killing branch
            dt = local ? E1 : t2;
            if (c.flags & JR_FLAG_RAO_BLACKWELL) dt = p > 0.0f ? p / (p + c.c_tilde * u) : 0.0f;
            if (restart) dt = 0.0f;
        }
        const bool use_flow = has_flow && !local && u01(r0.w) < c.flow.beta;
        to_sample = use_flow;
        const float x0 = par ? ys.x : xs.x, x1 = par ? ys.y : xs.y;  // = cur[i]
        if (dt > 0.0f && p > 0.0f) {
            uint32_t px = min((uint32_t)((double)x0 * (double)c.width), c.width - 1);
            uint32_t py = min((uint32_t)((double)x1 * (double)c.height), c.height - 1);
            const float WH = (float)c.width * (float)c.height;
            const float wgt = mh ? WH / p : c.c_tilde * dt * WH / p;
            splat_pix = (int32_t)(py * c.width + px);
            splat_val = make_float4(wgt * Fr, wgt * Fg, wgt * Fb, dt);
        }
        w.ua[i] = mh ? (local ? Ua : -Ua) : local ? Ua : use_flow ? -3.0f : -1.0f;
        if (drain && !local) {  // the tour ends here; no new tour in a drain
            nJ++;
            w.done[i] = 1;
            w.ua[i] = -2.0f;
            traced = false;
            to_sample = false;
        }
        active = drain && local;
        for (int b = 0; traced && 4 * b < D; ++b) {
            const uint4 r = draw(c.seed, tag, (uint32_t)(b + 1), chain, step);
            const uint64_t q0 = (uint64_t)(2 * b) * n + i;  // pairs 2b and 2b + 1: coordinates 4b .. 4b + 3
            float v0, v1, v2 = 0.f, v3 = 0.f;
            const bool two = 4 * b + 2 < D;
            if (local) {
                float sn, cs;
                float R = sqrtf(-2.0f * logf(1.0f - u01(r.x)));
                sincospif(2.0f * u01(r.y), &sn, &cs);
                const float2 c0 = b == 0 ? make_float2(x0, x1) : cur[q0];
                v0 = wrap01(c0.x + c.sigma * R * cs);
                v1 = wrap01(c0.y + c.sigma * R * sn);
                if (two) {
                    R = sqrtf(-2.0f * logf(1.0f - u01(r.z)));
                    sincospif(2.0f * u01(r.w), &sn, &cs);
                    const float2 c1 = cur[q0 + n];
                    v2 = wrap01(c1.x + c.sigma * R * cs);
                    v3 = wrap01(c1.y + c.sigma * R * sn);
                }
            } else {
                v0 = u01(r.x);
                v1 = u01(r.y);
                v2 = u01(r.z);
                v3 = u01(r.w);
            }
            cand[q0] = make_float2(v0, v1);
            if (two) cand[q0 + n] = make_float2(v2, v3);
            if (b == 0) {  // the path's start record
                float2* f = reinterpret_cast<float2*>(w.fy + i);
                f[0] = make_float2(v0, v1);
                f[1] = make_float2(v2, v3);
            }
        }
    } else if (par) {
        float2* x2 = reinterpret_cast<float2*>(c.x);
        const float2* y2 = reinterpret_cast<const float2*>(w.y);
        for (int k = 0; 2 * k < D; ++k) x2[(uint64_t)k * n + i] = y2[(uint64_t)k * n + i];
        par = 0;
    }
    w.par[i] = par;
}

__global__ void __launch_bounds__(128, 10) wf_step_kernel(ChainView c, uint64_t step, int finish, int begin,
                                                          int mode) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool valid = i < c.n;
    const uint64_t n = c.n;
    const WaveView& w = c.wf;
    const bool has_flow = c.flow.D != 0;
    const bool drain = mode == kModeDrain;
    __shared__ BlockCounts bc;
    block_counts_init(bc);
    uint32_t nJ = 0, nL = 0, nA = 0;
    unsigned status = 0;
    double ps = 0.0;
    bool to_sample = false, traced = valid, active = false;
    int32_t spix = -1;
    float4 sval = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid)
        step_chain(c, i, step, finish, begin, mode, nJ, nL, nA, status, ps, traced, to_sample, active, spix, sval);
    if (begin) splat_warp(c.fb, spix, sval);
    if (begin) {
        if (drain) enqueue(traced, (uint32_t)i, w.queue, w.qcount + 0);
        if (has_flow) enqueue(to_sample, (uint32_t)i, w.fq + n, w.qcount + kQFlowSample);
        if (drain) {  // counters[3]: 1 + the last drain step after which a tour was still open
            const unsigned na = __popc(__ballot_sync(kFull, active));
            if ((threadIdx.x & 31) == 0 && na) {
                atomicAdd(w.qcount + kQActive, na);
                atomicMax(c.counters + 3, (unsigned long long)step + 1);
            }
        }
    }
    count_and_flush_last(bc, nJ, nL, nA, status, ps, c);
}

// Whole paths of every queued chain in one persistent launch.  A lane keeps
// its path (ray, throughput T, emission F, vertex v) in registers and moves
// between three states: traversing its current ray; waiting to shade (its
// closest hit is known); idle (no path).  Traversal rounds are warp-
// synchronous while-while rounds with speculative traversal (Aila & Laine
// 2009): a lane that meets a leaf postpones it and keeps descending inner
// nodes until all but kSearchExit lanes hold a leaf.  A warp shades its
// waiting lanes together once kShadeBatch of them wait, or once they are at
// least as many as the traversing lanes (measured: 1.22 -> 1.25e9 chain
// steps/s against the batch rule alone); a shaded path either continues with
// its next ray or ends (F
// goes to fy, and, with a flow, the row joins the density queue: when its
// candidate will become a state with p > 0 and still lacks u(y); the finish of
// the next step kernel takes the same decision from the same values).  Idle lanes take new
// paths from the queue (dynamic fetch, so a warp does not idle for its
// longest path); a new path starts at the camera ray through the candidate's
// film point (y0, y1) with T = 1, F = 0.  ident = 1: the queue is the identity
// over all n chains (every step but a drain step).
// A path's loads never wait on one another: the start record fy[i] =
// (y0, y1, y2, y3) and the parity byte arrive together, and the two
// coordinates of vertex v + 1 are loaded when vertex v is shaded, so they
// arrive while the next ray traverses.  These per-chain loads and the store of
// F are marked evict-first (ld/st .cs): each is touched once per launch, and
// L1 is better kept for the BVH nodes, the triangles and the traversal stacks
// (measured: +0.3 %).
constexpr int kShadeBatch = 16;
enum PathState : uint32_t { kIdle = 0, kTraverse = 1, kWaitShade = 2 };


__global__ void __launch_bounds__(128) wf_path_kernel(SceneView s, ChainView c, int ident) {
    const WaveView& w = c.wf;
    const uint32_t* qin = w.queue;
    const unsigned count = ident ? (unsigned)c.n : w.qcount[0];
    if ((uint64_t)blockIdx.x * blockDim.x >= count) return;
    unsigned int* fetch = w.qcount + (kMaxDepth + 2);
    const uint64_t n = c.n;
    const int depth = (int)c.depth;
    const bool has_flow = c.flow.D != 0;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned status = 0;
    Work wk;
    Trav r;
    int stack[kStackSize];
    uint32_t state = kIdle, i = 0;
    int v = 0, leaf = kSentinel;
    bool failed = false, drained = false;
    float3 T = f3(1.f, 1.f, 1.f), F = f3(0.f, 0.f, 0.f);
    float u1 = 0.f, u2 = 0.f;  // the coordinates of vertex v
    bool cx = false;           // the candidate lives in x (else in y)
    while (true) {
        // shade the waiting lanes as a batch
        const unsigned waiting = __ballot_sync(kFull, state == kWaitShade);
        const unsigned tracing = __ballot_sync(kFull, state == kTraverse);
        if (waiting && (__popc(waiting) >= kShadeBatch || __popc(waiting) >= __popc(tracing))) {
            bool need_u = false;
            if (state == kWaitShade) {
                bool live = false;
                if (r.best >= 0) {
                    float3 o = r.o, d = r.d;
                    live = shade_vertex(s, r.best, r.tb, v, depth, v < depth ? u1 : 0.f, v < depth ? u2 : 0.f, o,
                                        d, T, F);
                    if (live) {
                        ++v;
                        trav_begin(s, r, o, d);
                        state = kTraverse;
                        if (v < depth) {  // vertex v's coordinate pair, one 8-byte load (evict-first)
                            const float2 uv =
                                __ldcs(reinterpret_cast<const float2*>(cx ? c.x : w.y) + (uint64_t)(1 + v) * n + i);
                            u1 = uv.x;
                            u2 = uv.y;
                        }
                    }
                }
                if (!live) {
                    __stcs(w.fy + i, make_float4(F.x, F.y, F.z, 0.f));
                    if (has_flow) {
                        unsigned ignored = 0;
                        const float py = lum(finite_or_zero(F, ignored));
                        const float ua = w.ua[i];
                        need_u = ua >= 0.0f ? ua * c.fpu[3 * n + i] < py : (ua == -1.0f && py > 0.0f);
                    }
                    state = kIdle;
                }
            }
            if (has_flow) enqueue(need_u, i, w.fq, w.qcount + kQFlowDensity);
        }
        // take new paths for idle lanes
        const unsigned idle = __ballot_sync(kFull, state == kIdle);
        if (!drained && idle && (__popc(idle) >= kRefill || idle == kFull)) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(fetch, (unsigned)__popc(idle));
            base = __shfl_sync(kFull, base, 0);
            if (base + (unsigned)__popc(idle) >= count) drained = true;
            if (state == kIdle) {
                const unsigned j = base + __popc(idle & lt);
                if (j < count) {
                    i = ident ? j : qin[j];
                    const float4 y = __ldcs(w.fy + i);
                    cx = __ldcs(w.par + i) != 0;
                    u1 = y.z;
                    u2 = y.w;
                    float3 o, d;
                    camera_ray(s, y.x, y.y, o, d);
                    T = f3(1.f, 1.f, 1.f);
                    F = f3(0.f, 0.f, 0.f);
                    v = 0;
                    trav_begin(s, r, o, d);
                    state = s.root != kSentinel ? kTraverse : kWaitShade;  // empty scene: a miss
                }
            }
        }
        if (!__any_sync(kFull, state != kIdle)) {
            if (drained) break;
            continue;
        }
        // one speculative while-while traversal round
        const bool trav = state == kTraverse;
        if (trav && leaf == kSentinel && r.ref < 0 && r.ref != kSentinel) {
            leaf = r.ref;
            r.ref = r.sp > 0 ? stack[--r.sp] : kSentinel;
        }
        const unsigned tracing_now = __ballot_sync(kFull, trav);
        while (__any_sync(kFull, trav && leaf == kSentinel && r.ref >= 0)) {
            if (trav && r.ref >= 0) {
                if (!trav_node<false>(s, r, stack, status, wk)) {
                    r.best = -1;
                    r.ref = kSentinel;
                    leaf = kSentinel;
                    failed = true;
                } else if (leaf == kSentinel && r.ref < 0 && r.ref != kSentinel) {
                    leaf = r.ref;
                    r.ref = r.sp > 0 ? stack[--r.sp] : kSentinel;
                }
            }
            if (search_done(__ballot_sync(kFull, trav && leaf == kSentinel && r.ref >= 0), tracing_now)) break;
        }
        if (trav) {
            if (leaf != kSentinel) {
                trav_test_leaf<false>(s, r, leaf, wk);
                leaf = kSentinel;
            }
            if (failed || r.ref == kSentinel) {
                state = kWaitShade;
                failed = false;
            }
        }
    }
    status = __reduce_or_sync(kFull, status);
    if (lane == 0 && status) atomicOr(c.status, status);
}

// ---------------------------------------------------------------------------
// Batched wavefront: the chain sets of a batch (one scene each) advance in the
// same step and path launches.  Their scenes are merged into one device scene
// (nodes, triangles and materials concatenated, with child, leaf and material
// indices rebased), so the traversal's pointers are uniform over a warp and a
// lane keeps only its set, the set's chain buffers and its root.

// Rebase one scene's nodes and triangles after they were copied into the
// merged arrays at offsets node_off, tri_off, mat_off.
__global__ void rebase_scene_kernel(Bvh4Node* nodes, uint32_t n_nodes, TriRecord* tris, uint32_t n_tris,
                                    int node_off, int tri_off, int mat_off) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_nodes) {
        int4 r = nodes[j].refs;
        int* rr = &r.x;
        for (int q = 0; q < 4; ++q) rr[q] = rebase_ref(rr[q], node_off, tri_off);
        nodes[j].refs = r;
    }
    if (j < n_tris) tris[j].e1_mat.w = __int_as_float(__float_as_int(tris[j].e1_mat.w) + mat_off);
}

// The step kernel over every set: one block per work item (128 chains of one
// set); the set's step index is entries[set].step + k.
__global__ void __launch_bounds__(128) wf_batch_step_kernel(const BatchEntry* entries, const BatchItem* items,
                                                                uint32_t k, int finish, int begin) {
    const BatchItem it = items[blockIdx.x];
    const BatchEntry& e = entries[it.set];
    const uint64_t i = it.begin + threadIdx.x;
    __shared__ BlockCounts bc;
    block_counts_init(bc);
    uint32_t nJ = 0, nL = 0, nA = 0;
    unsigned status = 0;
    double ps = 0.0;
    bool traced = true, to_sample = false, active = false;
    int32_t spix = -1;
    float4 sval = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < it.end)
        step_chain(e.c, i, e.step + k, finish, begin, kModeStep, nJ, nL, nA, status, ps, traced, to_sample, active,
                   spix, sval);
    if (begin) splat_warp(e.c.fb, spix, sval);
    // a set with a flow: its flow draws go to the set's sampling queue (a
    // block's chains are one set's, so the warp's enqueue has one queue)
    if (begin && e.c.flow.D != 0)
        enqueue(to_sample && i < it.end, (uint32_t)i, e.c.wf.fq + e.c.n, e.c.wf.qcount + kQFlowSample);
    count_and_flush_last(bc, nJ, nL, nA, status, ps, e.c);  // a block's chains are one set's
}

// The path kernel over every set's candidates: item j of the launch is chain
// j - off[q] of set q, off[q] <= j < off[q + 1] (off = the sets' chain
// prefix sums, copied to shared memory).  The lane logic is the single-set
// path kernel's; per lane it keeps the set, its depth, the candidate buffer
// and its stride, and starts each ray at the set's root in the merged scene.
__global__ void __launch_bounds__(128, 7) wf_batch_path_kernel(SceneView m, const BatchEntry* entries, const int* roots,
                                                            const uint64_t* chain_off, uint32_t n_sets,
                                                            unsigned int* fetch) {
    extern __shared__ uint64_t off_s[];
    for (uint32_t q = threadIdx.x; q <= n_sets; q += blockDim.x) off_s[q] = chain_off[q];
    __syncthreads();
    const unsigned count = (unsigned)off_s[n_sets];
    if ((uint64_t)blockIdx.x * blockDim.x >= count) return;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned status = 0;
    Work wk;
    Trav r;
    int stack[kStackSize];
    uint32_t state = kIdle, i = 0, set = 0, nst = 0;
    int v = 0, leaf = kSentinel, depth = 0;
    bool failed = false, drained = false;
    float3 T = f3(1.f, 1.f, 1.f), F = f3(0.f, 0.f, 0.f);
    float u1 = 0.f, u2 = 0.f;       // the coordinates of vertex v
    const float* cand = nullptr;     // the candidate's buffer (pair layout, nst chains)
    while (true) {
        // shade the waiting lanes as a batch
        const unsigned waiting = __ballot_sync(kFull, state == kWaitShade);
        const unsigned tracing = __ballot_sync(kFull, state == kTraverse);
        if (waiting && (__popc(waiting) >= kShadeBatch || __popc(waiting) >= __popc(tracing))) {
            bool need_u = false;
            if (state == kWaitShade) {
                bool live = false;
                if (r.best >= 0) {
                    float3 o = r.o, d = r.d;
                    live = shade_vertex(m, r.best, r.tb, v, depth, v < depth ? u1 : 0.f, v < depth ? u2 : 0.f, o,
                                        d, T, F);
                    if (live) {
                        ++v;
                        trav_begin_at(r, o, d, roots[set]);
                        state = kTraverse;
                        if (v < depth) {  // vertex v's coordinate pair, one 8-byte load
                            const float2 uv = __ldcs(reinterpret_cast<const float2*>(cand) + (uint64_t)(1 + v) * nst + i);
                            u1 = uv.x;
                            u2 = uv.y;
                        }
                    }
                }
                if (!live) {
                    const ChainView& c = entries[set].c;
                    __stcs(c.wf.fy + i, make_float4(F.x, F.y, F.z, 0.f));
                    if (status) {
                        atomicOr(c.status, status);
                        status = 0;
                    }
                    if (c.flow.D != 0) {  // as in the single-set path kernel
                        unsigned ignored = 0;
                        const float py = lum(finite_or_zero(F, ignored));
                        const float ua = c.wf.ua[i];
                        need_u = ua >= 0.0f ? ua * c.fpu[3 * c.n + i] < py : (ua == -1.0f && py > 0.0f);
                    }
                    state = kIdle;
                }
            }
            // rows whose u(y) the density pass must fill, appended to their set's
            // queue: lanes of one warp may hold different sets, so the lanes of
            // each set share one atomic (all 32 lanes take part)
            const unsigned peers = __match_any_sync(kFull, need_u ? set : 0xffffffffu);
            if (need_u) {
                const int leader = __ffs(peers) - 1;
                unsigned base = 0;
                if (lane == leader)
                    base = atomicAdd(entries[set].c.wf.qcount + kQFlowDensity, (unsigned)__popc(peers));
                base = __shfl_sync(peers, base, leader);
                entries[set].c.wf.fq[base + __popc(peers & lt)] = i;
            }
        }
        // take new paths for idle lanes
        const unsigned idle = __ballot_sync(kFull, state == kIdle);
        if (!drained && idle && (__popc(idle) >= kRefill || idle == kFull)) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(fetch, (unsigned)__popc(idle));
            base = __shfl_sync(kFull, base, 0);
            if (base + (unsigned)__popc(idle) >= count) drained = true;
            if (state == kIdle) {
                const unsigned j = base + __popc(idle & lt);
                if (j < count) {
                    uint32_t lo = 0, hi = n_sets;  // the set whose chain range holds j
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) / 2;
                        if (off_s[mid] <= j) lo = mid;
                        else hi = mid;
                    }
                    set = lo;
                    i = j - (uint32_t)off_s[lo];
                    const BatchEntry& e = entries[set];
                    const float4 y = __ldcs(e.c.wf.fy + i);
                    cand = __ldcs(e.c.wf.par + i) ? e.c.x : e.c.wf.y;
                    nst = (uint32_t)e.c.n;
                    depth = (int)e.c.depth;
                    u1 = y.z;
                    u2 = y.w;
                    float3 o, d;
                    camera_ray(e.s, y.x, y.y, o, d);
                    T = f3(1.f, 1.f, 1.f);
                    F = f3(0.f, 0.f, 0.f);
                    v = 0;
                    const int root = roots[set];
                    trav_begin_at(r, o, d, root);
                    state = root != kSentinel ? kTraverse : kWaitShade;  // empty scene: a miss
                }
            }
        }
        if (!__any_sync(kFull, state != kIdle)) {
            if (drained) break;
            continue;
        }
        // one speculative while-while traversal round
        const bool trav = state == kTraverse;
        if (trav && leaf == kSentinel && r.ref < 0 && r.ref != kSentinel) {
            leaf = r.ref;
            r.ref = r.sp > 0 ? stack[--r.sp] : kSentinel;
        }
        const unsigned tracing_now = __ballot_sync(kFull, trav);
        while (__any_sync(kFull, trav && leaf == kSentinel && r.ref >= 0)) {
            if (trav && r.ref >= 0) {
                if (!trav_node<false>(m, r, stack, status, wk)) {
                    r.best = -1;
                    r.ref = kSentinel;
                    leaf = kSentinel;
                    failed = true;
                } else if (leaf == kSentinel && r.ref < 0 && r.ref != kSentinel) {
                    leaf = r.ref;
                    r.ref = r.sp > 0 ? stack[--r.sp] : kSentinel;
                }
            }
            if (search_done(__ballot_sync(kFull, trav && leaf == kSentinel && r.ref >= 0), tracing_now)) break;
        }
        if (trav) {
            if (leaf != kSentinel) {
                trav_test_leaf<false>(m, r, leaf, wk);
                leaf = kSentinel;
            }
            if (failed || r.ref == kSentinel) {
                state = kWaitShade;
                failed = false;
            }
        }
    }
}

inline unsigned grid_for(uint64_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

// The flow stages of a step (a chain's candidate lives in x when its parity
// byte is 1, else in y).  Before the path kernel: y = T^{-1}(z) and u(y) of
// the flow draws.  After it: u(y) of the rows the path kernel queued.
cudaError_t launch_flow_draws(const ChainView& c, cudaStream_t st) {
    return launch_flow(c.flow, true, c.x, c.wf.y, c.wf.par, c.n, c.wf.fq + c.n, c.wf.qcount + kQFlowSample, 0,
                       c.wf.uy, nullptr, c.wf.fy, c.status, st, true);
}
cudaError_t launch_flow_densities(const ChainView& c, cudaStream_t st) {
    return launch_flow(c.flow, false, c.x, c.wf.y, c.wf.par, c.n, c.wf.fq, c.wf.qcount + kQFlowDensity, 0,
                       c.wf.uy, nullptr, nullptr, c.status, st, true);
}

}  // namespace

cudaError_t KernelTimer::mark(int k, cudaStream_t st) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    kind.push_back(k);
    return cudaEventRecord(e, st);
}

cudaError_t KernelTimer::totals(double ms[kKinds], uint64_t launches[kKinds]) const {
    for (int k = 0; k < kKinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (size_t i = 1; i < ev.size(); ++i) {
        float t = 0.f;
        cudaError_t r = cudaEventElapsedTime(&t, ev[i - 1], ev[i]);
        if (r != cudaSuccess) return r;
        if (kind[i] >= 0 && kind[i] < kKinds) {
            ms[kind[i]] += t;
            launches[kind[i]] += 1;
        }
    }
    return cudaSuccess;
}

KernelTimer::~KernelTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
}

cudaError_t launch_wavefront(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                             cudaStream_t st, int mode, KernelTimer* tm) {
    static DeviceOnce once;  // per device: the path kernel's persistent grid
    long long path_blocks = 0;
    {
        cudaError_t e0 = once.get(
            [](int dev, long long* v) {
                int sms = 0, per_sm = 0;
                cudaError_t r;
                if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
                    (r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wf_path_kernel, 128, 0)) !=
                        cudaSuccess)
                    return r;
                *v = (long long)sms * (per_sm > 0 ? per_sm : 1);
                return cudaSuccess;
            },
            &path_blocks);
        if (e0 != cudaSuccess) return e0;
    }
    const unsigned G = grid_for(c.n, 128);
    const bool has_flow = c.flow.D != 0;
    cudaError_t e = cudaSuccess;
    auto mark = [&](int kind) {
        if (tm && e == cudaSuccess) e = tm->mark(kind, st);
    };
    mark(-1);
    for (uint32_t k = 0; k < n_steps && e == cudaSuccess; ++k) {
        if ((e = cudaMemsetAsync(c.wf.qcount, 0, sizeof(unsigned int) * kQCount, st)) != cudaSuccess) return e;
        wf_step_kernel<<<G, 128, 0, st>>>(c, step_begin + k, k > 0, 1, mode);
        mark(KernelTimer::kStep);
        if (has_flow && (e = launch_flow_draws(c, st)) != cudaSuccess) return e;
        if (has_flow) mark(KernelTimer::kFlow);
        wf_path_kernel<<<(unsigned)path_blocks, 128, 0, st>>>(s, c, mode != kModeDrain);
        mark(KernelTimer::kPath);
        if (has_flow && (e = launch_flow_densities(c, st)) != cudaSuccess) return e;
        if (has_flow) mark(KernelTimer::kFlow);
    }
    if (e != cudaSuccess) return e;
    wf_step_kernel<<<G, 128, 0, st>>>(c, step_begin + n_steps, n_steps > 0, 0, mode);
    mark(KernelTimer::kStep);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_rebase_scene(Bvh4Node* nodes, uint32_t n_nodes, TriRecord* tris, uint32_t n_tris, int node_off,
                                int tri_off, int mat_off, cudaStream_t st) {
    const uint32_t n = n_nodes > n_tris ? n_nodes : n_tris;
    if (n == 0) return cudaSuccess;
    rebase_scene_kernel<<<grid_for(n, 256), 256, 0, st>>>(nodes, n_nodes, tris, n_tris, node_off, tri_off, mat_off);
    return cudaGetLastError();
}

cudaError_t batch_wavefront_grid(long long* blocks) {
    static DeviceOnce once;  // per device: the batched path kernel's persistent grid
    return once.get(
        [](int dev, long long* v) {
            int sms = 0, per_sm = 0;
            cudaError_t r;
            if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
                (r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wf_batch_path_kernel, 128,
                                                                   sizeof(uint64_t) * (kBatchMaxSets + 1))) !=
                    cudaSuccess)
                return r;
            *v = (long long)sms * (per_sm > 0 ? per_sm : 1);
            return cudaSuccess;
        },
        blocks);
}

cudaError_t launch_batch_wavefront(const BatchWave& bw, BatchEntry* entries, uint32_t n_steps,
                                   const std::vector<ChainView>& flow_sets, cudaStream_t st) {
    long long blocks = 0;
    cudaError_t e = batch_wavefront_grid(&blocks);
    if (e != cudaSuccess) return e;
    if (bw.n_items == 0) return cudaSuccess;
    if (bw.n_sets == 0 || bw.n_sets > kBatchMaxSets) return cudaErrorInvalidValue;
    const size_t shm = sizeof(uint64_t) * (bw.n_sets + 1);
    for (uint32_t k = 0; k < n_steps; ++k) {
        if ((e = cudaMemsetAsync(bw.fetch, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
        for (const ChainView& c : flow_sets)  // the sets' flow queues start empty
            if ((e = cudaMemsetAsync(c.wf.qcount + kQFlowDensity, 0, 2 * sizeof(unsigned int), st)) != cudaSuccess)
                return e;
        wf_batch_step_kernel<<<bw.n_items, 128, 0, st>>>(entries, bw.items, k, k > 0, 1);
        for (const ChainView& c : flow_sets)  // y = T^{-1}(z) and u(y) of the flow draws
            if ((e = launch_flow_draws(c, st)) != cudaSuccess) return e;
        wf_batch_path_kernel<<<(unsigned)blocks, 128, shm, st>>>(bw.merged, entries, bw.roots, bw.chain_off,
                                                                 bw.n_sets, bw.fetch);
        for (const ChainView& c : flow_sets)  // u(y) of the candidates that become states with p > 0
            if ((e = launch_flow_densities(c, st)) != cudaSuccess) return e;
    }
    wf_batch_step_kernel<<<bw.n_items, 128, 0, st>>>(entries, bw.items, n_steps, n_steps > 0, 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed-size scratch for jr_advance_static: the wavefront buffers of up to
// kStaticMaxChains chains live in one file-scope device array instead of
// memory allocated per chain set.  The array belongs to this file's module,
// which the CUDA runtime loads on a device on first use (lazy loading), and
// loading it allocates the array.  jr_chains_create therefore looks the
// address up (prepare_static_scratch), so the module is loaded, and the array
// allocated, where allocation is allowed; a device keeps it until the process
// exits.  Layout (256-byte aligned pieces): y [kMaxDim][n],
// fy [n] float4, ua [n], queue [n], par [n], qcount (256 bytes).
namespace {
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffY = 0;
constexpr size_t kOffFy = kOffY + align256(sizeof(float) * kMaxDim * kStaticMaxChains);
constexpr size_t kOffUa = kOffFy + align256(sizeof(float4) * kStaticMaxChains);
constexpr size_t kOffQueue = kOffUa + align256(sizeof(float) * kStaticMaxChains);
constexpr size_t kOffPar = kOffQueue + align256(sizeof(uint32_t) * kStaticMaxChains);
constexpr size_t kOffCount = kOffPar + align256(sizeof(uint8_t) * kStaticMaxChains);
constexpr size_t kStaticBytes = kOffCount + align256(sizeof(unsigned int) * kQCount);
static_assert(sizeof(unsigned int) * kQCount <= 256, "the static counters fit their 256 bytes");
static_assert(kStaticBytes == kStaticScratchBytes, "static scratch layout and its declared size disagree");

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_base[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (host code only sees a host-side stand-in for the symbol).
cudaError_t static_scratch_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_base[dev] = p;
    }
    *out = g_static_base[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t prepare_static_scratch() {
    void* base = nullptr;
    return static_scratch_base(&base);
}

cudaError_t launch_wavefront_static(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                                    cudaStream_t st) {
    if (c.n > kStaticMaxChains || c.dim > (uint32_t)kMaxDim) return cudaErrorInvalidValue;
    void* base = nullptr;
    cudaError_t e = static_scratch_base(&base);
    if (e != cudaSuccess) return e;
    unsigned char* b = static_cast<unsigned char*>(base);
    ChainView v = c;
    v.wf.y = reinterpret_cast<float*>(b + kOffY);
    v.wf.fy = reinterpret_cast<float4*>(b + kOffFy);
    v.wf.ua = reinterpret_cast<float*>(b + kOffUa);
    v.wf.queue = reinterpret_cast<uint32_t*>(b + kOffQueue);
    v.wf.par = b + kOffPar;
    v.wf.qcount = reinterpret_cast<unsigned int*>(b + kOffCount);
    // The array keeps the previous call's bytes: the parity must start at 0
    // (every state in x); the queue counters are cleared per step inside
    // launch_wavefront; y, ua and fy are written before use.
    if ((e = cudaMemsetAsync(v.wf.par, 0, c.n, st)) != cudaSuccess) return e;
    return launch_wavefront(s, v, step_begin, n_steps, st);
}

}  // namespace jr
