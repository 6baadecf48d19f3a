// Inference of the regeneration flow (density and sampling directions) on the
// tensor cores, sm_103a.
//
// The flow is the library's own regeneration distribution (not in the paper):
// mu = beta mu_flow + (1 - beta) uniform, u = beta q + (1 - beta), so that the
// killing rate k = c~ u / p of Section 6.2 keeps an exact density.  L = 6
// coupling layers, each an MLP (A -> 64 -> 64 -> A K logits, ReLU) feeding
// piecewise-linear CDFs of K = 16 bins (Mueller et al., "Neural Importance
// Sampling", 2019): bin masses Q = (1 - E) softmax(o) + E / K, density factor
// K Q[bin].
//
// Design:
//   * A CTA of 8 warps works on tiles of 128 rows, 16 rows per warp; the rows of
//     a warp never leave it.  The three GEMMs of a layer run as mma.sync
//     m16n8k16 (bf16 operands, FP32 accumulation) and stay in registers: the
//     accumulator fragments of one GEMM, biased, ReLU'd and rounded to bf16, are
//     the A fragments of the next.
//   * The biased logits of two coordinates at a time go through a per-warp
//     shared tile, so that each lane owns one (row, coordinate) pair with all
//     16 bins in registers: softmax, cumulative masses and bin search run
//     sequentially in the lane, with no shuffles.
//   * Weights stream through shared memory one layer at a time, in one
//     buffer: once every warp is done with a layer, one elected thread copies
//     the next layer's block (bf16 weights in a bank-conflict-free
//     XOR-swizzled layout, then the FP32 biases) with one cp.async.bulk; an
//     mbarrier counts the bytes in.  One buffer (about 65 KB per CTA at D = 22)
//     lets three CTAs share an SM, 24 warps to hide the softmax chains'
//     latency, where two buffers allowed two CTAs; the other CTAs run while
//     one waits for its copy (measured at D = 22 and 26: -5 to -8 % per row
//     from 2^16 rows up, within +3 % below).  Every wait is bounded; a wait
//     that runs out sets JR_STATUS_FLOW_WAIT and the kernel stops after its
//     copy has landed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jr.h"
#include "jr_device.cuh"
#include "jr_internal.h"

namespace jr {
namespace {

constexpr int kWarps = 8;
constexpr int kTile = 16 * kWarps;  // rows per CTA tile
constexpr int kThreads = 32 * kWarps;
constexpr uint32_t kNoRow = 0xffffffffu;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s
constexpr uint32_t kWaitIters = 1u << 26;

// Shared-memory layout (bytes): two mbarriers, perm [kFL][D], row ids
// [kTile], the rows' states [kTile][D + 1] FP32, per warp a logits tile
// [16][kLgStride] FP32 (two coordinates' 32 logits per row), one layer buffer
// (bar[0] counts its copies).
constexpr int kLgStride = 36;  // conflict-free 16-byte row reads by quarter warps
constexpr size_t kOffBar = 0, kOffPerm = 64, kOffRows = 256, kOffX = kOffRows + 4 * kTile;
constexpr size_t kLgBytes = sizeof(float) * kWarps * 16 * kLgStride;
__host__ __device__ constexpr size_t round128(size_t b) { return (b + 127) & ~(size_t)127; }
__host__ __device__ constexpr size_t x_bytes(uint32_t D) { return round128(sizeof(float) * kTile * (D + 1)); }
__host__ __device__ constexpr size_t buf_bytes(uint32_t AK) { return round128(flow_ws_layer_bytes(AK)); }
__host__ __device__ constexpr size_t infer_smem(uint32_t D, uint32_t AK) {
    return round128(kOffX) + x_bytes(D) + round128(kLgBytes) + buf_bytes(AK);
}
static_assert(kOffPerm + kFL * kMaxDim <= kOffRows, "perm table overlaps the row ids");

constexpr float kLog2e = 1.4426950408889634f;
// 2^x with the hardware's base-2 exponential (PTX ex2.approx).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of bar; false when the time or iteration budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0; it < kWaitIters; ++it) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(32);
        if ((it & 255) == 255 && globaltimer() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragments of two n-tiles (rows n0 .. n0 + 15) at k = k0 .. k0 + 15 of a
// swizzled [N][64] bf16 matrix, with one ldmatrix.x4: lanes 0-7 address the
// rows n0 + 0..7 at k-chunk k0/8, lanes 8-15 the same rows at chunk k0/8 + 1,
// lanes 16-31 rows n0 + 8..15 likewise.  Fragment (b[0], b[1]) is n-tile n0,
// (b[2], b[3]) n-tile n0 + 8.
__device__ __forceinline__ void frag_b64x2(const __nv_bfloat16* W, int n0, int k0, uint32_t (&b)[4]) {
    const int lane = threadIdx.x & 31;
    const int n = n0 + (lane & 7) + ((lane >> 4) << 3);
    const int c = (k0 >> 3) + ((lane >> 3) & 1);
    const __nv_bfloat16* p = W + n * 64 + ((c ^ (n & 7)) << 3);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"(smem_addr(p)));
}
// The same for the [64][16] W1 (one k-step; chunk c of row n at c ^ ((n >> 2) & 1)).
__device__ __forceinline__ void frag_b16x2(const __nv_bfloat16* W, int n0, uint32_t (&b)[4]) {
    const int lane = threadIdx.x & 31;
    const int n = n0 + (lane & 7) + ((lane >> 4) << 3);
    const int c = (lane >> 3) & 1;
    const __nv_bfloat16* p = W + n * 16 + ((c ^ ((n >> 2) & 1)) << 3);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"(smem_addr(p)));
}

// ReLU(acc + b) of 8 n-tiles (64 columns) as bf16 A fragments of a K = 64 GEMM.
__device__ __forceinline__ void relu_to_frags(const float (&acc)[8][4], const float* bias, int t, uint32_t (&a)[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        const float b00 = bias[c0], b01 = bias[c0 + 1], b10 = bias[c1], b11 = bias[c1 + 1];
        a[kk][0] = pack_bf16(fmaxf(acc[2 * kk][0] + b00, 0.f), fmaxf(acc[2 * kk][1] + b01, 0.f));
        a[kk][1] = pack_bf16(fmaxf(acc[2 * kk][2] + b00, 0.f), fmaxf(acc[2 * kk][3] + b01, 0.f));
        a[kk][2] = pack_bf16(fmaxf(acc[2 * kk + 1][0] + b10, 0.f), fmaxf(acc[2 * kk + 1][1] + b11, 0.f));
        a[kk][3] = pack_bf16(fmaxf(acc[2 * kk + 1][2] + b10, 0.f), fmaxf(acc[2 * kk + 1][3] + b11, 0.f));
    }
}

// One coordinate's CDF step for one row, all 16 bins in this lane.  L: the
// logits in base 2 (log2 e times the network's output: the layer's bias is
// stored scaled and the accumulator is scaled in the same FMA), so the softmax
// e_k = 2^(L_k - max L) = exp(l_k - max l) takes one ex2 per bin (base-2
// softmax, as in FlashAttention-2, Dao 2023; measured -3.6 % per density row).
// density: v = t in [0,1) becomes CDF(t); sampling: v = c becomes
// CDF^{-1}(c).  Returns log(K Q[bin]).  With S = sum e, Q_k = sc e_k + E/K,
// sc = (1 - E)/S.
template <bool kSample>
__device__ __forceinline__ float cdf_row(const float (&L)[kFK], float& v) {
    float m = fmax3(fmax3(L[0], L[1], L[2]), fmax3(L[3], L[4], L[5]), fmax3(L[6], L[7], L[8]));
    m = fmax3(m, fmax3(L[9], L[10], L[11]), fmax3(L[12], L[13], fmaxf(L[14], L[15])));
    float e[kFK];
#pragma unroll
    for (int k = 0; k < kFK; ++k) e[k] = exp2_approx(L[k] - m);
    float s4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) s4[k] = (e[4 * k] + e[4 * k + 1]) + (e[4 * k + 2] + e[4 * k + 3]);
    const float S = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    const float sc = __fdividef(1.0f - kFE, S);  // S in [1, 16]
    int b;
    if (!kSample) {
        b = min((int)(v * (float)kFK), kFK - 1);
    } else {
        float cum = 0.f;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kFK; ++k) {
            cum += fmaf(e[k], sc, kFE / kFK);
            cnt += cum <= v;
        }
        b = min(cnt, kFK - 1);
    }
    float lo_e = 0.f, qb_e = 0.f;
#pragma unroll
    for (int k = 0; k < kFK; ++k) {
        lo_e += k < b ? e[k] : 0.f;
        qb_e = k == b ? e[k] : qb_e;
    }
    const float lo = fmaf(sc, lo_e, (float)b * (kFE / kFK));
    const float qb = fmaf(sc, qb_e, kFE / kFK);
    if (!kSample) {
        v = lo + (v * (float)kFK - (float)b) * qb;
    } else {
        const float xs = ((float)b + (v - lo) / qb) * (1.0f / (float)kFK);
        v = fminf(fmaxf(xs, 0.0f), 0.99999994f);
    }
    return __logf((float)kFK * qb);
}

// One coupling layer for this warp's 16 rows (xw: [16][xs] FP32 states; pm:
// the layer's permutation; wl: the layer's block in shared memory).
template <bool kSample>
__device__ __forceinline__ void coupling(const unsigned char* wl, const uint8_t* pm, int A, int AK, float* xw, int xs,
                                         float* lg, float& lqp) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(wl);
    const __nv_bfloat16* W2 = W1 + kFH * kFAP;
    const __nv_bfloat16* W3 = W2 + kFH * kFH;
    const float* b1 = reinterpret_cast<const float*>(W3 + (size_t)AK * kFH);
    const float* b2 = b1 + kFH;
    const float* b3 = b2 + kFH;
    uint32_t a[4][4];
    {   // layer 1: K = 16 (the A conditioning coordinates, zero-padded)
        auto xa = [&](int r, int c) { return c < A ? xw[r * xs + pm[c]] : 0.f; };
        uint32_t a0[4] = {pack_bf16(xa(g, 2 * t), xa(g, 2 * t + 1)), pack_bf16(xa(g + 8, 2 * t), xa(g + 8, 2 * t + 1)),
                          pack_bf16(xa(g, 2 * t + 8), xa(g, 2 * t + 9)),
                          pack_bf16(xa(g + 8, 2 * t + 8), xa(g + 8, 2 * t + 9))};
        float acc[8][4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
            acc[q + 1][0] = acc[q + 1][1] = acc[q + 1][2] = acc[q + 1][3] = 0.f;
            uint32_t b[4];
            frag_b16x2(W1, 8 * q, b);
            mma(acc[q], a0, b[0], b[1]);
            mma(acc[q + 1], a0, b[2], b[3]);
        }
        relu_to_frags(acc, b1, t, a);
    }
    {   // layer 2: 64 -> 64
        float acc[8][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                uint32_t b[4];
                frag_b64x2(W2, 8 * q, 16 * kk, b);
                mma(acc[q], a[kk], b[0], b[1]);
                mma(acc[q + 1], a[kk], b[2], b[3]);
            }
        relu_to_frags(acc, b2, t, a);
    }
    // layer 3 and the couplings, 2 coordinates (4 n-tiles of logits) at a time:
    // the biased logits go through the warp's shared tile so that lane
    // (r = lane & 15, jj = lane >> 4) owns coordinate j0 + jj of row r
    const int r = lane & 15, jj = lane >> 4;
    for (int j0 = 0; j0 < A; j0 += 2) {
        const int nq = min(4, 2 * (A - j0));  // 2 or 4 n-tiles (warp-uniform)
        float acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int q = 0; q < 4; q += 2)
                if (q < nq) {
                    uint32_t b[4];
                    frag_b64x2(W3, 16 * j0 + 8 * q, 16 * kk, b);
                    mma(acc[q], a[kk], b[0], b[1]);
                    mma(acc[q + 1], a[kk], b[2], b[3]);
                }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < nq) {
                const int c = 8 * q + 2 * t;
                const float2 bb = *reinterpret_cast<const float2*>(b3 + 16 * j0 + c);
                *reinterpret_cast<float2*>(lg + g * kLgStride + c) =
                    make_float2(fmaf(acc[q][0], kLog2e, bb.x), fmaf(acc[q][1], kLog2e, bb.y));
                *reinterpret_cast<float2*>(lg + (g + 8) * kLgStride + c) =
                    make_float2(fmaf(acc[q][2], kLog2e, bb.x), fmaf(acc[q][3], kLog2e, bb.y));
            }
        __syncwarp();
        if (2 * jj < nq) {
            float L[kFK];
            const float4* src = reinterpret_cast<const float4*>(lg + r * kLgStride + 16 * jj);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 q4 = src[k];
                L[4 * k] = q4.x;
                L[4 * k + 1] = q4.y;
                L[4 * k + 2] = q4.z;
                L[4 * k + 3] = q4.w;
            }
            const int cb = pm[A + j0 + jj];
            float vv = xw[r * xs + cb];
            lqp += cdf_row<kSample>(L, vv);
            xw[r * xs + cb] = vv;
        }
        __syncwarp();
    }
}

// Rows: chains idx[j] (or j when idx is null) for j < *count_dev (or n_rows).
// A row lives in buffer bufA, or -- when par is given -- in bufA if par[i] is
// 1 and bufB otherwise; pairs = 1: the chain state's pair layout (xidx), else
// SoA [D][n].  Density: u_out[i] = beta q + 1 - beta,
// lq_out[i] = log q.  Sample: the row is replaced by T^{-1}(row), u_out and
// lq_out as above, and start[i] (if given) = the new row's first four
// coordinates.
template <bool kSample>
__global__ void __launch_bounds__(kThreads) flow_infer_kernel(FlowView f, float* bufA, float* bufB,
                                                              const uint8_t* par, uint64_t n, const uint32_t* idx,
                                                              const unsigned int* count_dev, uint32_t n_rows,
                                                              float* u_out, float* lq_out, float4* start,
                                                              unsigned int* status, int pairs) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint8_t* perm_s = smem + kOffPerm;
    uint32_t* rows = reinterpret_cast<uint32_t*>(smem + kOffRows);
    float* xt = reinterpret_cast<float*>(smem + round128(kOffX));
    const int D = (int)f.D, A = (int)f.A, AK = (int)f.AK, xs = D + 1;
    float* lgt = reinterpret_cast<float*>(smem + round128(kOffX) + x_bytes(f.D));
    unsigned char* wbuf0 = smem + round128(kOffX) + x_bytes(f.D) + round128(kLgBytes);
    const uint32_t lbytes = (uint32_t)flow_ws_layer_bytes(f.AK);

    const uint32_t count = count_dev ? *count_dev : n_rows;
    const uint32_t first = blockIdx.x * kTile;
    if (first >= count) return;
    const uint32_t stride = gridDim.x * kTile;
    const uint32_t my_tiles = (count - first + stride - 1) / stride;
    const uint32_t total = my_tiles * kFL;  // layer applications of this CTA
    auto layer_of = [&](uint32_t st) { return kSample ? kFL - 1 - (int)(st % kFL) : (int)(st % kFL); };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_fence_init();
    }
    for (int e = threadIdx.x; e < kFL * D; e += blockDim.x) perm_s[e] = f.perm[e];
    __syncthreads();
    if (threadIdx.x == 0 && total > 0) {  // the first layer's weights
        mbar_expect(&bar[0], lbytes + f.extra_tx);
        bulk_load(wbuf0, f.ws + (size_t)layer_of(0) * lbytes, lbytes, &bar[0]);
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* xw = xt + warp * 16 * xs;
    float* lg = lgt + warp * 16 * kLgStride;
    auto row_buf = [&](uint32_t i) -> float* { return (par && !par[i]) ? bufB : bufA; };
    float lqp = 0.f;  // this lane's part of log q of row lane & 15
    bool failed = false;

    uint32_t st = 0;
    for (; st < total; ++st) {
        const uint32_t tile0 = first + (st / kFL) * stride + warp * 16;  // this warp's first row
        if (st % kFL == 0) {  // load the warp's rows
            if (lane < 16) {
                const uint32_t j = tile0 + lane;
                rows[warp * 16 + lane] = j < count ? (idx ? idx[j] : j) : kNoRow;
            }
            __syncwarp();
            for (int e = lane; e < 16 * D; e += 32) {
                const int r = e / D, d = e % D;
                const uint32_t i = rows[warp * 16 + r];
                xw[r * xs + d] = i != kNoRow ? row_buf(i)[pairs ? xidx(d, i, n) : (uint64_t)d * n + i] : 0.5f;
            }
            lqp = 0.f;
            __syncwarp();
        }
        failed = !mbar_wait(&bar[0], st & 1);  // layer application st: the barrier's phase st
        if (!failed) {
            const int l = layer_of(st);
            coupling<kSample>(wbuf0, perm_s + l * D, A, AK, xw, xs, lg, lqp);
        }
        if (__syncthreads_or(failed)) break;  // every warp is done with the buffer
        if (threadIdx.x == 0 && st + 1 < total) {
            mbar_expect(&bar[0], lbytes);
            bulk_load(wbuf0, f.ws + (size_t)layer_of(st + 1) * lbytes, lbytes, &bar[0]);
        }
        if (st % kFL == kFL - 1) {  // write the warp's rows
            const float lq = lqp + __shfl_xor_sync(0xffffffffu, lqp, 16);  // row lane & 15
            if (kSample)
                for (int e = lane; e < 16 * D; e += 32) {
                    const int r = e / D, d = e % D;
                    const uint32_t i = rows[warp * 16 + r];
                    if (i != kNoRow) row_buf(i)[pairs ? xidx(d, i, n) : (uint64_t)d * n + i] = xw[r * xs + d];
                }
            if (lane < 16) {
                const int r = lane;
                const uint32_t i = rows[warp * 16 + r];
                if (i != kNoRow) {
                    if (u_out) u_out[i] = f.beta * __expf(lq) + (1.0f - f.beta);
                    if (lq_out) lq_out[i] = lq;
                    if (kSample && start) {
                        const float* x = xw + r * xs;
                        start[i] = make_float4(x[0], D > 1 ? x[1] : 0.f, D > 2 ? x[2] : 0.f, D > 3 ? x[3] : 0.f);
                    }
                }
            }
            __syncwarp();
        }
    }
    if (st < total && threadIdx.x == 0) {
        // A wait ran out: flag it, then let the copy already issued land
        // (bounded) before the CTA's shared memory goes away.
        if (status) atomicOr(status, JR_STATUS_FLOW_WAIT);
        (void)mbar_wait(&bar[0], st & 1);
    }
}

// Swizzled inference layout of one layer (see flow_ws_layer_bytes).
__global__ void pack_ws_kernel(const float* master, unsigned char* ws, uint32_t AK) {
    const int l = blockIdx.y;
    const size_t S = (size_t)kFH * kFAP + kFH + kFH * kFH + kFH + (size_t)AK * kFH + AK;
    const float* m = master + l * S;
    unsigned char* blk = ws + (size_t)l * flow_ws_layer_bytes(AK);
    __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(blk);
    __nv_bfloat16* W2 = W1 + kFH * kFAP;
    __nv_bfloat16* W3 = W2 + kFH * kFH;
    float* b = reinterpret_cast<float*>(W3 + (size_t)AK * kFH);
    const float* m1 = m;
    const float* mb1 = m1 + kFH * kFAP;
    const float* m2 = mb1 + kFH;
    const float* mb2 = m2 + kFH * kFH;
    const float* m3 = mb2 + kFH;
    const float* mb3 = m3 + (size_t)AK * kFH;
    const uint32_t n1 = kFH * kFAP, n2 = kFH * kFH, n3 = AK * kFH;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2 + n3 + 2 * kFH + AK;
         e += gridDim.x * blockDim.x) {
        if (e < n1) {
            const uint32_t r = e / kFAP, k = e % kFAP;
            W1[r * kFAP + ((((k >> 3) ^ ((r >> 2) & 1)) << 3) | (k & 7))] = __float2bfloat16_rn(m1[e]);
        } else if (e < n1 + n2) {
            const uint32_t q = e - n1, r = q / kFH, k = q % kFH;
            W2[r * kFH + ((((k >> 3) ^ (r & 7)) << 3) | (k & 7))] = __float2bfloat16_rn(m2[q]);
        } else if (e < n1 + n2 + n3) {
            const uint32_t q = e - n1 - n2, r = q / kFH, k = q % kFH;
            W3[r * kFH + ((((k >> 3) ^ (r & 7)) << 3) | (k & 7))] = __float2bfloat16_rn(m3[q]);
        } else {
            const uint32_t q = e - n1 - n2 - n3;
            b[q] = q < (uint32_t)kFH ? mb1[q] : q < (uint32_t)(2 * kFH) ? mb2[q - kFH] : mb3[q - 2 * kFH] * kLog2e;
        }
    }
}

}  // namespace

cudaError_t launch_flow_pack_ws(const float* master, unsigned char* ws, uint32_t AK, cudaStream_t st) {
    pack_ws_kernel<<<dim3(16, kFL), 256, 0, st>>>(master, ws, AK);
    return cudaGetLastError();
}

cudaError_t launch_flow(const FlowView& f, bool sample, float* bufA, float* bufB, const uint8_t* par, uint64_t n,
                        const uint32_t* idx, const unsigned int* count_dev, uint32_t n_rows, float* u_out,
                        float* lq_out, float4* start, unsigned int* status, cudaStream_t st, bool pairs) {
    static DeviceOnce once;  // per device: the SM count, after opting in to the largest layout
    const size_t shm = infer_smem(f.D, f.AK);
    long long sms = 0;
    cudaError_t e = once.get(
        [](int dev, long long* v) {
            const int most = (int)infer_smem(kMaxDim, kFMaxAK);
            int n = 0;
            cudaError_t r;
            if ((r = cudaFuncSetAttribute(flow_infer_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          most)) != cudaSuccess ||
                (r = cudaFuncSetAttribute(flow_infer_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          most)) != cudaSuccess ||
                (r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return r;
            *v = n;
            return cudaSuccess;
        },
        &sms);
    if (e != cudaSuccess) return e;
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, flow_infer_kernel<false>, kThreads, shm)) !=
        cudaSuccess)
        return e;
    unsigned g = (unsigned)(sms * (per > 0 ? per : 1));
    if (!count_dev) g = (unsigned)std::min<uint64_t>(g, (n_rows + kTile - 1) / kTile);
    if (g == 0) return cudaSuccess;
    if (sample)
        flow_infer_kernel<true><<<g, kThreads, shm, st>>>(f, bufA, bufB, par, n, idx, count_dev, n_rows, u_out,
                                                          lq_out, start, status, pairs ? 1 : 0);
    else
        flow_infer_kernel<false><<<g, kThreads, shm, st>>>(f, bufA, bufB, par, n, idx, count_dev, n_rows, u_out,
                                                           lq_out, nullptr, status, pairs ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace jr
