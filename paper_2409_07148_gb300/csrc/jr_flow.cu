// The learned regeneration flow on the tensor cores (sm_103a).
//
// Not in the paper: the library's own regeneration distribution
//   mu = beta mu_flow + (1 - beta) uniform,   u = beta q + (1 - beta),
// so the killing rate k = c~ u / p (Section 6.2) keeps an exact density.  The
// flow has L coupling layers on [0,1)^D; layer l conditions on x[perm[l][:A]]
// (A = D/2) and moves each x[perm[l][A + j]] through a piecewise-linear CDF of
// K bins whose masses come from an MLP (2 hidden layers of 64, ReLU):
//   Q_j = (1 - E) softmax(o_j) + E / K,  density factor K Q_j[bin],
// the piecewise-linear coupling of Mueller et al. ("Neural Importance
// Sampling", 2019).  The MLP GEMMs run as mma.sync m16n8k16 with bf16
// operands and FP32 accumulation; everything else is FP32.
//
// This file holds the training side (forward with stored layer inputs,
// backward, Adam, parameter packing, training rows from the chains); the
// inference kernels are in jr_flow_infer.cu.  The forward pass here works on
// tiles of 64 rows (4 warps x 16 rows) per CTA of 128 threads: per layer it
// stages the bf16 weights in shared memory; each warp runs the three GEMMs of
// its 16 rows; the 64-column chunks of logits go through shared memory to the
// per-coordinate softmax / bin / CDF step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jr.h"
#include "jr_device.cuh"
#include "jr_internal.h"

namespace jr {
namespace {

constexpr int kRows = 64;                 // rows per tile
constexpr int kXs = 33;                   // row stride of the state tile (floats)
constexpr int kLs = 65;                   // row stride of the logits chunk (floats)

struct FlowSmem {
    float x[kRows * kXs];
    float lq[kRows];
    float lg[kRows * kLs];
    float b1[kFH], b2[kFH], b3[kFMaxAK];
    uint32_t row_idx[kRows];
    __nv_bfloat16 xa[kRows * kFS1];
    __nv_bfloat16 h1[kRows * kFS2];
    __nv_bfloat16 h2[kRows * kFS2];
    __nv_bfloat16 w1[kFH * kFS1];
    __nv_bfloat16 w2[kFH * kFS2];
    __nv_bfloat16 w3[kFMaxAK * kFS2];
};

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D[16x8] += A[16x16] (row-major) * B[16x8] (col-major), bf16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// out[16 x (8 nt)] for this warp's 16 rows: in [rows][kin] (row stride sin) times
// W^T with W [N][kin] (row stride sw), n-tiles n0 .. n0 + nt.
template <int kNT>
__device__ __forceinline__ void warp_gemm(float (&acc)[kNT][4], const __nv_bfloat16* in, int sin, int row0,
                                          const __nv_bfloat16* W, int sw, int n0, int kin, int nt_valid) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int q = 0; q < kNT; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    for (int k0 = 0; k0 < kin; k0 += 16) {
        const __nv_bfloat16* ar = in + (row0 + g) * sin + k0 + 2 * t;
        const uint32_t a0 = ld_b32(ar), a1 = ld_b32(ar + 8 * sin), a2 = ld_b32(ar + 8), a3 = ld_b32(ar + 8 * sin + 8);
#pragma unroll
        for (int q = 0; q < kNT; ++q) {
            if (q < nt_valid) {
                const __nv_bfloat16* br = W + (n0 + 8 * q + g) * sw + k0 + 2 * t;
                mma_bf16(acc[q], a0, a1, a2, a3, ld_b32(br), ld_b32(br + 8));
            }
        }
    }
}

__device__ __forceinline__ const __nv_bfloat16* layer_w(const FlowView& f, int l) {
    return f.wb + (size_t)l * (kFH * kFS1 + kFH * kFS2 + (size_t)f.AK * kFS2);
}
__device__ __forceinline__ const float* layer_b(const FlowView& f, int l) {
    return f.bias + (size_t)l * (2 * kFH + f.AK);
}

// Stage the bf16 weights and FP32 biases of layer l (16-byte copies).
__device__ __forceinline__ void load_layer(const FlowView& f, int l, FlowSmem& sm) {
    const __nv_bfloat16* w = layer_w(f, l);
    const int n1 = kFH * kFS1, n2 = kFH * kFS2, n3 = f.AK * kFS2;
    const uint4* src = reinterpret_cast<const uint4*>(w);
    for (int e = threadIdx.x; e < n1 / 8; e += blockDim.x) reinterpret_cast<uint4*>(sm.w1)[e] = src[e];
    src = reinterpret_cast<const uint4*>(w + n1);
    for (int e = threadIdx.x; e < n2 / 8; e += blockDim.x) reinterpret_cast<uint4*>(sm.w2)[e] = src[e];
    src = reinterpret_cast<const uint4*>(w + n1 + n2);
    for (int e = threadIdx.x; e < n3 / 8; e += blockDim.x) reinterpret_cast<uint4*>(sm.w3)[e] = src[e];
    const float* b = layer_b(f, l);
    for (int e = threadIdx.x; e < 2 * kFH + f.AK; e += blockDim.x) {
        const float v = b[e];
        if (e < kFH) sm.b1[e] = v;
        else if (e < 2 * kFH) sm.b2[e - kFH] = v;
        else sm.b3[e - 2 * kFH] = v;
    }
}

// Softmax bin masses of coordinate chunk column c0 (16 logits) of row r.
__device__ __forceinline__ void bin_masses(const float* lg, float (&Q)[kFK]) {
    float m = lg[0];
#pragma unroll
    for (int k = 1; k < kFK; ++k) m = fmaxf(m, lg[k]);
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < kFK; ++k) {
        Q[k] = __expf(lg[k] - m);
        S += Q[k];
    }
    const float sc = (1.0f - kFE) / S;
#pragma unroll
    for (int k = 0; k < kFK; ++k) Q[k] = Q[k] * sc + kFE / kFK;
}

// One coupling layer on this CTA's tile (all threads call).
template <bool kSample>
__device__ __forceinline__ void coupling_layer(const FlowView& f, int l, FlowSmem& sm) {
    const int A = (int)f.A, D = (int)f.D;
    const uint8_t* pm = f.perm + l * D;
    __syncthreads();
    load_layer(f, l, sm);
    for (int e = threadIdx.x; e < kRows * kFAP; e += blockDim.x) {
        const int r = e / kFAP, c = e % kFAP;
        sm.xa[r * kFS1 + c] = __float2bfloat16_rn(c < A ? sm.x[r * kXs + pm[c]] : 0.0f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row0 = 16 * warp;
    {   // h1 = relu(W1 xa + b1)
        float acc[8][4];
        warp_gemm<8>(acc, sm.xa, kFS1, row0, sm.w1, kFS1, 0, kFAP, 8);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = 8 * q + 2 * t;
            __nv_bfloat16* o0 = sm.h1 + (row0 + g) * kFS2 + c;
            __nv_bfloat16* o1 = sm.h1 + (row0 + g + 8) * kFS2 + c;
            o0[0] = __float2bfloat16_rn(fmaxf(acc[q][0] + sm.b1[c], 0.f));
            o0[1] = __float2bfloat16_rn(fmaxf(acc[q][1] + sm.b1[c + 1], 0.f));
            o1[0] = __float2bfloat16_rn(fmaxf(acc[q][2] + sm.b1[c], 0.f));
            o1[1] = __float2bfloat16_rn(fmaxf(acc[q][3] + sm.b1[c + 1], 0.f));
        }
    }
    __syncwarp();
    {   // h2 = relu(W2 h1 + b2)
        float acc[8][4];
        warp_gemm<8>(acc, sm.h1, kFS2, row0, sm.w2, kFS2, 0, kFH, 8);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = 8 * q + 2 * t;
            __nv_bfloat16* o0 = sm.h2 + (row0 + g) * kFS2 + c;
            __nv_bfloat16* o1 = sm.h2 + (row0 + g + 8) * kFS2 + c;
            o0[0] = __float2bfloat16_rn(fmaxf(acc[q][0] + sm.b2[c], 0.f));
            o0[1] = __float2bfloat16_rn(fmaxf(acc[q][1] + sm.b2[c + 1], 0.f));
            o1[0] = __float2bfloat16_rn(fmaxf(acc[q][2] + sm.b2[c], 0.f));
            o1[1] = __float2bfloat16_rn(fmaxf(acc[q][3] + sm.b2[c + 1], 0.f));
        }
    }
    __syncwarp();
    // logits o = W3 h2 + b3, 64 columns (4 coordinates) at a time
    for (int c0 = 0; c0 < (int)f.AK; c0 += 64) {
        const int ncol = min(64, (int)f.AK - c0);
        float acc[8][4];
        warp_gemm<8>(acc, sm.h2, kFS2, row0, sm.w3, kFS2, c0, kFH, ncol / 8);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (8 * q < ncol) {
                const int c = 8 * q + 2 * t;
                float* o0 = sm.lg + (row0 + g) * kLs + c;
                float* o1 = sm.lg + (row0 + g + 8) * kLs + c;
                o0[0] = acc[q][0] + sm.b3[c0 + c];
                o0[1] = acc[q][1] + sm.b3[c0 + c + 1];
                o1[0] = acc[q][2] + sm.b3[c0 + c];
                o1[1] = acc[q][3] + sm.b3[c0 + c + 1];
            }
        }
        __syncwarp();
        // lane -> row row0 + (lane & 15), coordinates 2 (lane >> 4) and + 1 of the chunk
        const int r = row0 + (lane & 15);
        float dlq = 0.f;
        for (int jj = 2 * (lane >> 4); jj < 2 * (lane >> 4) + 2; ++jj) {
            if (16 * jj >= ncol) break;
            float Q[kFK];
            bin_masses(sm.lg + r * kLs + 16 * jj, Q);
            const int cb = pm[A + c0 / 16 + jj];
            float* xv = sm.x + r * kXs + cb;
            if (!kSample) {  // density direction: t -> CDF(t)
                const float tt = *xv;
                const int b = min((int)(tt * (float)kFK), kFK - 1);
                float lo = 0.f, qb = Q[0];
#pragma unroll
                for (int k = 0; k < kFK; ++k) {
                    if (k < b) lo += Q[k];
                    if (k == b) qb = Q[k];
                }
                *xv = lo + (tt * (float)kFK - (float)b) * qb;
                dlq += __logf((float)kFK * qb);
            } else {         // sampling direction: c -> CDF^{-1}(c)
                const float cc = *xv;
                float cum = 0.f, lo = 0.f, qb = Q[0];
                int b = 0;
#pragma unroll
                for (int k = 0; k < kFK; ++k) {
                    cum += Q[k];
                    if (cum <= cc) b = k + 1;
                }
                b = min(b, kFK - 1);
#pragma unroll
                for (int k = 0; k < kFK; ++k) {
                    if (k < b) lo += Q[k];
                    if (k == b) qb = Q[k];
                }
                const float xs = ((float)b + (cc - lo) / qb) * (1.0f / (float)kFK);
                *xv = fminf(fmaxf(xs, 0.0f), 0.99999994f);
                dlq += __logf((float)kFK * qb);
            }
        }
        dlq += __shfl_down_sync(0xffffffffu, dlq, 16);
        if (lane < 16) sm.lq[r] += dlq;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Training: the time-weighted maximum-likelihood loss  -sum_r w_r log q(x_r) /
// sum_r w_r  over a minibatch and its gradient w.r.t. the FP32 master
// parameters.  Per tile of 64 rows: a forward pass (density direction) stores
// the state entering every layer; the backward pass goes through the layers in
// reverse, recomputes the layer's MLP from the stored state, and back-propagates
// through the couplings (FP32) and the MLP (tensor cores: activation gradients
// dO W3, dh2 W2, dh1 W1 and weight gradients dO^T h2, dh2^T h1, dh1^T xa, all
// bf16 operands with FP32 accumulation; bf16 roundings of the forward pass
// pass gradients straight through).  Weight gradients go to an FP32 buffer
// with atomics.

constexpr int kSO = kFMaxAK + 8;  // row stride of the logits-gradient tile (bf16)

struct TrainSmem {
    FlowSmem f;
    float stash[kFL][kRows * kXs];  // state entering each layer
    float g[kRows * kXs];           // dL/d(state)
    float s[kRows];                 // dL/d(log q) per row
    __nv_bfloat16 dO[kRows * kSO];  // dL/d(logits)
    __nv_bfloat16 dh2[kRows * kFS2];
    __nv_bfloat16 dh1[kRows * kFS2];
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Warp GEMM with operands at arbitrary strides: A(m, k) = A[m*am + k*ak],
// B(k, n) = B[k*bk + n*bn]; rows m0 .. m0+15, n-tiles n0 + 8q (q < nt_valid).
template <int kNT>
__device__ __forceinline__ void warp_gemm_g(float (&acc)[kNT][4], const __nv_bfloat16* A, int am, int ak, int m0,
                                            const __nv_bfloat16* B, int bk, int bn, int n0, int K, int nt_valid) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int q = 0; q < kNT; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + 2 * t;
        const __nv_bfloat16* r0 = A + (m0 + g) * am;
        const __nv_bfloat16* r1 = A + (m0 + g + 8) * am;
        const uint32_t a0 = pack2(r0[ka * ak], r0[(ka + 1) * ak]);
        const uint32_t a1 = pack2(r1[ka * ak], r1[(ka + 1) * ak]);
        const uint32_t a2 = pack2(r0[(ka + 8) * ak], r0[(ka + 9) * ak]);
        const uint32_t a3 = pack2(r1[(ka + 8) * ak], r1[(ka + 9) * ak]);
#pragma unroll
        for (int q = 0; q < kNT; ++q) {
            if (q < nt_valid) {
                const __nv_bfloat16* bc = B + (n0 + 8 * q + g) * bn;
                const uint32_t b0 = pack2(bc[ka * bk], bc[(ka + 1) * bk]);
                const uint32_t b1 = pack2(bc[(ka + 8) * bk], bc[(ka + 9) * bk]);
                mma_bf16(acc[q], a0, a1, a2, a3, b0, b1);
            }
        }
    }
}

// Offsets of the parameters of one layer in the master layout.
__device__ __forceinline__ size_t off_b1() { return (size_t)kFH * kFAP; }
__device__ __forceinline__ size_t off_w2() { return off_b1() + kFH; }
__device__ __forceinline__ size_t off_b2() { return off_w2() + kFH * kFH; }
__device__ __forceinline__ size_t off_w3() { return off_b2() + kFH; }
__device__ __forceinline__ size_t off_b3(uint32_t AK) { return off_w3() + (size_t)AK * kFH; }

// Recompute xa, h1, h2 of layer l for the state in sm.f.x (all threads call).
__device__ __forceinline__ void mlp_hidden(const FlowView& f, int l, FlowSmem& sm) {
    const int A = (int)f.A, D = (int)f.D;
    const uint8_t* pm = f.perm + l * D;
    __syncthreads();
    load_layer(f, l, sm);
    for (int e = threadIdx.x; e < kRows * kFAP; e += blockDim.x) {
        const int r = e / kFAP, c = e % kFAP;
        sm.xa[r * kFS1 + c] = __float2bfloat16_rn(c < A ? sm.x[r * kXs + pm[c]] : 0.0f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row0 = 16 * warp;
    float acc[8][4];
    warp_gemm<8>(acc, sm.xa, kFS1, row0, sm.w1, kFS1, 0, kFAP, 8);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = 8 * q + 2 * t;
        sm.h1[(row0 + g) * kFS2 + c] = __float2bfloat16_rn(fmaxf(acc[q][0] + sm.b1[c], 0.f));
        sm.h1[(row0 + g) * kFS2 + c + 1] = __float2bfloat16_rn(fmaxf(acc[q][1] + sm.b1[c + 1], 0.f));
        sm.h1[(row0 + g + 8) * kFS2 + c] = __float2bfloat16_rn(fmaxf(acc[q][2] + sm.b1[c], 0.f));
        sm.h1[(row0 + g + 8) * kFS2 + c + 1] = __float2bfloat16_rn(fmaxf(acc[q][3] + sm.b1[c + 1], 0.f));
    }
    __syncwarp();
    warp_gemm<8>(acc, sm.h1, kFS2, row0, sm.w2, kFS2, 0, kFH, 8);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = 8 * q + 2 * t;
        sm.h2[(row0 + g) * kFS2 + c] = __float2bfloat16_rn(fmaxf(acc[q][0] + sm.b2[c], 0.f));
        sm.h2[(row0 + g) * kFS2 + c + 1] = __float2bfloat16_rn(fmaxf(acc[q][1] + sm.b2[c + 1], 0.f));
        sm.h2[(row0 + g + 8) * kFS2 + c] = __float2bfloat16_rn(fmaxf(acc[q][2] + sm.b2[c], 0.f));
        sm.h2[(row0 + g + 8) * kFS2 + c + 1] = __float2bfloat16_rn(fmaxf(acc[q][3] + sm.b2[c + 1], 0.f));
    }
    __syncthreads();
}

// Accumulate a 16-row x (8 nt) column block of a weight gradient into grad.
template <int kNT>
__device__ __forceinline__ void add_grad(float* grad, const float (&acc)[kNT][4], int m0, int ld, int nt_valid) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int q = 0; q < kNT; ++q) {
        if (q < nt_valid) {
            const int c = 8 * q + 2 * t;
            atomicAdd(grad + (m0 + g) * ld + c, acc[q][0]);
            atomicAdd(grad + (m0 + g) * ld + c + 1, acc[q][1]);
            atomicAdd(grad + (m0 + g + 8) * ld + c, acc[q][2]);
            atomicAdd(grad + (m0 + g + 8) * ld + c + 1, acc[q][3]);
        }
    }
}

// One minibatch: rows x[d][off + j], weights w[off + j], j < batch.
// wsum_dev = sum of the minibatch weights; loss_dev += -sum w log q / wsum.
__global__ void __launch_bounds__(128) flow_train_kernel(FlowView f, const float* x, const float* w, uint64_t n,
                                                         uint64_t off, uint32_t batch, const float* wsum_dev,
                                                         float* grad, float* loss_dev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& T = *reinterpret_cast<TrainSmem*>(smem_raw);
    FlowSmem& sm = T.f;
    const int D = (int)f.D, A = (int)f.A, AK = (int)f.AK;
    const size_t S = flow_layer_floats(f.D);
    const float inv_w = 1.0f / fmaxf(*wsum_dev, 1e-30f);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row0 = 16 * warp;
    const uint32_t j0 = blockIdx.x * kRows;
    // ---- forward (density direction), stashing the state entering each layer
    for (int r = threadIdx.x; r < kRows; r += blockDim.x) {
        const uint32_t j = j0 + r;
        const float wr = j < batch ? w[off + j] : 0.f;
        T.s[r] = -wr * inv_w;
        sm.lq[r] = 0.f;
    }
    for (int e = threadIdx.x; e < kRows * D; e += blockDim.x) {
        const int r = e / D, d = e % D;
        const uint32_t j = j0 + r;
        sm.x[r * kXs + d] = j < batch ? x[(uint64_t)d * n + off + j] : 0.5f;
        T.g[r * kXs + d] = 0.f;
    }
    for (int l = 0; l < kFL; ++l) {
        __syncthreads();
        for (int e = threadIdx.x; e < kRows * kXs; e += blockDim.x) T.stash[l][e] = sm.x[e];
        coupling_layer<false>(f, l, sm);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float part = 0.f;
        for (int r = threadIdx.x; r < kRows; r += 32) part += T.s[r] * sm.lq[r];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0) atomicAdd(loss_dev, part);
    }
    // ---- backward through the layers
    for (int l = kFL - 1; l >= 0; --l) {
        const uint8_t* pm = f.perm + l * D;
        float* gl = grad + (size_t)l * S;
        __syncthreads();
        for (int e = threadIdx.x; e < kRows * kXs; e += blockDim.x) sm.x[e] = T.stash[l][e];
        mlp_hidden(f, l, sm);
        // logits chunk by chunk -> dL/dO (bf16) and dL/dt of the transformed coordinates
        for (int c0 = 0; c0 < AK; c0 += 64) {
            const int ncol = min(64, AK - c0);
            float acc[8][4];
            warp_gemm<8>(acc, sm.h2, kFS2, row0, sm.w3, kFS2, c0, kFH, ncol / 8);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (8 * q < ncol) {
                    const int c = 8 * q + 2 * t;
                    sm.lg[(row0 + g) * kLs + c] = acc[q][0] + sm.b3[c0 + c];
                    sm.lg[(row0 + g) * kLs + c + 1] = acc[q][1] + sm.b3[c0 + c + 1];
                    sm.lg[(row0 + g + 8) * kLs + c] = acc[q][2] + sm.b3[c0 + c];
                    sm.lg[(row0 + g + 8) * kLs + c + 1] = acc[q][3] + sm.b3[c0 + c + 1];
                }
            }
            __syncwarp();
            const int r = row0 + (lane & 15);
            for (int jj = 2 * (lane >> 4); jj < 2 * (lane >> 4) + 2; ++jj) {
                if (16 * jj >= ncol) break;
                const float* lg = sm.lg + r * kLs + 16 * jj;
                float P[kFK];
                float m = lg[0];
#pragma unroll
                for (int k = 1; k < kFK; ++k) m = fmaxf(m, lg[k]);
                float Ssum = 0.f;
#pragma unroll
                for (int k = 0; k < kFK; ++k) {
                    P[k] = __expf(lg[k] - m);
                    Ssum += P[k];
                }
#pragma unroll
                for (int k = 0; k < kFK; ++k) P[k] /= Ssum;
                const int cb = pm[A + c0 / 16 + jj];
                const float tt = sm.x[r * kXs + cb];
                const int b = min((int)(tt * (float)kFK), kFK - 1);
                const float qb = (1.0f - kFE) * P[b] + kFE / kFK;
                const float up = T.g[r * kXs + cb];  // dL/d(output coordinate)
                const float sr = T.s[r];
                // dL/dQ_k = up ([k < b] + [k == b](tK - b)) + s [k == b] / Q_b
                float dQ[kFK];
                float dot = 0.f;
#pragma unroll
                for (int k = 0; k < kFK; ++k) {
                    dQ[k] = (k < b ? up : 0.f) + (k == b ? up * (tt * (float)kFK - (float)b) + sr / qb : 0.f);
                    dot += P[k] * dQ[k];
                }
                __nv_bfloat16* dst = T.dO + r * kSO + c0 + 16 * jj;
#pragma unroll
                for (int k = 0; k < kFK; ++k) dst[k] = __float2bfloat16_rn((1.0f - kFE) * P[k] * (dQ[k] - dot));
                T.g[r * kXs + cb] = up * (float)kFK * qb;  // dL/dt through the CDF
            }
            __syncwarp();
        }
        __syncthreads();
        // bias gradients (column sums over the tile)
        for (int c = threadIdx.x; c < AK; c += blockDim.x) {
            float sacc = 0.f;
            for (int r = 0; r < kRows; ++r) sacc += __bfloat162float(T.dO[r * kSO + c]);
            atomicAdd(gl + off_b3(f.AK) + c, sacc);
        }
        {   // dh2 = (dO W3) * [h2 > 0]
            float acc[8][4];
            warp_gemm_g<8>(acc, T.dO, kSO, 1, row0, sm.w3, kFS2, 1, 0, AK, 8);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * q + 2 * t;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int rr = row0 + g + (h >= 2 ? 8 : 0), cc = c + (h & 1);
                    const bool on = __bfloat162float(sm.h2[rr * kFS2 + cc]) > 0.f;
                    T.dh2[rr * kFS2 + cc] = __float2bfloat16_rn(on ? acc[q][h] : 0.f);
                }
            }
        }
        // dW3 = dO^T h2 (rows of dW3 = logits, 16 per m-tile, spread over the warps)
        for (int mt = warp; mt < AK / 16; mt += 4) {
            float acc[8][4];
            warp_gemm_g<8>(acc, T.dO, 1, kSO, 16 * mt, sm.h2, kFS2, 1, 0, kRows, 8);
            add_grad<8>(gl + off_w3(), acc, 16 * mt, kFH, 8);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < kFH; c += blockDim.x) {
            float sacc = 0.f;
            for (int r = 0; r < kRows; ++r) sacc += __bfloat162float(T.dh2[r * kFS2 + c]);
            atomicAdd(gl + off_b2() + c, sacc);
        }
        {   // dh1 = (dh2 W2) * [h1 > 0]
            float acc[8][4];
            warp_gemm_g<8>(acc, T.dh2, kFS2, 1, row0, sm.w2, kFS2, 1, 0, kFH, 8);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * q + 2 * t;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int rr = row0 + g + (h >= 2 ? 8 : 0), cc = c + (h & 1);
                    const bool on = __bfloat162float(sm.h1[rr * kFS2 + cc]) > 0.f;
                    T.dh1[rr * kFS2 + cc] = __float2bfloat16_rn(on ? acc[q][h] : 0.f);
                }
            }
        }
        {   // dW2 = dh2^T h1 (one m-tile per warp)
            float acc[8][4];
            warp_gemm_g<8>(acc, T.dh2, 1, kFS2, 16 * warp, sm.h1, kFS2, 1, 0, kRows, 8);
            add_grad<8>(gl + off_w2(), acc, 16 * warp, kFH, 8);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < kFH; c += blockDim.x) {
            float sacc = 0.f;
            for (int r = 0; r < kRows; ++r) sacc += __bfloat162float(T.dh1[r * kFS2 + c]);
            atomicAdd(gl + off_b1() + c, sacc);
        }
        {   // d x_A = dh1 W1 -> into the conditioner coordinates' gradient
            float acc[2][4];
            warp_gemm_g<2>(acc, T.dh1, kFS2, 1, row0, sm.w1, kFS1, 1, 0, kFH, 2);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = 8 * q + 2 * t;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int rr = row0 + g + (h >= 2 ? 8 : 0), cc = c + (h & 1);
                    if (cc < A) T.g[rr * kXs + pm[cc]] += acc[q][h];
                }
            }
        }
        {   // dW1 = dh1^T xa (one m-tile per warp, 16 columns)
            float acc[2][4];
            warp_gemm_g<2>(acc, T.dh1, 1, kFS2, 16 * warp, sm.xa, kFS1, 1, 0, kRows, 2);
            add_grad<2>(gl, acc, 16 * warp, kFAP, 2);
        }
    }
}

// Sum of the minibatch weights.
__global__ void wsum_kernel(const float* w, uint64_t off, uint32_t batch, float* out) {
    float s = 0.f;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < batch; j += gridDim.x * blockDim.x) s += w[off + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters.
__global__ void adam_kernel(float* p, const float* gr, float* m, float* v, uint64_t count, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < count;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const float gg = gr[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

// FP32 master parameters (the documented layout: per layer W1 [64][16], b1,
// W2 [64][64], b2, W3 [AK][64], b3) -> padded bf16 weights + FP32 biases.
__global__ void pack_kernel(const float* master, __nv_bfloat16* wb, float* bias, uint32_t AK) {
    const int l = blockIdx.y;
    const size_t S = (size_t)kFH * kFAP + kFH + kFH * kFH + kFH + (size_t)AK * kFH + AK;
    const float* m = master + l * S;
    __nv_bfloat16* w = wb + (size_t)l * (kFH * kFS1 + kFH * kFS2 + (size_t)AK * kFS2);
    float* b = bias + (size_t)l * (2 * kFH + AK);
    const uint32_t tot = kFH * kFS1 + kFH * kFS2 + AK * kFS2;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (e < (uint32_t)(kFH * kFS1)) {
            const uint32_t r = e / kFS1, c = e % kFS1;
            if (c < (uint32_t)kFAP) v = m[r * kFAP + c];
        } else if (e < (uint32_t)(kFH * kFS1 + kFH * kFS2)) {
            const uint32_t q = e - kFH * kFS1, r = q / kFS2, c = q % kFS2;
            if (c < (uint32_t)kFH) v = m[kFH * kFAP + kFH + r * kFH + c];
        } else {
            const uint32_t q = e - kFH * kFS1 - kFH * kFS2, r = q / kFS2, c = q % kFS2;
            if (c < (uint32_t)kFH) v = m[kFH * kFAP + kFH + kFH * kFH + kFH + r * kFH + c];
        }
        w[e] = __float2bfloat16_rn(v);
    }
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * kFH + AK; e += gridDim.x * blockDim.x) {
        if (e < (uint32_t)kFH) b[e] = m[kFH * kFAP + e];
        else if (e < (uint32_t)(2 * kFH)) b[e] = m[kFH * kFAP + kFH + kFH * kFH + (e - kFH)];
        else b[e] = m[kFH * kFAP + kFH + kFH * kFH + kFH + (size_t)AK * kFH + (e - 2 * kFH)];
    }
}

// Chain states as training rows for the flow: x_out [D][n] = the current
// states, w_out[i] = p / (p + c~ u) = E[dt | x] = 1 / (1 + k(x)), which turns
// the states' jump-chain law (proportional to p + c~ u) into pi.
__global__ void snapshot_kernel(ChainView c, float* x_out, float* w_out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    for (uint32_t d = 0; d < c.dim; ++d) x_out[d * c.n + i] = c.x[xidx(d, i, c.n)];
    const float p = c.fpu[3 * c.n + i], u = c.fpu[4 * c.n + i];
    w_out[i] = p > 0.f ? p / (p + c.c_tilde * u) : 0.f;
}

// The rows of weight > 0 appended to a ring: one counter update per warp.
__global__ void snapshot_append_kernel(ChainView c, float* x_ring, float* w_ring, uint64_t cap,
                                       unsigned long long* total) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    float w = 0.f;
    if (i < c.n) {
        const float p = c.fpu[3 * c.n + i], u = c.fpu[4 * c.n + i];
        w = p > 0.f ? p / (p + c.c_tilde * u) : 0.f;
    }
    const unsigned keep = __ballot_sync(0xffffffffu, w > 0.f);
    if (!keep) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(total, (unsigned long long)__popc(keep));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!(w > 0.f)) return;
    const uint64_t slot = (base + __popc(keep & ((1u << lane) - 1u))) % cap;
    for (uint32_t d = 0; d < c.dim; ++d) x_ring[d * cap + slot] = c.x[xidx(d, i, c.n)];
    w_ring[slot] = w;
}

}  // namespace

cudaError_t launch_snapshot(const ChainView& c, float* x_out, float* w_out, cudaStream_t st) {
    snapshot_kernel<<<(unsigned)((c.n + 255) / 256), 256, 0, st>>>(c, x_out, w_out);
    return cudaGetLastError();
}

cudaError_t launch_snapshot_append(const ChainView& c, float* x_ring, float* w_ring, uint64_t cap,
                                   unsigned long long* total, cudaStream_t st) {
    snapshot_append_kernel<<<(unsigned)((c.n + 255) / 256), 256, 0, st>>>(c, x_ring, w_ring, cap, total);
    return cudaGetLastError();
}

cudaError_t launch_flow_train_step(const FlowView& f, const float* x, const float* w, uint64_t n, uint64_t off,
                                   uint32_t batch, float* grad, float* wsum, float* loss, cudaStream_t st) {
    static DeviceOnce once;  // per device: the opt-in to the training kernel's shared memory
    const size_t shm = sizeof(TrainSmem);
    cudaError_t e0 = once.get(
        [&](int, long long*) {
            return cudaFuncSetAttribute(flow_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        },
        nullptr);
    if (e0 != cudaSuccess) return e0;
    wsum_kernel<<<std::min<uint32_t>(64, (batch + 255) / 256), 256, 0, st>>>(w, off, batch, wsum);
    flow_train_kernel<<<(batch + kRows - 1) / kRows, 128, shm, st>>>(f, x, w, n, off, batch, wsum, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, uint64_t count, float lr, uint64_t t,
                        cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - powf(b1, (float)t), bc2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<256, 256, 0, st>>>(p, g, m, v, count, lr, b1, b2, 1e-8f, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_flow_pack(const float* master, __nv_bfloat16* wb, float* bias, uint32_t AK, cudaStream_t st) {
    pack_kernel<<<dim3(16, kFL), 256, 0, st>>>(master, wb, bias, AK);
    return cudaGetLastError();
}

}  // namespace jr
