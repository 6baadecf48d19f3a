// Internal layout shared by the host runtime (jr_api.cu, bvh_build.cpp) and the
// kernels (jr_kernels.cu).  Not part of the C ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

namespace jr {

constexpr int kMaxDepth = 15;
constexpr int kMaxDim = 2 + 2 * kMaxDepth;  // 32
constexpr int kStackSize = 96;              // traversal stack entries
constexpr int kMaxBvhDepth = 62;            // depth limit of the binary SAH build (before the 4-wide collapse)
constexpr int kLeafMax = 8;                 // triangles per leaf (encoded count-1 in 3 bits)
constexpr uint32_t kNodeVisitBudget = 1u << 16;  // per ray; exceeding it is a watchdog event

constexpr uint32_t kTagStep = 0, kTagInit = 1, kTagPt = 2, kTagRestart = 3;
constexpr int kCounters = 8;   // ChainView::counters entries
constexpr int kCounterPSum = 5;  // MH: sum of p over the large-step proposals (double)
constexpr uint64_t kWavefrontMinChains = 1u << 18;  // JR_EXEC_AUTO picks the wavefront from here up

// 4-wide BVH node, 128 bytes (one L2 line): the boxes of up to 4 children,
// one float4 per plane with child j in component j, then the child refs:
// >= 0 inner node index; < 0 leaf = ~((first << 3) | (count - 1)); kNoChild
// marks an empty slot, whose box is the empty box (lo = +inf, hi = -inf), so
// that the slab test misses it.  pad.x holds the child count; the rest of the
// last 16 bytes is unused.
struct __align__(128) Bvh4Node {
    float4 lox, hix, loy, hiy, loz, hiz;
    int4 refs;
    int4 pad;
};
static_assert(sizeof(Bvh4Node) == 128, "a 4-wide node is one 128-byte line");
constexpr int kNoChild = INT32_MIN;

// Triangle in BVH leaf order, 48 bytes: v0 | original id, e1 | material, e2.
struct __align__(16) TriRecord {
    float4 v0_id;   // .w = __int_as_float(original index)
    float4 e1_mat;  // .w = __int_as_float(material index)
    float4 e2;
};

// Material, prepared on the host.
struct __align__(16) Material {
    int type;
    int emits;
    float phong_inv_n1;  // 1 / (n + 1)
    float phong_scale;   // (n + 2) / (n + 1)
    float3 albedo;
    float ior;
    float3 emission;
    float pad;
};

struct SceneView {
    const Bvh4Node* nodes;
    const TriRecord* tris;
    const Material* mats;
    int root;       // child ref of the root, or INT32_MIN when the scene is empty
    int n_nodes;
    uint32_t n_tris;  // triangle records (leaf order)
    float cam[12];
    uint32_t visit_budget;  // node visits per ray before the watchdog stops it (kNodeVisitBudget)
    int stack_limit;        // traversal stack entries a ray may use (<= kStackSize)
};

// The regeneration flow (jr_flow.cu): L coupling layers, MLP of 2 x 64 hidden
// units, K bins, conditioner width padded to kFAP; bf16 weight rows padded to
// strides kFS1 / kFS2 (conflict-free fragment loads).
constexpr int kFL = 6, kFH = 64, kFK = 16, kFAP = 16, kFS1 = 24, kFS2 = 72, kFMaxAK = 256;
constexpr float kFE = 1e-3f;  // bin-mass floor: Q = (1 - E) softmax + E / K

// Inference layout of one flow layer (bytes, 16-byte multiples): W1 [64][16],
// W2 [64][64], W3 [AK][64] bf16, then b1 [64], b2 [64], log2(e) b3 [AK] FP32.  Row n of
// a bf16 matrix is stored in 16-byte chunks; chunk c sits at position c ^ (n & 7)
// (W2, W3) or c ^ ((n >> 2) & 1) (W1), so the 8 rows of an mma B fragment hit
// 8 different bank groups.
__host__ __device__ constexpr size_t flow_ws_layer_bytes(uint32_t AK) {
    return 2 * ((size_t)kFH * kFAP + kFH * kFH + (size_t)AK * kFH) + 4 * (2 * (size_t)kFH + AK);
}

struct FlowView {
    uint32_t D = 0, A = 0, AK = 0;      // AK = A * K logits per layer
    const uint8_t* perm = nullptr;      // [kFL][D]
    const __nv_bfloat16* wb = nullptr;  // per layer: W1 [64][kFS1], W2 [64][kFS2], W3 [AK][kFS2]
    const float* bias = nullptr;        // per layer: b1 [64], b2 [64], b3 [AK]
    const unsigned char* ws = nullptr;  // inference layout, flow_ws_layer_bytes(AK) per layer
    float beta = 0.f;                   // mu = beta mu_flow + (1 - beta) uniform
    uint32_t extra_tx = 0;              // testing hook: bytes the first weight barrier expects beyond its copy
};

// Buffers of the wavefront execution mode (allocated on first use).
struct WaveView {
    float* y = nullptr;           // second state buffer, the pair layout of x (xidx)
    uint8_t* par = nullptr;       // [n] 1: the current state is in y, 0: in x
    float* ua = nullptr;          // [n] Ua of a local step, -1 for a regeneration step
    float4* fy = nullptr;         // [n] the candidate's (y0, y1, y2, y3) from the step launch until its path
                                  // starts, then F(y) (xyz; w unused)
    uint32_t* queue = nullptr;    // [n] the step's path queue (drain steps; otherwise every chain in order)
    unsigned int* qcount = nullptr;  // [kQCount]: queue lengths, fetch cursors, flow queue lengths
    float* uy = nullptr;          // [n] u of the step's candidate (with a flow)
    uint32_t* fq = nullptr;       // [2][n] candidates for the flow: density rows, then sampling rows
    uint8_t* done = nullptr;      // [n] 1: the chain finished its tour during a drain
};
constexpr int kQFlowDensity = 2 * (kMaxDepth + 2), kQFlowSample = kQFlowDensity + 1, kQActive = kQFlowSample + 1,
              kQCount = kQActive + 1;
// Step-kernel modes of the wavefront: a regular step of Alg. 2; a restart of
// every chain from mu (new tours, not regenerations); a drain step (a kill
// ends the chain's tour and the chain; no new tours start).
enum WaveMode { kModeStep = 0, kModeRestart = 1, kModeDrain = 2 };

// The state buffers (x, and the wavefront's y) hold coordinate pairs: the pair
// (x_{2k}, x_{2k+1}) of chain i is one float2 at pair index k n + i, so a path
// vertex's two coordinates are one 8-byte load from one sector.  D is always
// even (2 + 2 depth).  Coordinate d of chain i is float xidx(d, i, n).
__host__ __device__ inline uint64_t xidx(uint32_t d, uint64_t i, uint64_t n) {
    return ((((uint64_t)(d >> 1)) * n + i) << 1) | (uint64_t)(d & 1u);
}

struct ChainView {
    float* x;        // PSS coordinates, D x n floats as n float2 per coordinate pair (xidx)
    float* fpu;      // [5][n] F.r F.g F.b p u
    float4* fb;      // [H*W] RGB sum + dt, FP32 (folded into acc64 after each advance)
    double4_32a* acc64;  // [H*W]
    // [0] J (MH: large-step proposals), [1] local steps (MH: small-step
    // proposals), [2] accepted, [3] drain mark, [4] unused, [5] MH: the sum of
    // p over the large-step proposals (a double's bits), [6..7] unused
    unsigned long long* counters;
    unsigned int* status;
    uint64_t n;
    uint32_t chain_offset;
    uint32_t width, height, depth, dim;
    uint32_t flags;                // JR_FLAG_*; JR_FLAG_MH: the MH baseline instead of Jump Restore
    uint64_t seed;
    float c_tilde, sigma;
    float large_step;              // MH: large-step probability l of the mixture proposal
    uint64_t burn_in;              // MH: iterations before the estimator starts
    float* drift;                  // JR_FLAG_MALA: [D][n] the MALA drift m(x) of each state
    WaveView wf;
    FlowView flow;   // flow.D == 0: uniform regeneration (u = 1)
};

// A chain set of a batch as the batched kernels see it; `step` is the set's
// next Philox step index, advanced on the device by every batched launch.
struct BatchEntry {
    SceneView s;
    ChainView c;
    unsigned long long step;
};

// One work item of the batched kernel: chains [begin, end) of set `set`.
struct BatchItem {
    uint32_t set, begin, end;
};

// Batched wavefront (jr_wavefront.cu): the sets of a batch advance in shared
// step and path launches over one merged device scene.  rebase_ref moves a
// node child ref of a scene whose nodes and triangles were placed at node_off,
// tri_off in the merged arrays.
constexpr uint32_t kBatchMaxSets = 1024;
__host__ __device__ inline int rebase_ref(int r, int node_off, int tri_off) {
    if (r == kNoChild) return r;
    if (r >= 0) return r + node_off;
    const int enc = ~r;  // (first << 3) | (count - 1)
    return ~((((enc >> 3) + tri_off) << 3) | (enc & 7));
}
struct BatchWave {
    SceneView merged;           // every set's scene; root and camera unused
    const int* roots;           // [n_sets] each set's root ref in the merged scene
    const uint64_t* chain_off;  // [n_sets + 1] prefix sums of the sets' chain counts
    const BatchItem* items;     // [n_items] work items of 128 chains for the step launches
    uint32_t n_sets = 0, n_items = 0;
    unsigned int* fetch;        // the path launches' item cursor
};
// Rebase one scene's nodes and triangles, already copied into the
// merged arrays (refs via rebase_ref, material indices + mat_off).
cudaError_t launch_rebase_scene(Bvh4Node* nodes, uint32_t n_nodes, TriRecord* tris, uint32_t n_tris, int node_off,
                                int tri_off, int mat_off, cudaStream_t st);
// The batched path kernel's persistent grid (set up once per device; call it
// outside stream capture before the first launch_batch_wavefront).
cudaError_t batch_wavefront_grid(long long* blocks);
// n_steps batched wavefront steps of every set (step indices entries[q].step + k),
// ending with the closing step launch; the caller folds afterwards.  flow_sets:
// the host views of the sets with a flow attached (their flow launches run
// between the shared step and path launches).
cudaError_t launch_batch_wavefront(const BatchWave& bw, BatchEntry* entries, uint32_t n_steps,
                                   const std::vector<ChainView>& flow_sets, cudaStream_t st);

// One-time launch set-up per device (an opt-in to large dynamic shared
// memory, an occupancy-derived grid size), cached by device id: get() runs
// init(device, &value) for the current device on first use, under a lock, and
// returns the cached value afterwards; a failed init is retried on the next call.
struct DeviceOnce {
    static constexpr int kDevices = 64;
    std::mutex mu;
    bool done[kDevices] = {};
    long long value[kDevices] = {};
    template <class F>
    cudaError_t get(F&& init, long long* out) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        if (!done[dev]) {
            long long v = 0;
            if ((e = init(dev, &v)) != cudaSuccess) return e;
            value[dev] = v;
            done[dev] = true;
        }
        if (out) *out = value[dev];
        return cudaSuccess;
    }
};

// Host-side BVH build result.
struct HostBvh {
    std::vector<Bvh4Node> nodes;
    std::vector<TriRecord> tris;
    int root = 0;
    int depth = 0;
};

// bvh_build.cpp
bool build_bvh(const float* verts, uint32_t n_verts, const uint32_t* tris, uint32_t n_tris,
               const uint32_t* tri_mat, HostBvh* out, std::string* err);

// jr_kernels.cu -- launch wrappers; all return the cudaGetLastError() of the launch.
cudaError_t launch_init(const SceneView& s, const ChainView& c, cudaStream_t st);
// One chain per warp (JR_EXEC_WARP): brute-force intersection over every
// triangle, for small scenes; auto mode takes it for at most kWarpChainMaxTris
// triangles and fewer than 32 chains per SM.
constexpr uint32_t kWarpChainMaxTris = 128;
cudaError_t launch_step_warp(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                             cudaStream_t st);
cudaError_t launch_step(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                        uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix, unsigned long long* work_out, int block,
                        cudaStream_t st);
cudaError_t launch_fold(const ChainView& c, cudaStream_t st);
// JR_FLAG_MALA chain sets: n steps with Langevin local moves (megakernel, one
// chain per thread, 128 threads per block); F, p and drift of stored states;
// F [3][n] and dF/dx [3][D][n] of given states x [D][n].
cudaError_t launch_step_mala(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                             uint8_t* tr_flags, float* tr_dt, int32_t* tr_pix, cudaStream_t st);
cudaError_t launch_mala_reeval(const SceneView& s, const ChainView& c, cudaStream_t st);
cudaError_t launch_eval_grad(const SceneView& s, uint32_t depth, const float* x, uint64_t n, float* F, float* dF,
                             cudaStream_t st);
// Batched persistent launch + fold over n_sets chain sets (block = chains per
// work item = threads per block, a multiple of 32 in [32, 256]).
cudaError_t launch_batch(BatchEntry* entries, const BatchItem* items, uint32_t n_items, const uint64_t* px_off,
                         uint32_t n_sets, uint64_t total_px, unsigned int* cursor, uint32_t max_dim, int block,
                         uint32_t n_steps, cudaStream_t st);
// Device time per kernel class of a sequence of launches on one stream: an
// event is recorded after every launch, and the time since the previous event
// is charged to that launch's class.
struct KernelTimer {
    enum Kind { kStep = 0, kPath = 1, kReserved = 2, kFlow = 3, kKinds = 4 };
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;  // class of the launch that ends at ev[i] (-1: the start mark)
    cudaError_t mark(int k, cudaStream_t st);
    // After the stream is synchronised: ms[k] and launches[k] per class.
    cudaError_t totals(double ms[kKinds], uint64_t launches[kKinds]) const;
    ~KernelTimer();
};

// jr_wavefront.cu
// n_steps wavefront steps in `mode` (WaveMode); for kModeRestart step_begin is
// the restart epoch and n_steps is 1.  tm (optional) times every launch.
cudaError_t launch_wavefront(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                             cudaStream_t st, int mode = kModeStep, KernelTimer* tm = nullptr);
// The same wavefront launches with their buffers in a fixed file-scope device
// array (no allocation); c.wf is ignored.  c.n <= kStaticMaxChains.
constexpr uint64_t kStaticMaxChains = 1u << 16;
constexpr size_t kStaticScratchBytes =
    sizeof(float) * kMaxDim * kStaticMaxChains + sizeof(float4) * kStaticMaxChains +
    sizeof(float) * kStaticMaxChains + sizeof(uint32_t) * kStaticMaxChains + sizeof(uint8_t) * kStaticMaxChains +
    256;  // = 10 027 264 bytes (every piece but the counters is a multiple of 256)
cudaError_t launch_wavefront_static(const SceneView& s, const ChainView& c, uint64_t step_begin, uint32_t n_steps,
                                    cudaStream_t st);
// Load the module that holds the static scratch on the current device and cache
// the array's device address (the first call on a device allocates the array).
cudaError_t prepare_static_scratch();

// jr_flow.cu: flow rows through the tensor cores.  Density: u_out[i] = beta q
// + 1 - beta (and lq_out[i] = log q) for rows i of buf [D][n]; sample: buf
// rows replaced by T^{-1}(buf), and start[i] (if not null) = the row's first
// four coordinates (0 past D).  Rows are idx[j], j < *count_dev (device) or
// n_rows.
// pairs: the rows live in chain state buffers (the xidx pair layout), else in a
// caller's SoA buffer [D][n].
cudaError_t launch_flow(const FlowView& f, bool sample, float* bufA, float* bufB, const uint8_t* par, uint64_t n,
                        const uint32_t* idx, const unsigned int* count_dev, uint32_t n_rows, float* u_out,
                        float* lq_out, float4* start, unsigned int* status, cudaStream_t st, bool pairs = false);
// FP32 master parameters [kFL][S] -> the inference layout (flow_ws_layer_bytes per layer).
cudaError_t launch_flow_pack_ws(const float* master, unsigned char* ws, uint32_t AK, cudaStream_t st);
// FP32 master parameters [kFL][S] -> padded bf16 weights and biases.
cudaError_t launch_flow_pack(const float* master, __nv_bfloat16* wb, float* bias, uint32_t AK, cudaStream_t st);
__host__ __device__ inline size_t flow_layer_floats(uint32_t D) {
    const size_t A = D / 2, AK = A * kFK;
    return (size_t)kFH * kFAP + kFH + kFH * kFH + kFH + AK * kFH + AK;
}
// Training rows from chain states (x [D][n], w = p / (p + c~ u)).
cudaError_t launch_snapshot(const ChainView& c, float* x_out, float* w_out, cudaStream_t st);
cudaError_t launch_snapshot_append(const ChainView& c, float* x_ring, float* w_ring, uint64_t cap,
                                   unsigned long long* total, cudaStream_t st);
// One minibatch of the time-weighted maximum-likelihood loss: gradient into
// grad (added), minibatch weight sum into *wsum (added), loss into *loss (added).
cudaError_t launch_flow_train_step(const FlowView& f, const float* x, const float* w, uint64_t n, uint64_t off,
                                   uint32_t batch, float* grad, float* wsum, float* loss, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, uint64_t count, float lr, uint64_t t,
                        cudaStream_t st);
// image = accumulator / J (Jump Restore), or b_hat accumulator / mh_samples
// with b_hat = (sum of p over large steps) / (large steps) (MH, JR_FLAG_MH).
cudaError_t launch_resolve(const ChainView& c, float* rgb, uint64_t mh_samples, cudaStream_t st);
cudaError_t launch_reeval(const SceneView& s, const ChainView& c, cudaStream_t st);
cudaError_t launch_eval_states(const SceneView& s, uint32_t depth, float c_tilde, const float* x, uint64_t n,
                               float* F, float* p, float* u, float* k, int32_t* ids, cudaStream_t st);
cudaError_t launch_render_pt(const SceneView& s, uint32_t width, uint32_t height, uint32_t depth, uint64_t seed,
                             uint64_t sample_begin, uint64_t n, double* accum, cudaStream_t st);
// FP32 FMA throughput of the device (TFLOP/s, best of four timed launches of
// a kernel of independent FMA chains over every SM); ms_out = its launch time.
cudaError_t measure_fma_peak(double* tflops, double* ms_out, cudaStream_t st);
cudaError_t launch_philox(uint64_t seed, uint32_t tag, uint32_t block, uint64_t chain_begin, uint64_t step,
                          uint64_t n, uint32_t* out, cudaStream_t st);

}  // namespace jr
