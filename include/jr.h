/*
 * jr.h -- C ABI of the GB300-native Jump Restore light-transport library.
 *
 * Method: Holl, Singh, Seidel, "Jump Restore Light Transport" (arXiv 2409.07148).
 * Many independent Jump Restore chains (Alg. 2, Section 7.2) advance in lockstep
 * over primary sample space (PSS) x in [0,1)^D, D = 2 + 2 * max_depth:
 *   - local dynamics: one Metropolis-Hastings step (Alg. 1, Section 4) with a
 *     Gaussian small-step kernel of standard deviation `sigma` per coordinate,
 *     wrapped onto the unit torus (symmetric, so alpha = min(1, p(y)/p(x)));
 *   - global dynamics mu: uniform on [0,1)^D (the large-step distribution,
 *     Section 8), density u = 1;
 *   - killing rate k = c~ u / p (Section 6.2, invariant local dynamics and
 *     state-independent mu), k = +inf where p = 0;
 *   - target density p = luminance (0.2126, 0.7152, 0.0722) of the RGB path
 *     contribution F(x) of a unidirectional path tracer;
 *   - estimator: normalisation-free tour estimator (Section 6.3) with the
 *     left-rectangle rule of Section 7.4: pixel j = (c~/J) sum_i dt_i W H
 *     F(x_{i-1}) / p(x_{i-1}) over the steps whose state lies in pixel j, where
 *     J counts regenerations (completed tours).
 *
 * Conventions (all entry points):
 *   - Every call returns a jr_status; no exception or abort crosses the ABI.
 *     On error the outputs are left untouched and jr_last_error() returns a
 *     thread-local message.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that only enqueue device work are asynchronous on that
 *     stream; calls that return host data synchronise it.
 *   - Handles are opaque and owned by the library; free them with
 *     jr_*_destroy.  Host arrays passed in are caller-owned and copied before
 *     the call returns.  Device pointers passed in are caller-owned and must
 *     stay valid until the enqueued work completes.
 *   - Device-side faults of the method (non-finite F, traversal budget
 *     exhausted) are recorded in a status word read by jr_get_stats.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key =
 *     (lo32(seed), hi32(seed)) and counter = (block + 256 tag, chain id,
 *     lo32(step), hi32(step)); tag 0 = a chain step (block 0 gives U1, U2, Ua;
 *     blocks 1.. give the D coordinates: Gaussian pairs for a local move or
 *     uniforms for a regeneration), tag 1 = initial state (blocks 1..),
 *     tag 2 = plain path-tracing sample.  A uniform is (r >> 8) * 2^-24.
 */
#ifndef JR_H
#define JR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JR_OK = 0,
    JR_ERR_INVALID_ARG = 1, /* a null pointer, a size out of range, a malformed scene */
    JR_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
    JR_ERR_OOM = 3,         /* device or host allocation failed */
    JR_ERR_WATCHDOG = 4,    /* a device-side iteration budget was exhausted */
    JR_ERR_NUMERIC = 5,     /* a non-finite value reached the estimator */
    JR_ERR_STATE = 6        /* the handle is in a state that does not allow the call */
} jr_status;

#define JR_MATERIAL_FLOATS 12 /* [type, albedo rgb, emission rgb, phong n, ior, 0, 0, 0] */
#define JR_MAT_LAMBERT 0      /* two-sided Lambertian, cosine-weighted sampling, weight = albedo */
#define JR_MAT_PHONG 1        /* modified Phong lobe about the mirror direction, weight rho (n+2)/(n+1) cos */
#define JR_MAT_DIELECTRIC 2   /* smooth dielectric, Fresnel-chosen reflect/refract, weight 1 */
#define JR_MAX_DEPTH 15       /* D = 2 + 2 * max_depth <= 32 */
#define JR_FLAG_RAO_BLACKWELL 1u /* splat the conditional mean 1/(1+k) instead of the sampled dt */
/* The chain set runs the paper's MH baseline "Metropolis" (Section 8, practical
 * pairing) instead of Jump Restore: Alg. 1 (Section 4) with the mixture
 * proposal of Section 5 (eq. "mixture-proposal-kernel"), Q_l(x, .) = l mu +
 * (1 - l) zeta(x, .), mu uniform on [0,1)^D, zeta the Gaussian small step;
 * both parts are symmetric, so alpha = min(1, p(y)/p(x)) (1 if p(x) = 0).  The
 * estimate is the chain's ergodic average after `burn_in` iterations (Section
 * 9 uses l = 0.3 and 10,000): pixel j = b_hat (1/N) sum_i W H 1[pix(x_i) = j]
 * F(x_i) / p(x_i), x_i the state held at iteration i >= burn_in, N the number
 * of such iterations over all chains, and b_hat = the mean of p over the
 * large-step proposals (uniform draws: an unbiased estimate of the integral of
 * p).  Random numbers: the Restore step's counters; block 0 gives (U_s, -, U_a,
 * -), a large step if U_s < l; blocks 1.. give the D uniforms (large) or
 * Gaussian pairs (small).  Not with JR_FLAG_RAO_BLACKWELL, flows or drains. */
#define JR_FLAG_MH 2u
/* Langevin local dynamics (MALA; the paper's "MALA Restore" and, with
 * JR_FLAG_MH, its "MALA" baseline, Section 9): the local move (or the MH small
 * step) proposes y = (x + m(x) + sigma N) mod 1 with the drift
 * m(x) = clamp(sigma^2 / 2 grad log p(x), -2 sigma, 2 sigma) per coordinate and
 * accepts with min(1, p(y) q(x|y) / (p(x) q(y|x))), q(b|a) = prod_d
 * phi_sigma(b_d - a_d - m_d(a)) on the signed torus difference.  grad log p is
 * the forward-mode derivative of the path contribution (it flows through the
 * directions and the modified Phong weights; Lambertian and dielectric weights
 * are constant).  MALA is pi-invariant, so MALA Restore keeps k = c~ u / p.
 * Runs in the megakernel only (jr_advance picks it; 128 threads per block); not
 * with JR_FLAG_RAO_BLACKWELL, flows, drains, batches or jr_advance_static. */
#define JR_FLAG_MALA 4u

/* status-word bits (jr_stats.status_word) */
#define JR_STATUS_NONFINITE 1u  /* F(x) was NaN/Inf for some state: it was treated as 0 */
#define JR_STATUS_TRAVERSAL 2u  /* a ray exhausted the BVH node-visit budget: treated as a miss */
#define JR_STATUS_STACK 4u      /* a traversal stack overflowed: treated as a miss */
#define JR_STATUS_FLOW_WAIT 8u  /* a flow kernel's weight copy did not arrive in time: its outputs are invalid */

typedef struct jr_scene jr_scene;
typedef struct jr_chains jr_chains;

/* Scene: triangles with per-triangle material, a pinhole camera.  Host
 * arrays, caller-owned, copied by jr_scene_create.
 *   verts        n_verts x 3 float (x, y, z)
 *   tris         n_tris x 3 uint32 vertex indices; winding gives the
 *                geometric normal (v1 - v0) x (v2 - v0), the emitting side
 *   tri_material n_tris uint32 indices into materials
 *   materials    n_materials x JR_MATERIAL_FLOATS float
 *   camera       origin, forward, right, up (12 floats): film point (x0, x1)
 *                looks along forward + (2 x0 - 1) right + (1 - 2 x1) up. */
typedef struct {
    const float* verts;
    uint32_t n_verts;
    const uint32_t* tris;
    uint32_t n_tris;
    const uint32_t* tri_material;
    const float* materials;
    uint32_t n_materials;
    float camera[12];
} jr_scene_desc;

/* Render / chain parameters (Alg. 2 inputs: target via the scene, mu, zeta,
 * c~; Section 7.2). */
typedef struct {
    uint32_t width, height; /* image W x H; pixel (floor(x0 W), floor(x1 H)) */
    uint32_t max_depth;     /* scattering events per path, 0..JR_MAX_DEPTH */
    uint32_t flags;         /* JR_FLAG_* */
    uint64_t n_chains;      /* chains in this set, >= 1 */
    uint64_t chain_offset;  /* global id of the first chain (disjoint Philox streams) */
    uint64_t seed;          /* Philox key */
    float c_tilde;          /* c~ > 0 of the killing rate (the paper uses 1, Section 9) */
    float sigma;            /* std of the Gaussian small-step kernel zeta, > 0 */
    float large_step;       /* JR_FLAG_MH: large-step probability l in [0, 1] (Section 9: 0.3) */
    uint32_t burn_in;       /* JR_FLAG_MH: iterations (step index) before the estimator starts */
} jr_params;

typedef struct {
    uint64_t steps_per_chain; /* Alg. 2 iterations each chain has taken */
    uint64_t regenerations;   /* J: killings followed by a draw from mu (completed tours); MH: large-step proposals */
    uint64_t local_steps;     /* iterations that took the local branch; MH: small-step proposals */
    uint64_t accepted;        /* accepted local MH proposals; MH: accepted proposals of both kinds */
    uint32_t status_word;     /* JR_STATUS_* bits, sticky */
    uint32_t dim;             /* D */
    double p_sum_large;       /* MH: sum of p over the large-step proposals (b_hat = p_sum_large / regenerations) */
} jr_stats;

typedef struct {
    uint32_t n_tris, n_nodes, bvh_depth, n_materials;
    uint64_t device_bytes; /* nodes + triangles + materials */
} jr_scene_info;

/* Upload a scene and build its BVH (binned SAH, host, native code).  The
 * triangle arrays are copied; the call synchronises `stream` before it
 * returns.  n_tris may be 0 (every ray misses).  Errors: JR_ERR_INVALID_ARG
 * (index out of range, a triangle's vertex coordinate not finite, unknown
 * material type, n_tris >= 2^27), JR_ERR_OOM, JR_ERR_CUDA. */
jr_status jr_scene_create(const jr_scene_desc* desc, void* stream, jr_scene** out);
jr_status jr_scene_get_info(const jr_scene* scene, jr_scene_info* out);
void jr_scene_destroy(jr_scene* scene);

/* Create a set of chains (library-owned SoA state, RGBA float framebuffer,
 * FP64 accumulator, counters) and draw each initial state x0 ~ mu (Alg. 2
 * "initial state"; tag 1).  Asynchronous on `stream`.  The scene must outlive
 * the chains.  The first chain set created on a device also sets up the fixed
 * scratch array of jr_advance_static there (10,027,264 bytes, once per
 * device, held until the process exits).  Errors: JR_ERR_INVALID_ARG (sizes,
 * depth > JR_MAX_DEPTH, c_tilde <= 0, sigma <= 0, chain ids beyond 2^32),
 * JR_ERR_OOM. */
jr_status jr_chains_create(const jr_scene* scene, const jr_params* params, void* stream, jr_chains** out);
void jr_chains_destroy(jr_chains* chains);

/* Advance every chain by n_steps iterations of Alg. 2 (Section 7.2): clocks
 * t1 ~ Exp(1), t2 ~ Exp(k(x)); splat (dt, x) into the framebuffer; local MH
 * move if t1 < t2, else regenerate from mu and count a tour.  One persistent
 * launch; then the FP32 framebuffer is folded into the FP64 accumulator.
 * Asynchronous.  n_steps = 0 is a no-op.  Errors: JR_ERR_INVALID_ARG. */
jr_status jr_advance(jr_chains* chains, uint32_t n_steps, void* stream);

/* As jr_advance, and also write one record per (chain, step) into caller
 * device buffers laid out [chain][step] (n_chains x n_steps):
 *   flags: bit0 = the regeneration branch was taken, bit1 = a local proposal
 *          was accepted;  dt: the splatted holding time (0 if nothing was
 *          splatted);  pix: y*W + x of the splat, or -1.
 *   JR_FLAG_MH: bit0 = a large-step proposal, bit1 = the proposal was
 *          accepted; dt = 1 where the held state was splatted.
 * Any of the three pointers may be NULL. */
jr_status jr_advance_traced(jr_chains* chains, uint32_t n_steps, uint8_t* flags_dev, float* dt_dev,
                            int32_t* pix_dev, void* stream);

/* jr_advance with device timing per kernel class: an event is recorded after
 * every launch and the time since the previous one is charged to that launch's
 * class; ms_out[k] / launches_out[k] (host, 4 each) for k = 0 step kernels,
 * 1 path kernels (tracing and shading whole paths), 2 reserved (always 0),
 * 3 flow kernels (the megakernel counts as one step launch).  Same
 * chains and results as jr_advance; the events add a little time between
 * launches, so use it to split a step, not to time it.  Synchronises. */
jr_status jr_advance_timed(jr_chains* chains, uint32_t n_steps, double ms_out[4], uint64_t launches_out[4],
                           void* stream);

/* As jr_advance, with the instrumented kernel variant that also counts the
 * work it does: work_out = {ray casts, BVH node visits, ray/triangle tests}
 * summed over every chain and step.  The chains advance exactly as with
 * jr_advance (same Philox streams, same results).  Synchronises `stream`. */
jr_status jr_advance_counted(jr_chains* chains, uint32_t n_steps, uint64_t work_out[3], void* stream);

/* Threads per block of the megakernel for this chain set: a multiple of 32
 * in [32, 256] (default 128).  Results do not depend on it. */
jr_status jr_set_block_size(jr_chains* chains, uint32_t block);

/* Execution mode of jr_advance for this chain set (jr_advance_traced and
 * jr_advance_counted always use the megakernel):
 *   JR_EXEC_MEGAKERNEL  one thread per chain for the whole launch;
 *   JR_EXEC_WAVEFRONT   a step launch over all chains and a persistent path
 *                       launch per step; a lane traces whole paths and takes
 *                       a new one from the step's queue when its path ends
 *                       (better SIMD use for many chains with uneven path
 *                       lengths; its buffers, about (4 D + 38) bytes per
 *                       chain, are allocated by the first wavefront advance);
 *   JR_EXEC_WARP        one warp per chain for the whole launch: a lane holds
 *                       one coordinate and draws its own random numbers, and a
 *                       ray tests every triangle of the scene in parallel
 *                       (triangle k in lane k mod 32) before a warp reduction
 *                       picks the closest hit; for scenes of a few dozen
 *                       triangles and few chains, where one thread per chain is
 *                       bound by the latency of its serial steps; chain sets
 *                       with a flow run in the wavefront instead;
 *   JR_EXEC_AUTO        wavefront from 2^18 chains up; below that, one warp per
 *                       chain for scenes of at most 128 triangles and fewer
 *                       than 32 chains per SM (4 864 on a 152-SM GB300), else
 *                       the megakernel.
 * All modes run the same per-chain arithmetic on the same Philox streams and
 * give the same closest hits (the least (t, original triangle index) with
 * t > 0). */
#define JR_EXEC_AUTO 0u
#define JR_EXEC_MEGAKERNEL 1u
#define JR_EXEC_WAVEFRONT 2u
#define JR_EXEC_WARP 3u
jr_status jr_set_execution(jr_chains* chains, uint32_t mode);

/* jr_advance without any device allocation -- the paper has no counterpart;
 * this is a service of the library for callers that cannot allocate device
 * memory when they advance: code that runs inside a host framework that owns
 * all device memory (plugin interfaces whose execute step must not allocate),
 * or a loop that cannot afford cudaMalloc/cudaFree, which take the allocator's
 * locks and (cudaFree) synchronise the whole device.
 *
 * It runs the wavefront launches of jr_advance (JR_EXEC_WAVEFRONT), with the
 * same results, but their scratch (second state buffer, F records and
 * queues) lives in one fixed device array inside the library, sized for at
 * most JR_STATIC_MAX_CHAINS chains of any depth (D <= 32, which
 * jr_chains_create already enforces): 10,027,264 bytes.  The CUDA runtime
 * loads the array's module on a device lazily, and loading it allocates the
 * array; jr_chains_create does that (and looks up the array's device address
 * for the device then current), so the array is allocated on every device on
 * which a chain set was created, at that point, and held until the process
 * exits.  The chain set (state, framebuffer, accumulator, counters) is the
 * caller's, created beforehand with jr_chains_create on the same device.
 * jr_advance_static itself calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Every call shares the one array and it keeps the last call's contents: the
 * call clears what must start at zero, but calls whose work overlaps on the
 * GPU (other streams, other threads, other chain sets) race on it -- order
 * them on one stream.  The cached device address does not survive a reset of
 * the device (cudaDeviceReset or a lost primary context): the library's
 * handles and this address are then invalid, and the process must not use the
 * library again.
 * Errors: JR_ERR_INVALID_ARG for a null handle or more than
 * JR_STATIC_MAX_CHAINS chains; JR_ERR_STATE for chains with a flow attached
 * (they advance with jr_advance); in both cases nothing is launched.
 * JR_ERR_CUDA for a failed launch. */
#define JR_STATIC_MAX_CHAINS 65536u
jr_status jr_advance_static(jr_chains* chains, uint32_t n_steps, void* stream);

/* Resolve the estimate (Section 6.3): rgb_out[H][W][3] = accumulator / J
 * (zeros while J = 0); with JR_FLAG_MH, b_hat accumulator / N (see JR_FLAG_MH;
 * zeros before the first large step or the end of the burn-in).
 * out_is_device = 1: rgb_out is device memory and the call is asynchronous;
 * 0: host memory, the call synchronises `stream`. */
jr_status jr_resolve(jr_chains* chains, float* rgb_out, int out_is_device, void* stream);

/* Raw FP64 accumulator, out[H][W][4] = (sum of c~ dt W H F / p per channel,
 * sum of dt in the pixel), for batch statistics and shard reductions (MH: the
 * sum of W H F / p and the number of splatted iterations).  Same device/host
 * convention as jr_resolve. */
jr_status jr_get_accumulator(jr_chains* chains, double* out, int out_is_device, void* stream);

/* Counters and status word; synchronises `stream`.  Returns JR_ERR_NUMERIC or
 * JR_ERR_WATCHDOG (with the stats filled in) if the status word is non-zero. */
jr_status jr_get_stats(jr_chains* chains, jr_stats* out, void* stream);

/* Chain state in SoA layout: x_out[d][chain] (D x n_chains float) and
 * fpu_out[j][chain] (5 x n_chains float: F.r, F.g, F.b, p, u).  Host buffers;
 * synchronises `stream`.  Either pointer may be NULL. */
jr_status jr_get_state(jr_chains* chains, float* x_out, float* fpu_out, void* stream);

/* Overwrite the chain state (same layout, host buffers; every x in [0,1)).
 * fpu_in (the cached F, p, u of jr_get_state) may be NULL, in which case F, p
 * and u are re-evaluated on the device.  A checkpoint restored with
 * jr_set_state(x, fpu) + jr_set_counters continues bit-identically, because
 * the Philox counters depend only on (seed, chain id, step index).
 * Synchronises `stream`. */
jr_status jr_set_state(jr_chains* chains, const float* x_in, const float* fpu_in, void* stream);

/* Restore the per-set counters and step index of a checkpoint (host values). */
jr_status jr_set_counters(jr_chains* chains, const jr_stats* in, const double* accumulator_host, void* stream);

/* Evaluate the integrand and the Restore quantities for n given states
 * (Section 6.2 killing rate; Section 4 target density): device buffers,
 * x_dev[d][i] (D x n float, SoA) in; F_dev[c][i] (3 x n), p_dev, u_dev,
 * k_dev (n each; k = +inf where p = 0) out; hit_ids_dev[v][i]
 * ((max_depth+1) x n int32, -1 = no hit / not cast) optional (NULL).
 * Uses params->max_depth and c_tilde only.  Asynchronous. */
jr_status jr_eval_states(const jr_scene* scene, const jr_params* params, const float* x_dev, uint64_t n,
                         float* F_dev, float* p_dev, float* u_dev, float* k_dev, int32_t* hit_ids_dev,
                         void* stream);

/* Plain Monte Carlo path tracing (the regeneration-only special case c~ ->
 * inf of Section 6.3): samples sample_begin .. +n_samples (tag 2), each
 * adding W H F(x) to channels 0..2 of accum_dev[H][W][4] (device, FP64,
 * caller-owned, added to; channel 3 is not touched).  Pixel estimate =
 * accum / total samples.  Asynchronous. */
jr_status jr_render_pt(const jr_scene* scene, const jr_params* params, uint64_t sample_begin, uint64_t n_samples,
                       double* accum_dev, void* stream);

/* F and its gradient for given states (the gradient of JR_FLAG_MALA's drift):
 * x_dev [D][n] (device, SoA) in; F_dev [3][n] and dF_dev [3][D][n] (dF_dev[(c
 * D + d) n + i] = dF_c / dx_d of state i) out, either may be NULL.  Uses
 * params->max_depth only.  Asynchronous. */
jr_status jr_eval_grad(const jr_scene* scene, const jr_params* params, const float* x_dev, uint64_t n, float* F_dev,
                       float* dF_dev, void* stream);

/* Measured FP32 throughput of the current device, the denominator of the
 * path kernels' ALU roofline (the method has no part in it): a kernel of 8
 * independent FMA chains per thread on every SM at full occupancy, 2^21 FMA
 * per thread; *tflops_out = 2 x FMAs / the best of four launch times (CUDA
 * events on `stream`, each launch after an untimed one), ms_out (may be NULL)
 * that time.  Synchronises `stream`. */
jr_status jr_fp32_peak(double* tflops_out, double* ms_out, void* stream);

/* Raw Philox4x32-10 blocks for chains chain_begin .. +n at one (tag, block,
 * step): out_dev[i][4] uint32 (device).  For bit-exact RNG parity tests. */
jr_status jr_philox(uint64_t seed, uint32_t tag, uint32_t block, uint64_t chain_begin, uint64_t step, uint64_t n,
                    uint32_t* out_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Batches: many chain sets -- scenes of uneven size, images, depths -- advanced
 * by ONE persistent launch.  Blocks of the launch take work items (a block of
 * chains of one set) from a global cursor; items are ordered by estimated cost
 * (depth + 1) x log2(triangles), longest first.  Or, with JR_BATCH_WAVEFRONT,
 * by shared wavefront launches over all the sets.  Every set advances as
 * jr_advance would advance it on its own (same Philox streams, same
 * per-chain arithmetic; Alg. 2 of Section 7.2 per chain): the same states,
 * with F and p equal up to the rounding of separately compiled kernels (one
 * may contract a multiply-add into an FMA where the other does not).  The sets stay owned
 * by the caller and must outlive the batch; a set may still be advanced,
 * resolved or inspected on its own between batch advances.
 * Sets with a learned regeneration flow attached (jr_chains_set_flow, before or
 * after jr_batch_create) advance in the batched wavefront only: their flow
 * draws and density rows are queued per set by the shared launches and their
 * flow launches run between them.  A batch holding such a set selects
 * JR_BATCH_WAVEFRONT; another block size is then refused with JR_ERR_STATE.
 * Changing a set's flow re-captures the batch's graph on its next replay.
 */
typedef struct jr_batch jr_batch;

typedef struct {
    uint32_t n;                   /* candidates tried */
    uint32_t block[8];            /* chains per work item (= threads per block), or JR_BATCH_WAVEFRONT */
    double ns_per_chain_step[8];  /* measured device time per chain step */
    uint32_t best_block;          /* the candidate now in use */
} jr_tune_report;

/* jr_batch_set_block value that selects the batched wavefront: every set's
 * chains take part in the same step and path launches (whole paths per lane
 * with dynamic fetch, as JR_EXEC_WAVEFRONT for one set) over one device copy
 * of all the sets' scenes, merged when the batch first uses it (each distinct
 * scene once; at most 1024 sets, 2^28 triangles, 2^31 chains).  Every set
 * also gets its wavefront buffers.  n_steps steps take 2 n_steps + 2 launches
 * (plus one 4-byte memset per step).  The set-up fails with
 * JR_ERR_INVALID_ARG beyond those limits (the batch itself stays usable with
 * a megakernel block size). */
#define JR_BATCH_WAVEFRONT 0u

/* Build a batch over n_sets distinct chain sets (device descriptors, work
 * items, one set-up launch).  Synchronises `stream`. */
jr_status jr_batch_create(jr_chains* const* sets, uint32_t n_sets, void* stream, jr_batch** out);
void jr_batch_destroy(jr_batch* batch);

/* Chains per work item (= threads per block): a multiple of 32 in [32, 256];
 * or JR_BATCH_WAVEFRONT. */
jr_status jr_batch_set_block(jr_batch* batch, uint32_t block);

/* Advance every set of the batch by n_steps: one persistent launch plus one
 * fold launch for all sets (the batched wavefront: its launches, then the
 * fold).  Asynchronous, except the batched wavefront's one-time set-up. */
jr_status jr_batch_advance(jr_batch* batch, uint32_t n_steps, void* stream);

/* As jr_batch_advance, replayed from a CUDA graph that holds its launches
 * (two; the batched wavefront's 2 n_steps + 2 and their memsets), captured on
 * the first call and again whenever n_steps or the block size changes.  The
 * step indices live on the device, so every replay continues the chains.
 * Asynchronous after the first capture. */
jr_status jr_batch_advance_graph(jr_batch* batch, uint32_t n_steps, void* stream);

/* Autotuner: time probe_steps chain steps of the whole batch for each work-item
 * size in {32, 64, 128, 256} and for JR_BATCH_WAVEFRONT (CUDA events on
 * `stream`; the wavefront only for at most 1024 sets) and keep the fastest.
 * The probes are real steps: every set advances by n x probe_steps, n the
 * number of candidates.  Synchronises `stream`. */
jr_status jr_batch_autotune(jr_batch* batch, uint32_t probe_steps, void* stream, jr_tune_report* out);

/* ---------------------------------------------------------------------------
 * Learned regeneration (not in the paper; the library's addition).  A chain set
 * may regenerate from the mixture mu = beta mu_flow + (1 - beta) uniform, whose
 * density u = beta q + (1 - beta) enters the killing rate k = c~ u / p of
 * Section 6.2 exactly: q is the change-of-variables density of a normalizing
 * flow on [0,1)^D (or on the leading D' < D coordinates, the rest uniform: see
 * jr_chains_set_flow).  The flow: JR_FLOW_LAYERS coupling layers; layer l
 * conditions on x[perm[l][0 .. D/2)] and maps each x[perm[l][D/2 + j]] through
 * a piecewise-linear CDF of JR_FLOW_BINS bins (Mueller et al., "Neural
 * Importance Sampling", 2019) with bin masses Q = (1 - 1e-3) softmax(o) +
 * 1e-3 / JR_FLOW_BINS from an MLP o = W3 relu(W2 relu(W1 x_A + b1) + b2) + b3
 * (hidden width JR_FLOW_HIDDEN; bf16 tensor-core operands, FP32 accumulation).
 *
 * Parameter layout (float32, JR_FLOW_LAYERS consecutive layers of
 * S = 64*16 + 64 + 64*64 + 64 + (D/2)*16*64 + (D/2)*16 floats): W1 [64][16]
 * (columns >= D/2 zero), b1 [64], W2 [64][64], b2 [64], W3 [(D/2)*16][64]
 * (row j*16 + b: bin b of transformed coordinate j), b3 [(D/2)*16].
 * perm: int32 [JR_FLOW_LAYERS][D], each row a permutation of 0..D-1.
 */
#define JR_FLOW_LAYERS 6
#define JR_FLOW_HIDDEN 64
#define JR_FLOW_BINS 16
typedef struct jr_flow jr_flow;

/* Floats of the parameter array for dimension `dim` (0 if dim is not even in
 * 2..32). */
uint64_t jr_flow_param_count(uint32_t dim);

/* Create a flow from host arrays (copied); synchronises `stream`. */
jr_status jr_flow_create(uint32_t dim, const int32_t* perm, const float* params, void* stream, jr_flow** out);
void jr_flow_destroy(jr_flow* flow);
/* Replace / read the FP32 parameters (host arrays, the layout above). */
jr_status jr_flow_set_params(jr_flow* flow, const float* params, void* stream);
jr_status jr_flow_get_params(jr_flow* flow, float* params, void* stream);
/* JR_STATUS_* bits (sticky) of the flow's own jr_flow_log_density /
 * jr_flow_sample launches; launches made for a chain set report to that set's
 * status word instead.  Synchronises. */
jr_status jr_flow_get_status(jr_flow* flow, uint32_t* status_out, void* stream);

/* log q(x) for n rows of x_dev [D][n] (device, SoA) into lq_dev [n].  Async. */
jr_status jr_flow_log_density(jr_flow* flow, const float* x_dev, uint64_t n, float* lq_dev, void* stream);
/* In place: rows z of xz_dev [D][n] in [0,1)^D become x = T^{-1}(z); lq_dev
 * [n] gets log q(x).  Async. */
jr_status jr_flow_sample(jr_flow* flow, float* xz_dev, uint64_t n, float* lq_dev, void* stream);

/* Copy perm and parameters of src into dst (same D) on the device. */
jr_status jr_flow_copy_params(jr_flow* dst, const jr_flow* src, void* stream);

/* Training rows from the chains' current states: x_dev [D][n_chains] (device)
 * gets the states, w_dev [n_chains] the weights p / (p + c~ u) = E[dt | x],
 * the expected holding time of Alg. 2, so that the weighted states follow pi
 * (the states themselves follow the jump chain's law, proportional to
 * p + c~ u).  Call between advances (the states are then in x).  Async. */
jr_status jr_chains_snapshot(jr_chains* chains, float* x_dev, float* w_dev, void* stream);

/* The same rows, keeping only those of weight > 0 (states with p > 0), appended
 * to a ring buffer of `capacity` rows: x_ring [D][capacity], w_ring [capacity]
 * (device, caller-owned).  *total_dev (device, caller-owned, start at 0) counts
 * every row ever appended; row r lands in slot r % capacity, so the buffer
 * holds min(total, capacity) rows, in slots [0, min(total, capacity)).  The
 * order of rows within one call is unspecified.  Async. */
jr_status jr_chains_snapshot_append(jr_chains* chains, float* x_ring, float* w_ring, uint64_t capacity,
                                    unsigned long long* total_dev, void* stream);

/* Time-weighted maximum likelihood: the loss -sum_r w_r log q(x_r) / sum_r w_r
 * over rows [off, off + batch) of x_dev [D][n], w_dev [n] (device), and its
 * gradient w.r.t. the parameters (host, jr_flow_param_count floats, the layout
 * above).  bf16 roundings pass gradients straight through.  Synchronises. */
jr_status jr_flow_gradient(jr_flow* flow, const float* x_dev, const float* w_dev, uint64_t n, uint64_t off,
                           uint32_t batch, float* grad_host, float* loss_host, void* stream);

/* iters Adam steps (lr; beta 0.9 / 0.999) of the same loss on minibatches of
 * `batch` rows (a multiple of 64) at pseudo-random offsets (seed); the packed
 * bf16 weights follow every step, so train a flow that no chain set is using.
 * loss_host (may be NULL) gets the loss of every step.  Synchronises. */
jr_status jr_flow_train(jr_flow* flow, const float* x_dev, const float* w_dev, uint64_t n, uint32_t iters,
                        uint32_t batch, float lr, uint64_t seed, float* loss_host, void* stream);
/* The same on the first n_rows rows of x_dev [D][stride], w_dev [stride] (a
 * partly filled jr_chains_snapshot_append ring): minibatches are windows of
 * `batch` rows inside [0, n_rows); batch <= n_rows <= stride.  Synchronises. */
jr_status jr_flow_train_rows(jr_flow* flow, const float* x_dev, const float* w_dev, uint64_t stride,
                             uint64_t n_rows, uint32_t iters, uint32_t batch, float lr, uint64_t seed,
                             float* loss_host, void* stream);

/* Complete every chain's current tour, then start every chain on a new tour.
 * The estimator of Section 6.3 divides by J, the number of completed tours;
 * a run stopped after a fixed number of steps leaves one unfinished tour per
 * chain whose splats are not matched in J (a bias of order chains / J whose
 * size depends on mu).  Here the chains still inside a tour keep stepping
 * (regular Alg. 2 steps, counted in the step index) and a kill ends the tour
 * and the chain, for at most max_steps steps; `remaining` (may be NULL) gets
 * the chains whose tour is still open after them (0: every tour completed, and
 * the accumulated image is the completed-tour estimator).  Then each chain
 * starts a new tour from mu (Philox tag 3, keyed by a restart count; not a
 * regeneration).  Wavefront mode; synchronises `stream` once per drain step. */
jr_status jr_complete_tours(jr_chains* chains, uint32_t max_steps, uint64_t* remaining, void* stream);

/* Attach a flow (or detach with flow = NULL) with mixture weight beta in
 * [0, 1): first the current tours are completed under the old mu (as in
 * jr_complete_tours, at most max_drain_steps steps), then every chain starts a
 * new tour from the new mu.  So no tour mixes two regeneration densities.  The
 * flow's dimension D' is the chains' D, or 4 <= D' < D: the flow then models
 * the leading D' coordinates and the others stay uniform, mu_flow(x) =
 * q(x[0 .. D')) and u = beta q(x[0 .. D')) + 1 - beta (a flow draw maps the
 * first D' of the step's uniforms through the flow and keeps the rest).  The
 * flow must outlive its use; chains with a flow advance in the wavefront mode
 * (jr_advance only).  Errors: JR_ERR_INVALID_ARG (null chains, D' not D and
 * not in 4 .. D - 1, beta outside [0, 1)), JR_ERR_STATE (MH or MALA chains). */
jr_status jr_chains_set_flow(jr_chains* chains, const jr_flow* flow, float beta, uint32_t max_drain_steps,
                             uint64_t* remaining, void* stream);

/* ---------------------------------------------------------------------------
 * Failure detection and its testing hooks (the paper has no counterpart).  The
 * device reports the method's faults in the status word (JR_STATUS_*), which
 * jr_get_stats turns into JR_ERR_WATCHDOG / JR_ERR_NUMERIC; these calls let a
 * test provoke each failure from the host, without faulting the device.
 */

/* Traversal limits of this chain set's launches: a ray that visits more than
 * node_visit_budget BVH nodes, or whose stack would hold more than
 * stack_entries entries (<= 96), stops and counts as a miss, and the set's
 * status word gets JR_STATUS_TRAVERSAL or JR_STATUS_STACK.  0 keeps the
 * default (2^16 visits; 96 entries, which the BVH builder guarantees is never
 * exceeded).  Errors: JR_ERR_INVALID_ARG for stack_entries > 96. */
jr_status jr_chains_set_limits(jr_chains* chains, uint32_t node_visit_budget, uint32_t stack_entries);

/* The library's (n+1)-th device allocation from now fails as if the device were
 * out of memory (n >= 0; n < 0 switches the hook off).  The call that meets it
 * returns JR_ERR_OOM, frees what it had allocated and leaves its outputs
 * untouched.  Process-wide; for tests. */
jr_status jr_debug_fail_alloc(int64_t n);

/* enable != 0: this flow's own launches (jr_flow_log_density, jr_flow_sample)
 * arm their first weight barrier for 16 bytes more than the copy delivers, so
 * the kernel's bounded wait (2 s) runs out: it sets JR_STATUS_FLOW_WAIT,
 * waits (bounded) for its copies in flight and returns without writing its
 * outputs.  For tests of that path; 0 switches it off. */
jr_status jr_debug_flow_wait(jr_flow* flow, int enable);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* jr_last_error(void);
/* Library version string. */
const char* jr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* JR_H */
