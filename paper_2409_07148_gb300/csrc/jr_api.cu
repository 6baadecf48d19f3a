// Host runtime behind the C ABI of include/jr.h: argument checks, device
// memory for scenes and chain sets, launch sequencing, error reporting.  No
// exception or abort crosses the ABI; every failure becomes a jr_status and a
// thread-local message.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/jr.h"
#include "jr_internal.h"

using namespace jr;

namespace {

thread_local std::string g_err;

jr_status fail(jr_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

jr_status cuda_fail(cudaError_t e, const char* what) {
    (void)cudaGetLastError();  // clear a sticky launch error so later calls see a clean slate
    return fail(e == cudaErrorMemoryAllocation ? JR_ERR_OOM : JR_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define JR_CUDA(call, what)                      \
    do {                                         \
        cudaError_t e_ = (call);                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Testing hook (jr_debug_fail_alloc): when >= 0, the number of device
// allocations still to succeed before one fails with cudaErrorMemoryAllocation.
std::atomic<long long> g_fail_alloc_in{-1};

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
    long long k = g_fail_alloc_in.load();
    while (k >= 0 && !g_fail_alloc_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) return cudaErrorMemoryAllocation;
    return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

}  // namespace

struct jr_scene {
    Bvh4Node* nodes = nullptr;
    TriRecord* tris = nullptr;
    Material* mats = nullptr;
    SceneView view{};
    jr_scene_info info{};
    ~jr_scene() {
        cudaFree(nodes);
        cudaFree(tris);
        cudaFree(mats);
    }
};

struct jr_chains {
    const jr_scene* scene = nullptr;
    jr_params params{};
    ChainView view{};
    uint64_t steps = 0;
    int block = 128;
    uint32_t exec = JR_EXEC_AUTO;
    uint64_t epochs = 0;  // restarts from a new regeneration distribution (Philox tag 3 key)
    uint64_t flow_gen = 0;      // bumped whenever the attached flow (or its weight) changes
    uint32_t visit_budget = 0;  // traversal watchdog limits of this set's launches (0: the scene's)
    int stack_limit = 0;
    // The scene as this set's launches see it (with the set's traversal limits).
    SceneView scene_view() const {
        SceneView v = scene->view;
        if (visit_budget) v.visit_budget = visit_budget;
        if (stack_limit) v.stack_limit = stack_limit;
        return v;
    }
    ~jr_chains() {
        cudaFree(view.wf.y);
        cudaFree(view.wf.par);
        cudaFree(view.wf.ua);
        cudaFree(view.wf.fy);
        cudaFree(view.wf.uy);
        cudaFree(view.wf.fq);
        cudaFree(view.wf.done);
        cudaFree(view.wf.queue);
        cudaFree(view.wf.qcount);
        cudaFree(view.x);
        cudaFree(view.fpu);
        cudaFree(view.fb);
        cudaFree(view.acc64);
        cudaFree(view.counters);
        cudaFree(view.status);
        cudaFree(view.drift);
    }
};

// Post-burn-in iterations of an MH chain set over all chains (the N of its estimator).
static uint64_t mh_samples(const jr_chains* c) {
    if (!(c->view.flags & JR_FLAG_MH)) return 0;
    return c->steps > c->view.burn_in ? (c->steps - c->view.burn_in) * c->view.n : 0;
}

extern "C" {

const char* jr_last_error(void) { return g_err.c_str(); }

const char* jr_version(void) { return "jr-gb300 0.1 (sm_103a)"; }

jr_status jr_scene_create(const jr_scene_desc* desc, void* stream, jr_scene** out) {
    if (!desc || !out) return fail(JR_ERR_INVALID_ARG, "jr_scene_create: null argument");
    if (desc->n_tris > 0 && (!desc->verts || !desc->tris || !desc->tri_material))
        return fail(JR_ERR_INVALID_ARG, "jr_scene_create: null triangle arrays");
    if (desc->n_materials == 0 || !desc->materials)
        return fail(JR_ERR_INVALID_ARG, "jr_scene_create: at least one material is required");
    for (uint32_t t = 0; t < desc->n_tris; ++t)
        if (desc->tri_material[t] >= desc->n_materials)
            return fail(JR_ERR_INVALID_ARG, "jr_scene_create: triangle material index out of range");
    std::vector<Material> mats(desc->n_materials);
    for (uint32_t m = 0; m < desc->n_materials; ++m) {
        const float* r = desc->materials + (size_t)JR_MATERIAL_FLOATS * m;
        Material& q = mats[m];
        q.type = (int)r[0];
        if (r[0] != (float)q.type || q.type < JR_MAT_LAMBERT || q.type > JR_MAT_DIELECTRIC)
            return fail(JR_ERR_INVALID_ARG, "jr_scene_create: unknown material type");
        q.albedo = make_float3(r[1], r[2], r[3]);
        q.emission = make_float3(r[4], r[5], r[6]);
        q.emits = (r[4] != 0.f || r[5] != 0.f || r[6] != 0.f);
        q.phong_inv_n1 = 1.0f / (r[7] + 1.0f);
        q.phong_scale = (r[7] + 2.0f) / (r[7] + 1.0f);
        q.ior = r[8];
        q.pad = 0.f;
        if (q.type == JR_MAT_PHONG && !(r[7] >= 0.f)) return fail(JR_ERR_INVALID_ARG, "jr_scene_create: Phong n < 0");
        if (q.type == JR_MAT_DIELECTRIC && !(r[8] > 0.f)) return fail(JR_ERR_INVALID_ARG, "jr_scene_create: ior <= 0");
    }
    HostBvh bvh;
    std::string err;
    try {
        if (!build_bvh(desc->verts, desc->n_verts, desc->tris, desc->n_tris, desc->tri_material, &bvh, &err))
            return fail(JR_ERR_INVALID_ARG, "jr_scene_create: " + err);
    } catch (const std::bad_alloc&) {
        return fail(JR_ERR_OOM, "jr_scene_create: host allocation failed in the BVH build");
    } catch (const std::exception& ex) {
        return fail(JR_ERR_INVALID_ARG, std::string("jr_scene_create: BVH build failed: ") + ex.what());
    }
    jr_scene* s = new (std::nothrow) jr_scene();
    if (!s) return fail(JR_ERR_OOM, "jr_scene_create: host allocation failed");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = dev_alloc(&s->nodes, bvh.nodes.size())) != cudaSuccess ||
        (e = dev_alloc(&s->tris, bvh.tris.size())) != cudaSuccess ||
        (e = dev_alloc(&s->mats, mats.size())) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->nodes, bvh.nodes.data(), sizeof(Bvh4Node) * bvh.nodes.size(), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->tris, bvh.tris.data(), sizeof(TriRecord) * bvh.tris.size(), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->mats, mats.data(), sizeof(Material) * mats.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        delete s;
        return cuda_fail(e, "jr_scene_create");
    }
    s->view.nodes = s->nodes;
    s->view.tris = s->tris;
    s->view.mats = s->mats;
    s->view.root = bvh.root;
    s->view.n_nodes = (int)bvh.nodes.size();
    s->view.n_tris = (uint32_t)bvh.tris.size();
    s->view.visit_budget = kNodeVisitBudget;
    s->view.stack_limit = kStackSize;
    std::memcpy(s->view.cam, desc->camera, sizeof(float) * 12);
    s->info.n_tris = desc->n_tris;
    s->info.n_nodes = (uint32_t)bvh.nodes.size();
    s->info.bvh_depth = (uint32_t)bvh.depth;
    s->info.n_materials = desc->n_materials;
    s->info.device_bytes =
        sizeof(Bvh4Node) * bvh.nodes.size() + sizeof(TriRecord) * bvh.tris.size() + sizeof(Material) * mats.size();
    *out = s;
    return JR_OK;
}

jr_status jr_scene_get_info(const jr_scene* scene, jr_scene_info* out) {
    if (!scene || !out) return fail(JR_ERR_INVALID_ARG, "jr_scene_get_info: null argument");
    *out = scene->info;
    return JR_OK;
}

void jr_scene_destroy(jr_scene* scene) { delete scene; }

static jr_status check_params(const jr_params* p, const char* who) {
    if (!p) return fail(JR_ERR_INVALID_ARG, std::string(who) + ": null params");
    if (p->width == 0 || p->height == 0 || (uint64_t)p->width * p->height > (1u << 26))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": image size out of range (1 .. 2^26 pixels)");
    if (p->max_depth > JR_MAX_DEPTH) return fail(JR_ERR_INVALID_ARG, std::string(who) + ": max_depth > 15");
    if (!(p->c_tilde > 0.f) || !std::isfinite(p->c_tilde))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": c_tilde must be finite and > 0");
    if (!(p->sigma > 0.f) || !std::isfinite(p->sigma))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": sigma must be finite and > 0");
    if (p->flags & ~(JR_FLAG_RAO_BLACKWELL | JR_FLAG_MH | JR_FLAG_MALA))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": unknown flag");
    if ((p->flags & JR_FLAG_MALA) && (p->flags & JR_FLAG_RAO_BLACKWELL))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": MALA chains splat the sampled holding time");
    if ((p->flags & JR_FLAG_MH) && (p->flags & JR_FLAG_RAO_BLACKWELL))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": the MH baseline has no holding times to Rao-Blackwellise");
    if ((p->flags & JR_FLAG_MH) && !(p->large_step >= 0.f && p->large_step <= 1.f))
        return fail(JR_ERR_INVALID_ARG, std::string(who) + ": large_step must be in [0, 1]");
    return JR_OK;
}

jr_status jr_chains_create(const jr_scene* scene, const jr_params* params, void* stream, jr_chains** out) {
    if (!scene || !out) return fail(JR_ERR_INVALID_ARG, "jr_chains_create: null argument");
    jr_status ps = check_params(params, "jr_chains_create");
    if (ps != JR_OK) return ps;
    if (params->n_chains == 0) return fail(JR_ERR_INVALID_ARG, "jr_chains_create: n_chains must be >= 1");
    if (params->chain_offset + params->n_chains > (1ull << 32))
        return fail(JR_ERR_INVALID_ARG, "jr_chains_create: chain ids must stay below 2^32");
    jr_chains* c = new (std::nothrow) jr_chains();
    if (!c) return fail(JR_ERR_OOM, "jr_chains_create: host allocation failed");
    c->scene = scene;
    c->params = *params;
    ChainView& v = c->view;
    v.n = params->n_chains;
    v.chain_offset = (uint32_t)params->chain_offset;
    v.width = params->width;
    v.height = params->height;
    v.depth = params->max_depth;
    v.dim = 2 + 2 * params->max_depth;
    v.flags = params->flags;
    v.seed = params->seed;
    v.c_tilde = params->c_tilde;
    v.sigma = params->sigma;
    v.large_step = (params->flags & JR_FLAG_MH) ? params->large_step : 0.f;
    v.burn_in = (params->flags & JR_FLAG_MH) ? params->burn_in : 0;
    const size_t npx = (size_t)params->width * params->height;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = dev_alloc(&v.x, (size_t)v.dim * v.n)) != cudaSuccess || (e = dev_alloc(&v.fpu, 5 * v.n)) != cudaSuccess ||
        (e = dev_alloc(&v.fb, npx)) != cudaSuccess || (e = dev_alloc(&v.acc64, npx)) != cudaSuccess ||
        (e = dev_alloc(&v.counters, kCounters)) != cudaSuccess || (e = dev_alloc(&v.status, 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(v.fb, 0, sizeof(float4) * npx, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(v.acc64, 0, sizeof(double4_32a) * npx, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(v.counters, 0, sizeof(unsigned long long) * kCounters, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(v.status, 0, sizeof(unsigned int), st)) != cudaSuccess ||
        ((v.flags & JR_FLAG_MALA) && (e = dev_alloc(&v.drift, (size_t)v.dim * v.n)) != cudaSuccess) ||
        (e = launch_init(scene->view, v, st)) != cudaSuccess ||
        ((v.flags & JR_FLAG_MALA) && (e = launch_mala_reeval(scene->view, v, st)) != cudaSuccess) ||
        (e = prepare_static_scratch()) != cudaSuccess) {  // jr_advance_static's array, see jr_wavefront.cu
        delete c;
        return cuda_fail(e, "jr_chains_create");
    }
    *out = c;
    return JR_OK;
}

void jr_chains_destroy(jr_chains* chains) { delete chains; }

// Wavefront buffers, allocated on the first wavefront advance of a chain set.
static jr_status ensure_wavefront(jr_chains* c, cudaStream_t st) {
    WaveView& w = c->view.wf;
    if (w.y) return JR_OK;
    const uint64_t n = c->view.n;
    cudaError_t e;
    if ((e = dev_alloc(&w.y, (size_t)c->view.dim * n)) != cudaSuccess || (e = dev_alloc(&w.par, n)) != cudaSuccess ||
        (e = dev_alloc(&w.ua, n)) != cudaSuccess || (e = dev_alloc(&w.fy, n)) != cudaSuccess ||
        (e = dev_alloc(&w.queue, n)) != cudaSuccess ||
        (e = dev_alloc(&w.qcount, kQCount)) != cudaSuccess || (e = dev_alloc(&w.uy, n)) != cudaSuccess ||
        (e = dev_alloc(&w.fq, 2 * n)) != cudaSuccess || (e = dev_alloc(&w.done, n)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.done, 0, n, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.par, 0, n, st)) != cudaSuccess) {
        cudaFree(w.done);
        cudaFree(w.y);
        cudaFree(w.par);
        cudaFree(w.ua);
        cudaFree(w.fy);
        cudaFree(w.queue);
        cudaFree(w.qcount);
        cudaFree(w.uy);
        cudaFree(w.fq);
        w = WaveView{};
        return cuda_fail(e, "jr_advance (wavefront buffers)");
    }
    return JR_OK;
}

// One warp per chain: asked for, or (auto) a small scene with fewer chains
// than 32 per SM -- while one thread per chain would leave the SMs without
// even one warp each (measured on the Cornell box and a depth-6 furnace: one
// chain per warp 6.1x / 2.2x faster at 256 chains, 2.5x / 0.94x at 4 096;
// the megakernel 1.5x / 0.56x ahead at 8 192).  Only for sets without a flow
// (the wavefront takes those).
static bool warp_per_chain(const jr_chains* c) {
    if (c->view.flow.D != 0) return false;
    if (c->exec == JR_EXEC_WARP) return true;
    if (c->exec != JR_EXEC_AUTO || c->scene->view.n_tris > kWarpChainMaxTris) return false;
    static DeviceOnce once;  // per device: its SM count
    long long sms = 0;
    if (once.get(
            [](int dev, long long* v) {
                int n = 0;
                cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
                *v = n;
                return e;
            },
            &sms) != cudaSuccess)
        return false;
    return c->view.n < (uint64_t)(32 * sms);
}

static jr_status advance_impl(jr_chains* c, uint32_t n_steps, uint8_t* f, float* dt, int32_t* pix,
                              unsigned long long* work, void* stream, const char* who) {
    if (!c) return fail(JR_ERR_INVALID_ARG, std::string(who) + ": null chains");
    if (n_steps == 0) return JR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const bool plain = !f && !dt && !pix && !work;
    const bool has_flow = c->view.flow.D != 0;
    if (c->view.flags & JR_FLAG_MALA) {  // Langevin moves: the megakernel only
        if (work) return fail(JR_ERR_STATE, std::string(who) + ": the counted advance does not run MALA chains");
        JR_CUDA(launch_step_mala(c->scene_view(), c->view, c->steps, n_steps, f, dt, pix, st), who);
        JR_CUDA(launch_fold(c->view, st), who);
        c->steps += n_steps;
        return JR_OK;
    }
    if (has_flow && !plain)
        return fail(JR_ERR_STATE, std::string(who) + ": traced and counted advances do not run with a flow attached");
    const bool wave = plain && (has_flow || c->exec == JR_EXEC_WAVEFRONT ||
                                (c->exec == JR_EXEC_AUTO && c->view.n >= kWavefrontMinChains));
    if (wave) {
        jr_status a = ensure_wavefront(c, st);
        if (a != JR_OK) return a;
        JR_CUDA(launch_wavefront(c->scene_view(), c->view, c->steps, n_steps, st), who);
    } else if (plain && warp_per_chain(c)) {
        JR_CUDA(launch_step_warp(c->scene_view(), c->view, c->steps, n_steps, st), who);
    } else {
        JR_CUDA(launch_step(c->scene_view(), c->view, c->steps, n_steps, f, dt, pix, work, c->block, st), who);
    }
    JR_CUDA(launch_fold(c->view, st), who);
    c->steps += n_steps;
    return JR_OK;
}

jr_status jr_advance(jr_chains* chains, uint32_t n_steps, void* stream) {
    return advance_impl(chains, n_steps, nullptr, nullptr, nullptr, nullptr, stream, "jr_advance");
}

jr_status jr_advance_traced(jr_chains* chains, uint32_t n_steps, uint8_t* flags_dev, float* dt_dev,
                            int32_t* pix_dev, void* stream) {
    return advance_impl(chains, n_steps, flags_dev, dt_dev, pix_dev, nullptr, stream, "jr_advance_traced");
}

jr_status jr_advance_timed(jr_chains* c, uint32_t n_steps, double ms_out[4], uint64_t launches_out[4], void* stream) {
    if (!c || !ms_out || !launches_out) return fail(JR_ERR_INVALID_ARG, "jr_advance_timed: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const bool wave = c->view.flow.D != 0 || c->exec == JR_EXEC_WAVEFRONT ||
                      (c->exec == JR_EXEC_AUTO && c->view.n >= kWavefrontMinChains);
    KernelTimer tm;
    if (n_steps > 0 && (c->view.flags & JR_FLAG_MALA)) {
        JR_CUDA(tm.mark(-1, st), "jr_advance_timed");
        JR_CUDA(launch_step_mala(c->scene_view(), c->view, c->steps, n_steps, nullptr, nullptr, nullptr, st),
                "jr_advance_timed");
        JR_CUDA(tm.mark(KernelTimer::kStep, st), "jr_advance_timed");
        JR_CUDA(launch_fold(c->view, st), "jr_advance_timed");
        c->steps += n_steps;
    } else if (n_steps > 0) {
        if (wave) {
            jr_status a = ensure_wavefront(c, st);
            if (a != JR_OK) return a;
            JR_CUDA(launch_wavefront(c->scene_view(), c->view, c->steps, n_steps, st, kModeStep, &tm),
                    "jr_advance_timed");
        } else {
            JR_CUDA(tm.mark(-1, st), "jr_advance_timed");
            if (warp_per_chain(c))
                JR_CUDA(launch_step_warp(c->scene_view(), c->view, c->steps, n_steps, st), "jr_advance_timed");
            else
                JR_CUDA(launch_step(c->scene_view(), c->view, c->steps, n_steps, nullptr, nullptr, nullptr, nullptr,
                                    c->block, st),
                        "jr_advance_timed");
            JR_CUDA(tm.mark(KernelTimer::kStep, st), "jr_advance_timed");
        }
        JR_CUDA(launch_fold(c->view, st), "jr_advance_timed");
        c->steps += n_steps;
    }
    JR_CUDA(cudaStreamSynchronize(st), "jr_advance_timed");
    JR_CUDA(tm.totals(ms_out, launches_out), "jr_advance_timed");
    return JR_OK;
}

jr_status jr_advance_static(jr_chains* chains, uint32_t n_steps, void* stream) {
    if (!chains) return fail(JR_ERR_INVALID_ARG, "jr_advance_static: null chains");
    if (chains->view.n > kStaticMaxChains)
        return fail(JR_ERR_INVALID_ARG, "jr_advance_static: " + std::to_string(chains->view.n) +
                                            " chains exceed the fixed scratch of " +
                                            std::to_string(kStaticMaxChains) + " chains; use jr_advance");
    if (chains->view.flow.D != 0)
        return fail(JR_ERR_STATE, "jr_advance_static: chains with a flow attached advance with jr_advance");
    if (chains->view.flags & JR_FLAG_MALA)
        return fail(JR_ERR_STATE, "jr_advance_static: MALA chains advance with jr_advance (megakernel)");
    if (n_steps == 0) return JR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    JR_CUDA(launch_wavefront_static(chains->scene_view(), chains->view, chains->steps, n_steps, st),
            "jr_advance_static");
    JR_CUDA(launch_fold(chains->view, st), "jr_advance_static");
    chains->steps += n_steps;
    return JR_OK;
}

jr_status jr_set_execution(jr_chains* chains, uint32_t mode) {
    if (!chains) return fail(JR_ERR_INVALID_ARG, "jr_set_execution: null chains");
    if (mode > JR_EXEC_WARP) return fail(JR_ERR_INVALID_ARG, "jr_set_execution: unknown mode");
    chains->exec = mode;
    return JR_OK;
}

jr_status jr_set_block_size(jr_chains* chains, uint32_t block) {
    if (!chains) return fail(JR_ERR_INVALID_ARG, "jr_set_block_size: null chains");
    if (block < 32 || block > 256 || block % 32 != 0)
        return fail(JR_ERR_INVALID_ARG, "jr_set_block_size: block must be a multiple of 32 in [32, 256]");
    chains->block = (int)block;
    return JR_OK;
}

jr_status jr_chains_set_limits(jr_chains* chains, uint32_t node_visit_budget, uint32_t stack_entries) {
    if (!chains) return fail(JR_ERR_INVALID_ARG, "jr_chains_set_limits: null chains");
    if (stack_entries > (uint32_t)kStackSize)
        return fail(JR_ERR_INVALID_ARG, "jr_chains_set_limits: at most " + std::to_string(kStackSize) +
                                            " stack entries");
    chains->visit_budget = node_visit_budget;
    chains->stack_limit = (int)stack_entries;
    return JR_OK;
}

jr_status jr_debug_fail_alloc(int64_t n) {
    g_fail_alloc_in.store(n < 0 ? -1 : (long long)n);
    return JR_OK;
}

jr_status jr_advance_counted(jr_chains* chains, uint32_t n_steps, uint64_t work_out[3], void* stream) {
    if (!chains || !work_out) return fail(JR_ERR_INVALID_ARG, "jr_advance_counted: null argument");
    unsigned long long* w = nullptr;
    JR_CUDA(dev_alloc(&w, 3), "jr_advance_counted");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(w, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
        cudaFree(w);
        return cuda_fail(e, "jr_advance_counted");
    }
    jr_status s = advance_impl(chains, n_steps, nullptr, nullptr, nullptr, w, stream, "jr_advance_counted");
    unsigned long long h[3] = {0, 0, 0};
    if (s == JR_OK) {
        if ((e = cudaMemcpyAsync(h, w, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            cudaFree(w);
            return cuda_fail(e, "jr_advance_counted");
        }
        for (int k = 0; k < 3; ++k) work_out[k] = h[k];
    }
    cudaFree(w);
    return s;
}

jr_status jr_resolve(jr_chains* c, float* rgb_out, int out_is_device, void* stream) {
    if (!c || !rgb_out) return fail(JR_ERR_INVALID_ARG, "jr_resolve: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t npx = (size_t)c->view.width * c->view.height;
    if (out_is_device) {
        JR_CUDA(launch_resolve(c->view, rgb_out, mh_samples(c), st), "jr_resolve");
        return JR_OK;
    }
    float* tmp = nullptr;
    JR_CUDA(dev_alloc(&tmp, 3 * npx), "jr_resolve");
    cudaError_t e;
    if ((e = launch_resolve(c->view, tmp, mh_samples(c), st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rgb_out, tmp, sizeof(float) * 3 * npx, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        cudaFree(tmp);
        return cuda_fail(e, "jr_resolve");
    }
    cudaFree(tmp);
    return JR_OK;
}

jr_status jr_get_accumulator(jr_chains* c, double* out, int out_is_device, void* stream) {
    if (!c || !out) return fail(JR_ERR_INVALID_ARG, "jr_get_accumulator: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double4_32a) * (size_t)c->view.width * c->view.height;
    JR_CUDA(cudaMemcpyAsync(out, c->view.acc64, bytes, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st),
            "jr_get_accumulator");
    if (!out_is_device) JR_CUDA(cudaStreamSynchronize(st), "jr_get_accumulator");
    return JR_OK;
}

jr_status jr_get_stats(jr_chains* c, jr_stats* out, void* stream) {
    if (!c || !out) return fail(JR_ERR_INVALID_ARG, "jr_get_stats: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long cnt[kCounters];
    unsigned int status = 0;
    JR_CUDA(cudaMemcpyAsync(cnt, c->view.counters, sizeof(cnt), cudaMemcpyDeviceToHost, st), "jr_get_stats");
    JR_CUDA(cudaMemcpyAsync(&status, c->view.status, sizeof(status), cudaMemcpyDeviceToHost, st), "jr_get_stats");
    JR_CUDA(cudaStreamSynchronize(st), "jr_get_stats");
    out->steps_per_chain = c->steps;
    out->regenerations = cnt[0];
    out->local_steps = cnt[1];
    out->accepted = cnt[2];
    out->status_word = status;
    out->dim = c->view.dim;
    std::memcpy(&out->p_sum_large, &cnt[kCounterPSum], sizeof(double));
    if (status & (JR_STATUS_TRAVERSAL | JR_STATUS_STACK))
        return fail(JR_ERR_WATCHDOG, "jr_get_stats: a ray exhausted the traversal budget or stack");
    if (status & JR_STATUS_NONFINITE) return fail(JR_ERR_NUMERIC, "jr_get_stats: non-finite path contribution");
    return JR_OK;
}

jr_status jr_get_state(jr_chains* c, float* x_out, float* fpu_out, void* stream) {
    if (!c) return fail(JR_ERR_INVALID_ARG, "jr_get_state: null chains");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t n = c->view.n, D = c->view.dim;
    std::vector<float> pairs;
    if (x_out) {  // the device keeps coordinate pairs (xidx); the caller gets [D][n]
        try {
            pairs.resize((size_t)D * n);
        } catch (const std::bad_alloc&) {
            return fail(JR_ERR_OOM, "jr_get_state: host allocation failed");
        }
        JR_CUDA(cudaMemcpyAsync(pairs.data(), c->view.x, sizeof(float) * D * n, cudaMemcpyDeviceToHost, st),
                "jr_get_state");
    }
    if (fpu_out)
        JR_CUDA(cudaMemcpyAsync(fpu_out, c->view.fpu, sizeof(float) * 5 * n, cudaMemcpyDeviceToHost, st),
                "jr_get_state");
    JR_CUDA(cudaStreamSynchronize(st), "jr_get_state");
    if (x_out)
        for (uint32_t d = 0; d < D; ++d)
            for (uint64_t i = 0; i < n; ++i) x_out[d * n + i] = pairs[xidx(d, i, n)];
    return JR_OK;
}

jr_status jr_set_state(jr_chains* c, const float* x_in, const float* fpu_in, void* stream) {
    if (!c || !x_in) return fail(JR_ERR_INVALID_ARG, "jr_set_state: null argument");
    for (uint64_t k = 0; k < (uint64_t)c->view.dim * c->view.n; ++k)
        if (!(x_in[k] >= 0.0f && x_in[k] < 1.0f)) return fail(JR_ERR_INVALID_ARG, "jr_set_state: x outside [0,1)");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t n = c->view.n, D = c->view.dim;
    std::vector<float> pairs;
    try {
        pairs.resize((size_t)D * n);
    } catch (const std::bad_alloc&) {
        return fail(JR_ERR_OOM, "jr_set_state: host allocation failed");
    }
    for (uint32_t d = 0; d < D; ++d)
        for (uint64_t i = 0; i < n; ++i) pairs[xidx(d, i, n)] = x_in[d * n + i];
    JR_CUDA(cudaMemcpyAsync(c->view.x, pairs.data(), sizeof(float) * D * n, cudaMemcpyHostToDevice, st),
            "jr_set_state");
    if (c->view.flags & JR_FLAG_MALA)  // F, p and the drift from the states themselves
        JR_CUDA(launch_mala_reeval(c->scene_view(), c->view, st), "jr_set_state");
    else if (fpu_in)
        JR_CUDA(cudaMemcpyAsync(c->view.fpu, fpu_in, sizeof(float) * 5 * c->view.n, cudaMemcpyHostToDevice, st),
                "jr_set_state");
    else
        JR_CUDA(launch_reeval(c->scene_view(), c->view, st), "jr_set_state");
    JR_CUDA(cudaStreamSynchronize(st), "jr_set_state");
    return JR_OK;
}

jr_status jr_set_counters(jr_chains* c, const jr_stats* in, const double* acc_host, void* stream) {
    if (!c || !in) return fail(JR_ERR_INVALID_ARG, "jr_set_counters: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long cnt[kCounters] = {in->regenerations, in->local_steps, in->accepted, 0, 0, 0, 0, 0};
    std::memcpy(&cnt[kCounterPSum], &in->p_sum_large, sizeof(double));
    unsigned int status = in->status_word;
    JR_CUDA(cudaMemcpyAsync(c->view.counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice, st), "jr_set_counters");
    JR_CUDA(cudaMemcpyAsync(c->view.status, &status, sizeof(status), cudaMemcpyHostToDevice, st), "jr_set_counters");
    if (acc_host)
        JR_CUDA(cudaMemcpyAsync(c->view.acc64, acc_host, sizeof(double4_32a) * (size_t)c->view.width * c->view.height,
                                cudaMemcpyHostToDevice, st),
                "jr_set_counters");
    JR_CUDA(cudaStreamSynchronize(st), "jr_set_counters");
    c->steps = in->steps_per_chain;
    return JR_OK;
}

jr_status jr_eval_states(const jr_scene* scene, const jr_params* params, const float* x_dev, uint64_t n, float* F_dev,
                         float* p_dev, float* u_dev, float* k_dev, int32_t* hit_ids_dev, void* stream) {
    if (!scene || !params || (n > 0 && !x_dev)) return fail(JR_ERR_INVALID_ARG, "jr_eval_states: null argument");
    if (params->max_depth > JR_MAX_DEPTH) return fail(JR_ERR_INVALID_ARG, "jr_eval_states: max_depth > 15");
    if (!(params->c_tilde > 0.f)) return fail(JR_ERR_INVALID_ARG, "jr_eval_states: c_tilde must be > 0");
    JR_CUDA(launch_eval_states(scene->view, params->max_depth, params->c_tilde, x_dev, n, F_dev, p_dev, u_dev, k_dev,
                               hit_ids_dev, (cudaStream_t)stream),
            "jr_eval_states");
    return JR_OK;
}

jr_status jr_eval_grad(const jr_scene* scene, const jr_params* params, const float* x_dev, uint64_t n, float* F_dev,
                       float* dF_dev, void* stream) {
    if (!scene || !params || (n > 0 && !x_dev)) return fail(JR_ERR_INVALID_ARG, "jr_eval_grad: null argument");
    if (params->max_depth > JR_MAX_DEPTH) return fail(JR_ERR_INVALID_ARG, "jr_eval_grad: max_depth > 15");
    JR_CUDA(launch_eval_grad(scene->view, params->max_depth, x_dev, n, F_dev, dF_dev, (cudaStream_t)stream),
            "jr_eval_grad");
    return JR_OK;
}

jr_status jr_render_pt(const jr_scene* scene, const jr_params* params, uint64_t sample_begin, uint64_t n_samples,
                       double* accum_dev, void* stream) {
    if (!scene || !params || !accum_dev) return fail(JR_ERR_INVALID_ARG, "jr_render_pt: null argument");
    if (params->width == 0 || params->height == 0 || params->max_depth > JR_MAX_DEPTH)
        return fail(JR_ERR_INVALID_ARG, "jr_render_pt: bad image size or depth");
    JR_CUDA(launch_render_pt(scene->view, params->width, params->height, params->max_depth, params->seed, sample_begin,
                             n_samples, accum_dev, (cudaStream_t)stream),
            "jr_render_pt");
    return JR_OK;
}

jr_status jr_fp32_peak(double* tflops_out, double* ms_out, void* stream) {
    if (!tflops_out) return fail(JR_ERR_INVALID_ARG, "jr_fp32_peak: null output");
    JR_CUDA(measure_fma_peak(tflops_out, ms_out, (cudaStream_t)stream), "jr_fp32_peak");
    return JR_OK;
}

jr_status jr_philox(uint64_t seed, uint32_t tag, uint32_t block, uint64_t chain_begin, uint64_t step, uint64_t n,
                    uint32_t* out_dev, void* stream) {
    if (n > 0 && !out_dev) return fail(JR_ERR_INVALID_ARG, "jr_philox: null output");
    JR_CUDA(launch_philox(seed, tag, block, chain_begin, step, n, out_dev, (cudaStream_t)stream), "jr_philox");
    return JR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many chain sets (scenes of uneven size, images, depths) advanced by
// one persistent launch, optionally replayed from a captured CUDA graph.
struct jr_batch {
    std::vector<jr_chains*> sets;
    std::vector<uint64_t> dev_steps;  // the step index each set has on the device side
    std::vector<uint64_t> dev_flow_gen;  // the flow generation of each set's device descriptor
    BatchEntry* entries = nullptr;
    uint64_t* px_off = nullptr;
    unsigned int* cursor = nullptr;
    BatchItem* items = nullptr;
    size_t items_cap = 0;
    uint32_t n_items = 0;
    uint32_t max_dim = 0;
    uint64_t total_px = 0, total_chains = 0;
    int block = 128;  // chains per megakernel work item; 0: the batched wavefront
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t graph_steps = 0;
    int graph_block = -1;
    // the batched wavefront, set up on first use: the merged scene, roots,
    // chain prefix sums, step-launch work items, the path launches' cursor
    Bvh4Node* m_nodes = nullptr;
    TriRecord* m_tris = nullptr;
    Material* m_mats = nullptr;
    int* roots = nullptr;
    uint64_t* chain_off = nullptr;
    BatchItem* wf_items = nullptr;
    unsigned int* fetch = nullptr;
    BatchWave bw{};
    bool wf_ready = false;
    ~jr_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(entries);
        cudaFree(px_off);
        cudaFree(cursor);
        cudaFree(items);
        cudaFree(m_nodes);
        cudaFree(m_tris);
        cudaFree(m_mats);
        cudaFree(roots);
        cudaFree(chain_off);
        cudaFree(wf_items);
        cudaFree(fetch);
    }
};

namespace {

// Work items: blocks of `block` chains, most expensive first (a chain step
// costs about (depth + 1) ray casts of log(triangles) traversal depth).
jr_status build_items(jr_batch* b, int block, cudaStream_t st) {
    struct Cand {
        double cost;
        BatchItem it;
    };
    std::vector<Cand> v;
    for (uint32_t k = 0; k < b->sets.size(); ++k) {
        const jr_chains* c = b->sets[k];
        const double per_chain = (c->view.depth + 1.0) * std::log2(c->scene->info.n_tris + 2.0);
        for (uint64_t beg = 0; beg < c->view.n; beg += (uint64_t)block) {
            const uint64_t end = std::min<uint64_t>(beg + block, c->view.n);
            v.push_back({per_chain * (double)(end - beg), BatchItem{k, (uint32_t)beg, (uint32_t)end}});
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const Cand& a, const Cand& c) { return a.cost > c.cost; });
    std::vector<BatchItem> h(v.size());
    for (size_t q = 0; q < v.size(); ++q) h[q] = v[q].it;
    if (h.size() > b->items_cap) {
        cudaFree(b->items);
        b->items = nullptr;
        b->items_cap = 0;
        JR_CUDA(dev_alloc(&b->items, h.size()), "jr_batch (work items)");
        b->items_cap = h.size();
    }
    JR_CUDA(cudaMemcpyAsync(b->items, h.data(), sizeof(BatchItem) * h.size(), cudaMemcpyHostToDevice, st),
            "jr_batch (work items)");
    JR_CUDA(cudaStreamSynchronize(st), "jr_batch (work items)");
    b->n_items = (uint32_t)h.size();
    b->block = block;
    return JR_OK;
}

bool batch_has_flow(const jr_batch* b) {
    for (const jr_chains* c : b->sets)
        if (c->view.flow.D != 0) return true;
    return false;
}

// The host views of the sets with a flow attached (their flow launches).
std::vector<ChainView> flow_views(const jr_batch* b) {
    std::vector<ChainView> v;
    for (const jr_chains* c : b->sets)
        if (c->view.flow.D != 0) v.push_back(c->view);
    return v;
}

// Bring the device-side step index of every set up to date with its host
// counter (a set may have been advanced on its own since the last batch), and
// a set's device descriptor with its flow when jr_chains_set_flow changed it
// (a captured graph holds the old flow's launches, so it is dropped).
jr_status sync_steps(jr_batch* b, cudaStream_t st) {
    for (size_t k = 0; k < b->sets.size(); ++k) {
        const jr_chains* c = b->sets[k];
        if (c->flow_gen != b->dev_flow_gen[k]) {
            BatchEntry h{};
            h.s = c->scene_view();
            h.c = c->view;
            h.step = c->steps;
            JR_CUDA(cudaMemcpyAsync(b->entries + k, &h, sizeof(h), cudaMemcpyHostToDevice, st), "jr_batch (flow)");
            JR_CUDA(cudaStreamSynchronize(st), "jr_batch (flow)");
            b->dev_flow_gen[k] = c->flow_gen;
            b->dev_steps[k] = c->steps;
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            b->exec = nullptr;
            b->graph = nullptr;
        }
        const uint64_t s = b->sets[k]->steps;
        if (s != b->dev_steps[k]) {
            unsigned long long v = s;
            JR_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(b->entries + k) + offsetof(BatchEntry, step), &v,
                                    sizeof(v), cudaMemcpyHostToDevice, st),
                    "jr_batch (step index)");
            JR_CUDA(cudaStreamSynchronize(st), "jr_batch (step index)");
            b->dev_steps[k] = s;
        }
    }
    return JR_OK;
}

void after_launch(jr_batch* b, uint32_t n_steps) {
    for (size_t k = 0; k < b->sets.size(); ++k) {
        b->sets[k]->steps += n_steps;
        b->dev_steps[k] += n_steps;
    }
}

// Set up the batched wavefront once: every set's wavefront buffers (and the
// device descriptors that point at them), the merged scene (each distinct
// scene copied once and rebased), the sets' roots in it, the chain prefix
// sums and the step launches' work items.
jr_status prepare_wave(jr_batch* b, cudaStream_t st) {
    if (b->wf_ready) return JR_OK;
    const uint32_t S = (uint32_t)b->sets.size();
    if (S > kBatchMaxSets)
        return fail(JR_ERR_INVALID_ARG, "jr_batch: the batched wavefront takes at most " +
                                            std::to_string(kBatchMaxSets) + " sets");
    for (jr_chains* c : b->sets) {
        jr_status a = ensure_wavefront(c, st);
        if (a != JR_OK) return a;
    }
    std::vector<BatchEntry> h(S);
    std::vector<const jr_scene*> uniq;
    std::vector<uint64_t> noff, toff, moff;  // per distinct scene
    uint64_t nn = 0, nt = 0, nm = 0;
    std::vector<int> root(S);
    std::vector<uint64_t> coff(S + 1, 0);
    std::vector<BatchItem> items;
    for (uint32_t k = 0; k < S; ++k) {
        const jr_chains* c = b->sets[k];
        h[k].s = c->scene_view();
        h[k].c = c->view;
        h[k].step = b->dev_steps[k];
        size_t u = 0;
        while (u < uniq.size() && uniq[u] != c->scene) ++u;
        if (u == uniq.size()) {
            uniq.push_back(c->scene);
            noff.push_back(nn);
            toff.push_back(nt);
            moff.push_back(nm);
            nn += (uint64_t)c->scene->view.n_nodes;
            nt += c->scene->info.n_tris;
            nm += c->scene->info.n_materials;
        }
        root[k] = rebase_ref(c->scene->view.root, (int)noff[u], (int)toff[u]);
        coff[k + 1] = coff[k] + c->view.n;
        for (uint64_t beg = 0; beg < c->view.n; beg += 128)
            items.push_back(BatchItem{k, (uint32_t)beg, (uint32_t)std::min<uint64_t>(beg + 128, c->view.n)});
    }
    if (nt >= (1ull << 28) || nn >= (1ull << 31) || coff[S] >= (1ull << 31))
        return fail(JR_ERR_INVALID_ARG, "jr_batch: the merged scene or the chain count is too large for the "
                                        "batched wavefront (2^28 triangles, 2^31 nodes or chains)");
    const char* who = "jr_batch (batched wavefront set-up)";
    // a set-up that failed part way may have left buffers: free them first
    cudaFree(b->m_nodes);
    cudaFree(b->m_tris);
    cudaFree(b->m_mats);
    cudaFree(b->roots);
    cudaFree(b->chain_off);
    cudaFree(b->wf_items);
    cudaFree(b->fetch);
    b->m_nodes = nullptr;
    b->m_tris = nullptr;
    b->m_mats = nullptr;
    b->roots = nullptr;
    b->chain_off = nullptr;
    b->wf_items = nullptr;
    b->fetch = nullptr;
    JR_CUDA(dev_alloc(&b->m_nodes, std::max<uint64_t>(nn, 1)), who);
    JR_CUDA(dev_alloc(&b->m_tris, std::max<uint64_t>(nt, 1)), who);
    JR_CUDA(dev_alloc(&b->m_mats, std::max<uint64_t>(nm, 1)), who);
    JR_CUDA(dev_alloc(&b->roots, S), who);
    JR_CUDA(dev_alloc(&b->chain_off, S + 1), who);
    JR_CUDA(dev_alloc(&b->wf_items, std::max<size_t>(items.size(), 1)), who);
    JR_CUDA(dev_alloc(&b->fetch, 1), who);
    for (size_t u = 0; u < uniq.size(); ++u) {
        const jr_scene* sc = uniq[u];
        const uint32_t n_nodes = (uint32_t)sc->view.n_nodes, n_tris = sc->info.n_tris,
                       n_mats = sc->info.n_materials;
        if (n_nodes)
            JR_CUDA(cudaMemcpyAsync(b->m_nodes + noff[u], sc->nodes, sizeof(Bvh4Node) * n_nodes,
                                    cudaMemcpyDeviceToDevice, st),
                    who);
        if (n_tris)
            JR_CUDA(cudaMemcpyAsync(b->m_tris + toff[u], sc->tris, sizeof(TriRecord) * n_tris,
                                    cudaMemcpyDeviceToDevice, st),
                    who);
        if (n_mats)
            JR_CUDA(cudaMemcpyAsync(b->m_mats + moff[u], sc->mats, sizeof(Material) * n_mats,
                                    cudaMemcpyDeviceToDevice, st),
                    who);
        JR_CUDA(launch_rebase_scene(b->m_nodes + noff[u], n_nodes, b->m_tris + toff[u], n_tris, (int)noff[u],
                                    (int)toff[u], (int)moff[u], st),
                who);
    }
    JR_CUDA(cudaMemcpyAsync(b->entries, h.data(), sizeof(BatchEntry) * S, cudaMemcpyHostToDevice, st), who);
    JR_CUDA(cudaMemcpyAsync(b->roots, root.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st), who);
    JR_CUDA(cudaMemcpyAsync(b->chain_off, coff.data(), sizeof(uint64_t) * (S + 1), cudaMemcpyHostToDevice, st), who);
    if (!items.empty())
        JR_CUDA(cudaMemcpyAsync(b->wf_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                                st),
                who);
    JR_CUDA(cudaStreamSynchronize(st), who);
    BatchWave& bw = b->bw;
    bw.merged = SceneView{};
    bw.merged.nodes = b->m_nodes;
    bw.merged.tris = b->m_tris;
    bw.merged.mats = b->m_mats;
    bw.merged.root = kNoChild;
    bw.merged.n_nodes = (int)nn;
    bw.merged.n_tris = (uint32_t)nt;
    bw.merged.visit_budget = kNodeVisitBudget;
    bw.merged.stack_limit = kStackSize;
    bw.roots = b->roots;
    bw.chain_off = b->chain_off;
    bw.items = b->wf_items;
    bw.n_sets = S;
    bw.n_items = (uint32_t)items.size();
    bw.fetch = b->fetch;
    long long blocks = 0;
    JR_CUDA(batch_wavefront_grid(&blocks), who);
    b->wf_ready = true;
    return JR_OK;
}

// Enqueue one batch advance (no allocation, so it can be captured): the
// megakernel launch, or the batched wavefront's launches; then the fold,
// which also moves every set's device step index on by n_steps.
cudaError_t enqueue_batch(jr_batch* b, uint32_t n_steps, cudaStream_t st) {
    const uint32_t S = (uint32_t)b->sets.size();
    if (b->block == 0) {
        cudaError_t e = launch_batch_wavefront(b->bw, b->entries, n_steps, flow_views(b), st);
        if (e != cudaSuccess) return e;
        return launch_batch(b->entries, b->items, 0, b->px_off, S, b->total_px, b->cursor, b->max_dim, 128,
                            n_steps, st);
    }
    return launch_batch(b->entries, b->items, b->n_items, b->px_off, S, b->total_px, b->cursor, b->max_dim, b->block,
                        n_steps, st);
}

jr_status batch_launch(jr_batch* b, uint32_t n_steps, cudaStream_t st, const char* who) {
    if (b->block != 0 && batch_has_flow(b))
        return fail(JR_ERR_STATE, std::string(who) + ": a set has a flow attached; select JR_BATCH_WAVEFRONT");
    if (b->block == 0) {
        jr_status a = prepare_wave(b, st);
        if (a != JR_OK) return a;
    }
    JR_CUDA(enqueue_batch(b, n_steps, st), who);
    return JR_OK;
}

}  // namespace

extern "C" {

jr_status jr_batch_create(jr_chains* const* sets, uint32_t n_sets, void* stream, jr_batch** out) {
    if (!sets || !out || n_sets == 0) return fail(JR_ERR_INVALID_ARG, "jr_batch_create: null argument or no sets");
    cudaStream_t st = (cudaStream_t)stream;
    jr_batch* b = new (std::nothrow) jr_batch();
    if (!b) return fail(JR_ERR_OOM, "jr_batch_create: host allocation failed");
    std::vector<BatchEntry> h(n_sets);
    std::vector<uint64_t> off(n_sets + 1, 0);
    for (uint32_t k = 0; k < n_sets; ++k) {
        jr_chains* c = sets[k];
        if (!c) {
            delete b;
            return fail(JR_ERR_INVALID_ARG, "jr_batch_create: null chain set");
        }
        for (uint32_t q = 0; q < k; ++q)
            if (sets[q] == c) {
                delete b;
                return fail(JR_ERR_INVALID_ARG, "jr_batch_create: a chain set appears twice");
            }
        if (c->view.flags & JR_FLAG_MALA) {
            delete b;
            return fail(JR_ERR_STATE, "jr_batch_create: MALA chain sets advance on their own (megakernel)");
        }
        h[k].s = c->scene_view();
        h[k].c = c->view;
        h[k].step = c->steps;
        off[k + 1] = off[k] + (uint64_t)c->view.width * c->view.height;
        b->max_dim = std::max(b->max_dim, c->view.dim);
        b->total_chains += c->view.n;
        b->sets.push_back(c);
        b->dev_steps.push_back(c->steps);
        b->dev_flow_gen.push_back(c->flow_gen);
    }
    b->total_px = off[n_sets];
    cudaError_t e;
    if ((e = dev_alloc(&b->entries, n_sets)) != cudaSuccess || (e = dev_alloc(&b->px_off, n_sets + 1)) != cudaSuccess ||
        (e = dev_alloc(&b->cursor, 1)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->entries, h.data(), sizeof(BatchEntry) * n_sets, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(b->px_off, off.data(), sizeof(uint64_t) * (n_sets + 1), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(b->cursor, 0, sizeof(unsigned int), st)) != cudaSuccess) {
        delete b;
        return cuda_fail(e, "jr_batch_create");
    }
    jr_status r = build_items(b, 128, st);
    if (r == JR_OK && batch_has_flow(b)) b->block = 0;  // sets with a flow advance in the batched wavefront only
    if (r == JR_OK) r = batch_launch(b, 0, st, "jr_batch_create");  // set-up launch: no steps
    if (r != JR_OK) {
        delete b;
        return r;
    }
    *out = b;
    return JR_OK;
}

void jr_batch_destroy(jr_batch* batch) { delete batch; }

jr_status jr_batch_set_block(jr_batch* b, uint32_t block) {
    if (!b) return fail(JR_ERR_INVALID_ARG, "jr_batch_set_block: null batch");
    if (block == JR_BATCH_WAVEFRONT) {
        b->block = 0;
        return JR_OK;
    }
    if (block < 32 || block > 256 || block % 32 != 0)
        return fail(JR_ERR_INVALID_ARG,
                    "jr_batch_set_block: block must be a multiple of 32 in [32, 256], or JR_BATCH_WAVEFRONT");
    if (batch_has_flow(b))
        return fail(JR_ERR_STATE, "jr_batch_set_block: sets with a flow attached advance in the batched wavefront");
    return build_items(b, (int)block, nullptr);
}

jr_status jr_batch_advance(jr_batch* b, uint32_t n_steps, void* stream) {
    if (!b) return fail(JR_ERR_INVALID_ARG, "jr_batch_advance: null batch");
    if (n_steps == 0) return JR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    jr_status r = sync_steps(b, st);
    if (r == JR_OK) r = batch_launch(b, n_steps, st, "jr_batch_advance");
    if (r == JR_OK) after_launch(b, n_steps);
    return r;
}

jr_status jr_batch_advance_graph(jr_batch* b, uint32_t n_steps, void* stream) {
    if (!b) return fail(JR_ERR_INVALID_ARG, "jr_batch_advance_graph: null batch");
    if (n_steps == 0) return JR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    jr_status r = sync_steps(b, st);
    if (r == JR_OK && b->block != 0 && batch_has_flow(b))
        r = fail(JR_ERR_STATE, "jr_batch_advance_graph: a set has a flow attached; select JR_BATCH_WAVEFRONT");
    if (r == JR_OK && b->block == 0) r = prepare_wave(b, st);
    if (r != JR_OK) return r;
    if (!b->exec || b->graph_steps != n_steps || b->graph_block != b->block) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaStream_t cap = nullptr;
        JR_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "jr_batch_advance_graph");
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = enqueue_batch(b, n_steps, cap);
            e = cudaStreamEndCapture(cap, &b->graph);
            if (e == cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (b->graph) cudaGraphDestroy(b->graph);
            b->graph = nullptr;
            b->exec = nullptr;
            return cuda_fail(e, "jr_batch_advance_graph (capture)");
        }
        b->graph_steps = n_steps;
        b->graph_block = b->block;
    }
    JR_CUDA(cudaGraphLaunch(b->exec, st), "jr_batch_advance_graph");
    after_launch(b, n_steps);
    return JR_OK;
}

jr_status jr_batch_autotune(jr_batch* b, uint32_t probe_steps, void* stream, jr_tune_report* out) {
    if (!b || !out || probe_steps == 0) return fail(JR_ERR_INVALID_ARG, "jr_batch_autotune: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const bool flows = batch_has_flow(b);  // only the batched wavefront runs flows
    const uint32_t all[] = {32, 64, 128, 256, JR_BATCH_WAVEFRONT}, wave_only[] = {JR_BATCH_WAVEFRONT};
    const uint32_t* cands = flows ? wave_only : all;
    const uint32_t n_cands = flows ? 1 : b->sets.size() <= kBatchMaxSets ? 5 : 4;
    jr_tune_report rep{};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    JR_CUDA(cudaEventCreate(&e0), "jr_batch_autotune");
    JR_CUDA(cudaEventCreate(&e1), "jr_batch_autotune");
    double best = INFINITY;
    jr_status r = JR_OK;
    for (uint32_t q = 0; q < n_cands && r == JR_OK; ++q) {
        if (cands[q] == JR_BATCH_WAVEFRONT) {
            b->block = 0;
            r = prepare_wave(b, st);  // one-time set-up, outside the timed probe
        } else {
            r = build_items(b, (int)cands[q], st);
        }
        if (r == JR_OK) r = sync_steps(b, st);
        if (r != JR_OK) break;
        cudaError_t e;
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) {
            r = cuda_fail(e, "jr_batch_autotune");
            break;
        }
        r = batch_launch(b, probe_steps, st, "jr_batch_autotune");
        if (r != JR_OK) break;
        after_launch(b, probe_steps);
        float ms = 0.f;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            r = cuda_fail(e, "jr_batch_autotune");
            break;
        }
        const double ns = 1e6 * ms / ((double)b->total_chains * probe_steps);
        rep.block[rep.n] = cands[q];
        rep.ns_per_chain_step[rep.n] = ns;
        rep.n++;
        if (ns < best) {
            best = ns;
            rep.best_block = cands[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != JR_OK) return r;
    if (rep.best_block == JR_BATCH_WAVEFRONT) {
        b->block = 0;
    } else {
        r = build_items(b, (int)rep.best_block, st);
        if (r != JR_OK) return r;
    }
    *out = rep;
    return JR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The learned regeneration flow (jr_flow.cu): parameters, evaluation, and the
// attachment to a chain set.
struct jr_flow {
    uint32_t D = 0, A = 0, AK = 0;
    uint8_t* perm = nullptr;       // [kFL][D]
    float* master = nullptr;       // [kFL][S] FP32, the documented layout
    __nv_bfloat16* wb = nullptr;   // packed bf16 weights
    float* bias = nullptr;         // packed FP32 biases
    unsigned char* ws = nullptr;   // inference layout
    unsigned int* status = nullptr;  // JR_STATUS_* bits of the flow's own launches
    float* adam_m = nullptr;       // optimiser moments [kFL][S]
    float* adam_v = nullptr;
    float* grad = nullptr;         // [kFL][S] gradient accumulator
    uint64_t adam_t = 0;
    uint32_t extra_tx = 0;  // testing hook, see jr_debug_flow_wait
    FlowView view(float beta) const {
        FlowView f;
        f.extra_tx = extra_tx;
        f.D = D;
        f.A = A;
        f.AK = AK;
        f.perm = perm;
        f.wb = wb;
        f.bias = bias;
        f.ws = ws;
        f.beta = beta;
        return f;
    }
    ~jr_flow() {
        cudaFree(perm);
        cudaFree(master);
        cudaFree(wb);
        cudaFree(bias);
        cudaFree(ws);
        cudaFree(status);
        cudaFree(adam_m);
        cudaFree(adam_v);
        cudaFree(grad);
    }
};

extern "C" {

uint64_t jr_flow_param_count(uint32_t dim) {
    if (dim < 2 || dim > (uint32_t)kMaxDim || dim % 2) return 0;
    return (uint64_t)kFL * flow_layer_floats(dim);
}

namespace {
// Both packed copies of the master parameters: the training layout and the
// inference layout.
cudaError_t pack_all(jr_flow* f, cudaStream_t st) {
    cudaError_t e = launch_flow_pack(f->master, f->wb, f->bias, f->AK, st);
    return e != cudaSuccess ? e : launch_flow_pack_ws(f->master, f->ws, f->AK, st);
}
}  // namespace

jr_status jr_flow_create(uint32_t dim, const int32_t* perm, const float* params, void* stream, jr_flow** out) {
    if (!perm || !params || !out) return fail(JR_ERR_INVALID_ARG, "jr_flow_create: null argument");
    if (dim < 2 || dim > (uint32_t)kMaxDim || dim % 2)
        return fail(JR_ERR_INVALID_ARG, "jr_flow_create: dim must be even, 2..32");
    std::vector<uint8_t> pm((size_t)kFL * dim);
    for (int l = 0; l < kFL; ++l) {
        std::vector<int> seen(dim, 0);
        for (uint32_t d = 0; d < dim; ++d) {
            const int32_t v = perm[l * dim + d];
            if (v < 0 || (uint32_t)v >= dim || seen[v]++)
                return fail(JR_ERR_INVALID_ARG, "jr_flow_create: perm[l] must be a permutation of 0..dim-1");
            pm[l * dim + d] = (uint8_t)v;
        }
    }
    jr_flow* f = new (std::nothrow) jr_flow();
    if (!f) return fail(JR_ERR_OOM, "jr_flow_create: host allocation failed");
    f->D = dim;
    f->A = dim / 2;
    f->AK = f->A * kFK;
    const size_t S = flow_layer_floats(dim), P = (size_t)kFL * S;
    const size_t nwb = (size_t)kFL * (kFH * kFS1 + kFH * kFS2 + (size_t)f->AK * kFS2);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = dev_alloc(&f->perm, pm.size())) != cudaSuccess || (e = dev_alloc(&f->master, P)) != cudaSuccess ||
        (e = dev_alloc(&f->wb, nwb)) != cudaSuccess ||
        (e = dev_alloc(&f->bias, (size_t)kFL * (2 * kFH + f->AK))) != cudaSuccess ||
        (e = dev_alloc(&f->ws, (size_t)kFL * flow_ws_layer_bytes(f->AK))) != cudaSuccess ||
        (e = dev_alloc(&f->status, 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(f->status, 0, sizeof(unsigned int), st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(f->perm, pm.data(), pm.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(f->master, params, sizeof(float) * P, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = pack_all(f, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        delete f;
        return cuda_fail(e, "jr_flow_create");
    }
    *out = f;
    return JR_OK;
}

void jr_flow_destroy(jr_flow* flow) { delete flow; }

jr_status jr_flow_set_params(jr_flow* f, const float* params, void* stream) {
    if (!f || !params) return fail(JR_ERR_INVALID_ARG, "jr_flow_set_params: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    JR_CUDA(cudaMemcpyAsync(f->master, params, sizeof(float) * kFL * flow_layer_floats(f->D), cudaMemcpyHostToDevice,
                            st),
            "jr_flow_set_params");
    JR_CUDA(pack_all(f, st), "jr_flow_set_params");
    JR_CUDA(cudaStreamSynchronize(st), "jr_flow_set_params");
    return JR_OK;
}

jr_status jr_flow_get_status(jr_flow* f, uint32_t* status_out, void* stream) {
    if (!f || !status_out) return fail(JR_ERR_INVALID_ARG, "jr_flow_get_status: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int v = 0;
    JR_CUDA(cudaMemcpyAsync(&v, f->status, sizeof(v), cudaMemcpyDeviceToHost, st), "jr_flow_get_status");
    JR_CUDA(cudaStreamSynchronize(st), "jr_flow_get_status");
    *status_out = v;
    return JR_OK;
}

jr_status jr_debug_flow_wait(jr_flow* f, int enable) {
    if (!f) return fail(JR_ERR_INVALID_ARG, "jr_debug_flow_wait: null flow");
    f->extra_tx = enable ? 16u : 0u;
    return JR_OK;
}

jr_status jr_flow_get_params(jr_flow* f, float* params, void* stream) {
    if (!f || !params) return fail(JR_ERR_INVALID_ARG, "jr_flow_get_params: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    JR_CUDA(cudaMemcpyAsync(params, f->master, sizeof(float) * kFL * flow_layer_floats(f->D), cudaMemcpyDeviceToHost,
                            st),
            "jr_flow_get_params");
    JR_CUDA(cudaStreamSynchronize(st), "jr_flow_get_params");
    return JR_OK;
}

jr_status jr_flow_log_density(jr_flow* f, const float* x_dev, uint64_t n, float* lq_dev, void* stream) {
    if (!f || (n > 0 && (!x_dev || !lq_dev))) return fail(JR_ERR_INVALID_ARG, "jr_flow_log_density: null argument");
    if (n >= (1ull << 32)) return fail(JR_ERR_INVALID_ARG, "jr_flow_log_density: n must be below 2^32");
    JR_CUDA(launch_flow(f->view(0.f), false, const_cast<float*>(x_dev), nullptr, nullptr, n, nullptr, nullptr,
                        (uint32_t)n, nullptr, lq_dev, nullptr, f->status, (cudaStream_t)stream),
            "jr_flow_log_density");
    return JR_OK;
}

jr_status jr_flow_sample(jr_flow* f, float* xz_dev, uint64_t n, float* lq_dev, void* stream) {
    if (!f || (n > 0 && (!xz_dev || !lq_dev))) return fail(JR_ERR_INVALID_ARG, "jr_flow_sample: null argument");
    if (n >= (1ull << 32)) return fail(JR_ERR_INVALID_ARG, "jr_flow_sample: n must be below 2^32");
    JR_CUDA(launch_flow(f->view(0.f), true, xz_dev, nullptr, nullptr, n, nullptr, nullptr, (uint32_t)n, nullptr,
                        lq_dev, nullptr, f->status, (cudaStream_t)stream),
            "jr_flow_sample");
    return JR_OK;
}

jr_status jr_flow_copy_params(jr_flow* dst, const jr_flow* src, void* stream) {
    if (!dst || !src) return fail(JR_ERR_INVALID_ARG, "jr_flow_copy_params: null argument");
    if (dst->D != src->D) return fail(JR_ERR_INVALID_ARG, "jr_flow_copy_params: dimensions differ");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = (size_t)kFL * flow_layer_floats(src->D);
    JR_CUDA(cudaMemcpyAsync(dst->perm, src->perm, (size_t)kFL * src->D, cudaMemcpyDeviceToDevice, st),
            "jr_flow_copy_params");
    JR_CUDA(cudaMemcpyAsync(dst->master, src->master, sizeof(float) * P, cudaMemcpyDeviceToDevice, st),
            "jr_flow_copy_params");
    JR_CUDA(pack_all(dst, st), "jr_flow_copy_params");
    return JR_OK;
}

jr_status jr_chains_snapshot(jr_chains* c, float* x_dev, float* w_dev, void* stream) {
    if (!c || !x_dev || !w_dev) return fail(JR_ERR_INVALID_ARG, "jr_chains_snapshot: null argument");
    JR_CUDA(launch_snapshot(c->view, x_dev, w_dev, (cudaStream_t)stream), "jr_chains_snapshot");
    return JR_OK;
}

jr_status jr_chains_snapshot_append(jr_chains* c, float* x_ring, float* w_ring, uint64_t capacity,
                                    unsigned long long* total_dev, void* stream) {
    if (!c || !x_ring || !w_ring || !total_dev) return fail(JR_ERR_INVALID_ARG, "jr_chains_snapshot_append: null argument");
    if (capacity == 0) return fail(JR_ERR_INVALID_ARG, "jr_chains_snapshot_append: capacity must be > 0");
    JR_CUDA(launch_snapshot_append(c->view, x_ring, w_ring, capacity, total_dev, (cudaStream_t)stream),
            "jr_chains_snapshot_append");
    return JR_OK;
}

jr_status jr_flow_gradient(jr_flow* f, const float* x_dev, const float* w_dev, uint64_t n, uint64_t off,
                           uint32_t batch, float* grad_host, float* loss_host, void* stream) {
    if (!f || !x_dev || !w_dev || !grad_host) return fail(JR_ERR_INVALID_ARG, "jr_flow_gradient: null argument");
    if (batch == 0 || off + batch > n) return fail(JR_ERR_INVALID_ARG, "jr_flow_gradient: rows out of range");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = (size_t)kFL * flow_layer_floats(f->D);
    float* buf = nullptr;  // gradient, then the weight sum and the loss
    JR_CUDA(dev_alloc(&buf, P + 2), "jr_flow_gradient");
    cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(float) * (P + 2), st);
    if (e == cudaSuccess) e = launch_flow_train_step(f->view(0.f), x_dev, w_dev, n, off, batch, buf, buf + P, buf + P + 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad_host, buf, sizeof(float) * P, cudaMemcpyDeviceToHost, st);
    float tail[2] = {0.f, 0.f};
    if (e == cudaSuccess) e = cudaMemcpyAsync(tail, buf + P, sizeof(tail), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "jr_flow_gradient");
    if (loss_host) *loss_host = tail[1];
    return JR_OK;
}

jr_status jr_flow_train(jr_flow* f, const float* x_dev, const float* w_dev, uint64_t n, uint32_t iters,
                        uint32_t batch, float lr, uint64_t seed, float* loss_host, void* stream) {
    return jr_flow_train_rows(f, x_dev, w_dev, n, n, iters, batch, lr, seed, loss_host, stream);
}

jr_status jr_flow_train_rows(jr_flow* f, const float* x_dev, const float* w_dev, uint64_t n, uint64_t n_rows,
                             uint32_t iters, uint32_t batch, float lr, uint64_t seed, float* loss_host,
                             void* stream) {
    if (!f || !x_dev || !w_dev) return fail(JR_ERR_INVALID_ARG, "jr_flow_train: null argument");
    if (n_rows > n) return fail(JR_ERR_INVALID_ARG, "jr_flow_train: n_rows exceeds the row stride");
    if (batch == 0 || batch % 64 != 0 || batch > n_rows)
        return fail(JR_ERR_INVALID_ARG, "jr_flow_train: batch must be a positive multiple of 64, at most n_rows");
    if (!(lr > 0.f)) return fail(JR_ERR_INVALID_ARG, "jr_flow_train: lr must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = (size_t)kFL * flow_layer_floats(f->D);
    if (!f->grad) {
        cudaError_t e;
        if ((e = dev_alloc(&f->grad, P)) != cudaSuccess || (e = dev_alloc(&f->adam_m, P)) != cudaSuccess ||
            (e = dev_alloc(&f->adam_v, P)) != cudaSuccess ||
            (e = cudaMemsetAsync(f->adam_m, 0, sizeof(float) * P, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(f->adam_v, 0, sizeof(float) * P, st)) != cudaSuccess) {
            cudaFree(f->grad);
            cudaFree(f->adam_m);
            cudaFree(f->adam_v);
            f->grad = f->adam_m = f->adam_v = nullptr;
            return cuda_fail(e, "jr_flow_train (optimiser state)");
        }
    }
    float* scal = nullptr;  // [iters][2]: minibatch weight sum, loss
    JR_CUDA(dev_alloc(&scal, 2 * (size_t)std::max<uint32_t>(iters, 1)), "jr_flow_train");
    cudaError_t e = cudaMemsetAsync(scal, 0, sizeof(float) * 2 * std::max<uint32_t>(iters, 1), st);
    uint64_t rng = seed * 0x9E3779B97F4A7C15ull + 0xD1B54A32D192ED03ull;
    for (uint32_t it = 0; it < iters && e == cudaSuccess; ++it) {
        rng ^= rng >> 30;  // splitmix64 (Steele, Lea, Flood 2014): the minibatch window
        rng *= 0xBF58476D1CE4E5B9ull;
        rng ^= rng >> 27;
        rng *= 0x94D049BB133111EBull;
        rng ^= rng >> 31;
        const uint64_t off = rng % (n_rows - batch + 1);
        if ((e = cudaMemsetAsync(f->grad, 0, sizeof(float) * P, st)) != cudaSuccess) break;
        if ((e = launch_flow_train_step(f->view(0.f), x_dev, w_dev, n, off, batch, f->grad, scal + 2 * it,
                                        scal + 2 * it + 1, st)) != cudaSuccess)
            break;
        if ((e = launch_adam(f->master, f->grad, f->adam_m, f->adam_v, P, lr, ++f->adam_t, st)) != cudaSuccess) break;
        if ((e = launch_flow_pack(f->master, f->wb, f->bias, f->AK, st)) != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = launch_flow_pack_ws(f->master, f->ws, f->AK, st);
    std::vector<float> h(2 * (size_t)std::max<uint32_t>(iters, 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), scal, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(scal);
    if (e != cudaSuccess) return cuda_fail(e, "jr_flow_train");
    if (loss_host)
        for (uint32_t it = 0; it < iters; ++it) loss_host[it] = h[2 * it + 1];
    return JR_OK;
}

}  // extern "C"

namespace {

// Drain: advance only the chains that are inside a tour until every tour has
// ended (a kill ends the tour and the chain); the steps are regular steps of
// Alg. 2 for those chains.  Returns the chains still in a tour after
// max_steps (0 when every tour completed).
jr_status drain_impl(jr_chains* c, uint32_t max_steps, uint64_t* remaining, cudaStream_t st, const char* who) {
    jr_status a = ensure_wavefront(c, st);
    if (a != JR_OK) return a;
    JR_CUDA(cudaMemsetAsync(c->view.wf.done, 0, c->view.n, st), who);
    unsigned int active = (unsigned int)std::min<uint64_t>(c->view.n, 0xffffffffu);
    uint32_t k = 0;
    // Steps are enqueued in groups that grow while tours stay open, so the
    // host waits rarely.  A step after the last tour has ended is a no-op; the
    // drain mark (1 + the last step after which a tour was open) gives the
    // steps the drain really took, as if the host had checked after every step.
    JR_CUDA(cudaMemsetAsync(c->view.counters + 3, 0, sizeof(unsigned long long), st), who);
    const uint64_t s0 = c->steps;
    uint32_t group = 1;
    while (active > 0 && k < max_steps) {
        const uint32_t g = std::min(group, max_steps - k);
        // one launch sequence per group: a single closing finish launch, not one per step
        JR_CUDA(launch_wavefront(c->scene_view(), c->view, s0 + k, g, st, kModeDrain), who);
        k += g;
        JR_CUDA(cudaMemcpyAsync(&active, c->view.wf.qcount + kQActive, sizeof(active), cudaMemcpyDeviceToHost, st),
                who);
        JR_CUDA(cudaStreamSynchronize(st), who);
        group = std::min<uint32_t>(2 * group, 16);
    }
    if (k > 0) {
        unsigned long long mark = 0;
        JR_CUDA(cudaMemcpyAsync(&mark, c->view.counters + 3, sizeof(mark), cudaMemcpyDeviceToHost, st), who);
        JR_CUDA(cudaStreamSynchronize(st), who);
        c->steps = active > 0 ? s0 + k : std::max<uint64_t>(mark, s0) + 1;
    }
    JR_CUDA(launch_fold(c->view, st), who);
    if (remaining) *remaining = active;
    return JR_OK;
}

// Restart: every chain starts a new tour from the current mu.
jr_status restart_impl(jr_chains* c, cudaStream_t st, const char* who) {
    jr_status a = ensure_wavefront(c, st);
    if (a != JR_OK) return a;
    c->epochs += 1;
    JR_CUDA(launch_wavefront(c->scene_view(), c->view, c->epochs, 1, st, kModeRestart), who);
    return JR_OK;
}

}  // namespace

extern "C" {

jr_status jr_complete_tours(jr_chains* c, uint32_t max_steps, uint64_t* remaining, void* stream) {
    if (!c) return fail(JR_ERR_INVALID_ARG, "jr_complete_tours: null chains");
    if (c->view.flags & JR_FLAG_MH) return fail(JR_ERR_STATE, "jr_complete_tours: an MH chain set has no tours");
    if (c->view.flags & JR_FLAG_MALA)
        return fail(JR_ERR_STATE, "jr_complete_tours: the drain runs in the wavefront, which has no MALA moves");
    cudaStream_t st = (cudaStream_t)stream;
    jr_status r = drain_impl(c, max_steps, remaining, st, "jr_complete_tours");
    if (r == JR_OK) r = restart_impl(c, st, "jr_complete_tours");
    return r;
}

jr_status jr_chains_set_flow(jr_chains* c, const jr_flow* f, float beta, uint32_t max_drain_steps,
                             uint64_t* remaining, void* stream) {
    if (!c) return fail(JR_ERR_INVALID_ARG, "jr_chains_set_flow: null chains");
    if (c->view.flags & (JR_FLAG_MH | JR_FLAG_MALA))
        return fail(JR_ERR_STATE, "jr_chains_set_flow: MH and MALA chains regenerate from the uniform mu only");
    // A flow of lower dimension models the leading coordinates only (the rest
    // stay uniform); it must cover the path's start record, coordinates 0..3.
    if (f && !(f->D == c->view.dim || (f->D >= 4 && f->D < c->view.dim)))
        return fail(JR_ERR_INVALID_ARG, "jr_chains_set_flow: the flow's dimension must equal the chains' or lie in 4 .. D - 1");
    if (f && !(beta >= 0.f && beta < 1.f))
        return fail(JR_ERR_INVALID_ARG, "jr_chains_set_flow: beta must be in [0, 1)");
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t rem = 0;
    jr_status r = drain_impl(c, max_drain_steps, &rem, st, "jr_chains_set_flow");  // finish the tours of the old mu
    if (r != JR_OK) return r;
    if (remaining) *remaining = rem;
    c->view.flow = f ? f->view(beta) : FlowView{};
    c->flow_gen += 1;
    return restart_impl(c, st, "jr_chains_set_flow");
}

}  // extern "C"
