#!/usr/bin/env python3
"""Throughput of Jump Restore chains on one GB300 (and N under torchrun).

One bench step = one jr_advance of every chain by `--chain-steps` iterations of
Alg. 2 (local MH move or regeneration, path construction + BVH traversal,
killing rate, splat) on the 512x512, depth-8 Cornell-box-with-two-20k-triangle
spheres workload with 2^20 chains -- i.e. 2^20 x 256 chain steps per bench step.

Prints ONE JSON line (rank 0).  `value` = chain steps/s over all ranks, device
timed with CUDA events on the launching stream; the L2 is flushed (a 512 MB
write) between timed launches.  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Restore chain steps/s on 1 GB300; time to relMSE 1e-2, learned vs plain regen"
UNIT = "chain steps/s"
# FP32 operations issued per unit of traversal work (counted from the kernel
# source: a visit of a 4-wide node = 4 slab tests of 6 FMA (2 FLOP each) on
# the octant's near and far planes + 4 min/max + 1 scaled compare (2), then 5
# compares of the sorting network;
# a triangle test = Moller-Trumbore: 2 cross, 4 dot, 1 reciprocal, 3 scaled
# products, 3 subtractions, 5 compares).
FLOP_PER_NODE = 77
FLOP_PER_TRI = 45
FP32_LANES = 128   # FP32 lanes per SM on sm_103a (the nominal-peak cross-check only)
# DRAM traffic of one wf_path_kernel launch (dram__bytes_read.sum +
# dram__bytes_write.sum), the mean over 8 launches of an ncu capture of the
# 2^18-chain case, scaled by 4 to the 2^20-chain workload (the paths of a
# launch grow with the chains).  It stands only while the kernel sources still
# hash to the values it was taken on (27.085 MB read + 0.218 MB written).
PATH_TRAFFIC = {"bytes_per_launch": 4 * (25.717e6 + 0.195e6),
                "sources": {"jr_wavefront.cu": "abfea2ffc0480f4e", "jr_device.cuh": "fe26fff844d2d218"},
                "summary": "profiles/path_kernel_cornell_spheres_512x512.md"}


def path_traffic(workload_name, chains):
    """Per-launch DRAM bytes of the path kernel, or None when the sources
    changed since the capture or the workload is not the one it scales to."""
    import hashlib
    if workload_name != "cornell_spheres" or chains != 1 << 20 or PATH_TRAFFIC["bytes_per_launch"] is None:
        return None
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2409_07148_gb300", "csrc")
    for f, h in PATH_TRAFFIC["sources"].items():
        with open(os.path.join(src, f), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != h:
                return None
    return PATH_TRAFFIC["bytes_per_launch"]


def workload(name):
    from paper_2409_07148_gb300 import scenes
    if name == "cornell_spheres":
        sc = scenes.cornell_spheres()
        return sc, dict(chains=1 << 20, chain_steps=256)
    if name == "cornell":
        sc = scenes.cornell()
        return sc, dict(chains=256, chain_steps=10_000)
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_rate(sc, wl, budget_s=12.0, seed=0, n_threads=0, max_chains=1 << 12):
    """The FP64 oracle as it stands (its own BVH; all host cores, or n_threads)
    on a bounded sample: a prefix of the chains, a few chain steps each."""
    from oracle import oracle as O
    osc = O.Scene(sc, bvh=sc.n_tris > 64)
    cores = n_threads or O.threads_default()
    n_chains = min(wl["chains"], max_chains)
    steps = 2
    ch = O.Chains(osc, sc.D, sc.width, sc.height, seed=seed, n_chains=n_chains)
    t0 = time.perf_counter()
    ch.advance(steps, n_threads=n_threads)
    dt = time.perf_counter() - t0
    # grow the sample to about budget_s of CPU work (bounded)
    total_steps, total_t = n_chains * steps, dt
    grow = max(1, min(64, int(budget_s / max(dt, 1e-3))))
    if grow > 1 and dt < budget_s:
        k = min(grow * steps, 256)
        t0 = time.perf_counter()
        ch.advance(k, n_threads=n_threads)
        total_t += time.perf_counter() - t0
        total_steps += n_chains * k
    return total_steps / total_t, cores, f"{n_chains} chains x {total_steps // n_chains} chain steps of the same workload"


def cpu_oracle_config1():
    """The oracle on the whole 64x64 Cornell workload (24 triangles, depth 3,
    256 chains x 10^4 steps, seed 0), all host cores: chain steps/s."""
    from oracle import oracle as O
    from paper_2409_07148_gb300 import scenes
    sc = scenes.cornell()
    ch = O.Chains(O.Scene(sc), sc.D, sc.width, sc.height, seed=0, n_chains=256)
    t0 = time.perf_counter()
    ch.advance(10_000)
    dt = time.perf_counter() - t0
    return 256 * 10_000 / dt, O.threads_default(), dt


def gpu_config1(stream):
    """The same whole 64x64 Cornell workload on this GPU (auto execution: one
    chain per warp for this 24-triangle scene), after a warm-up set, timed with
    CUDA events on its stream: chain steps/s and seconds."""
    import torch
    from paper_2409_07148_gb300 import jr, scenes
    sc = scenes.cornell()
    g = jr.Scene(sc, stream=stream)
    warm = jr.Chains(g, sc.width, sc.height, sc.depth, 256, seed=1, stream=stream)
    warm.advance(1000, stream=stream)
    ch = jr.Chains(g, sc.width, sc.height, sc.depth, 256, seed=0, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    ch.advance(10_000, stream=stream)
    e1.record(stream)
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    return 256 * 10_000 / dt, dt


def run_batched(args):
    """The 64-scene batch: one persistent launch per advance, replayed from a
    CUDA graph, work-item size picked by the library's autotuner (outside the
    timed region; its probe steps are real steps)."""
    import torch
    from paper_2409_07148_gb300 import jr, scenes
    ws, rank, _ = dist_env()
    K = args.chain_steps or 16
    stream = torch.cuda.Stream()
    scs = scenes.batched_workload(seed=rank)
    with torch.cuda.stream(stream):
        sets, handles = [], []
        for sc in scs:
            g = jr.Scene(sc, stream=stream)
            c = jr.Chains(g, sc.width, sc.height, sc.depth, sc.width * sc.height, seed=0, stream=stream)
            handles.append(g)
            sets.append(c)
        b = jr.Batch(sets, stream=stream)
        tune = b.autotune(2, stream=stream)
        b.advance_graph(K, stream=stream)  # capture
        for _ in range(args.warmup):
            b.advance_graph(K, stream=stream)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        stream.synchronize()
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        times = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.advance_graph(K, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        clocks = sampler.stop()
        chains = sum(c.n for c in sets)
        ok = all(c.stats(stream=stream)["status_word"] == 0 for c in sets)
    wave = tune["best_block"] == 0
    # per advance: the batched wavefront's step and path launches per chain
    # step, its closing step launch and the fold; else one persistent launch
    # and the fold
    launches = 2 * K + 2 if wave else 2
    if rank != 0:
        return
    total = sum(times)
    line = {"metric": METRIC, "value": chains * K * args.steps / total, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched64", "scenes": len(scs), "n_tris_total": sum(s.n_tris for s in scs),
                       "pixels_total": sum(s.width * s.height for s in scs), "chains": chains,
                       "chain_steps_per_step": K, "depths": sorted({s.depth for s in scs}),
                       "launch": ("batched wavefront: a step and a path launch per chain step, a closing step "
                                  "launch and the fold per advance, replayed from a CUDA graph") if wave else
                                 "one persistent launch + one fold per advance, replayed from a CUDA graph",
                       "autotune": tune, "l2": "flushed by a 512 MB write between timed launches",
                       "status_ok": ok},
            "clocks": clocks, "gpu_launches": launches * args.steps}
    print(json.dumps(line), flush=True)


def relmse(img, ref, eps=1e-2):
    """mean over pixels and channels of (I - R)^2 / (R^2 + eps)."""
    return float(((img - ref) ** 2 / (ref ** 2 + eps)).mean())


def run_caustic(args):
    print(json.dumps(time_to_target(args)), flush=True)


def time_to_target(args):
    """Time to relMSE 1e-2, learned vs plain regeneration, on the slit-caustic
    scene (1024^2, depth 10, 2^20 chains) or, with --workload terrain, on the
    fBm terrain lit by 256 small emitters (2048^2, depth 12, 2^22 chains).  Reference: plain path tracing on the GPU (its own noise is
    estimated from two independent halves and reported).  Each arm runs epochs
    of `epoch` chain steps; after every epoch the open tours are completed (so
    the checkpoint image is the completed-tour estimator) and the relMSE is
    taken off the clock.  The learned arm trains the flow on a snapshot of the
    chain states (weights p / (p + c~ u)) between epochs and regenerates from
    mu = beta mu_flow + (1 - beta) uniform in the next epoch."""
    if args.ref_samples is None:
        args.ref_samples = {"terrain": 1 << 37, "spheres_t2t": 1 << 35}.get(args.workload, 1 << 36)
    import torch
    from paper_2409_07148_gb300 import jr, scenes
    from paper_2409_07148_gb300.flowinit import init_flow_params
    if args.workload == "terrain":
        side = args.side or 2048
        sc = scenes.terrain(width=side, height=side, depth=12)
        C = args.chains or (1 << 22)
    elif args.workload == "spheres_t2t":
        side = args.side or 512
        sc = scenes.cornell_spheres(width=side, height=side, depth=8)
        C = args.chains or (1 << 20)
    else:
        side = args.side or 1024
        sc = scenes.caustic_slit(width=side, height=side, depth=10)
        C = args.chains or (1 << 20)
    wname = f"{sc.name}_{side}x{side}_depth{sc.depth}"
    stream = torch.cuda.Stream()
    target, tmax, epoch = 1e-2, args.time_limit, args.epoch
    with torch.cuda.stream(stream):
        g = jr.Scene(sc, stream=stream)
        # reference: two independent halves of plain path tracing (optionally
        # kept in a file, keyed by the scene size and the sample count)
        cache = args.ref_file and f"{args.ref_file}.{sc.name}.{side}.{args.ref_samples}.npz"
        t0 = time.perf_counter()
        if cache and os.path.exists(cache):
            z = np.load(cache)
            halves = [torch.from_numpy(z["h0"]).cuda(), torch.from_numpy(z["h1"]).cuda()]
        else:
            halves = []
            chunk = 1 << 28
            n_half = args.ref_samples // 2
            for h in range(2):
                acc = torch.zeros((side, side, 4), dtype=torch.float64, device="cuda")
                for s0 in range(0, n_half, chunk):
                    jr.render_pt(g, side, side, sc.depth, min(chunk, n_half - s0), seed=1000 + h, sample_begin=s0,
                                 accum=acc, stream=stream)
                halves.append(acc[..., :3] / n_half)
            stream.synchronize()
            if cache:
                np.savez(cache, h0=halves[0].cpu().numpy(), h1=halves[1].cpu().numpy())
        t_ref = time.perf_counter() - t0
        ref = 0.5 * (halves[0] + halves[1])
        ref_noise = relmse(halves[0], halves[1]) / 4.0   # relMSE of the mean of two halves vs truth, roughly

        def run_mala(mh):
            """MALA Restore (mh=False) or the MALA baseline (mh=True, large steps
            l = --mh-large-step, burn-in --mh-burn-in), sigma = --mala-sigma,
            --mala-chains chains, in the MALA megakernel.  It has no drain, so a
            MALA Restore checkpoint resolves with the chains' open tours."""
            Cm = args.mala_chains or C
            flags = jr.JR_FLAG_MALA | (jr.JR_FLAG_MH if mh else 0)
            ch = jr.Chains(g, side, side, sc.depth, Cm, seed=8, sigma=args.mala_sigma, flags=flags,
                           large_step=args.mh_large_step, burn_in=args.mh_burn_in if mh else 0, stream=stream)
            sampler = ClockSampler(torch.cuda.current_device())
            sampler.start()
            clock, curve, e, done = 0.0, [], 0, 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while mh and done < args.mh_burn_in:
                k = min(args.epoch_max, args.mh_burn_in - done)
                ch.advance(k, stream=stream)
                done += k
            torch.cuda.synchronize()
            clock = time.perf_counter() - t0
            t_burn = clock
            while clock < tmax:
                n_ep = min(int(round(epoch * args.epoch_growth ** e)), args.epoch_max)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ch.advance(n_ep, stream=stream)
                torch.cuda.synchronize()
                clock += time.perf_counter() - t0
                img = torch.zeros((side, side, 3), dtype=torch.float32, device="cuda")
                ch.resolve(out=img, stream=stream)
                stream.synchronize()
                curve.append((clock, relmse(img.double(), ref)))
                e += 1
                if curve[-1][1] <= target:
                    break
            clocks = sampler.stop()
            st = ch.stats(stream=stream, check=False)
            hit = next((t for t, r in curve if r <= target), None)
            return {"time_to_target_s": hit, "final_relmse": curve[-1][1] if curve else None, "chains": Cm,
                    "sigma": args.mala_sigma, "burn_in_s": round(t_burn, 3) if mh else None,
                    "curve": [[round(t, 3), r] for t, r in curve[:: max(1, len(curve) // 40)]],
                    "regenerations_or_large_steps": st["regenerations"], "local_steps": st["local_steps"],
                    "accepted": st["accepted"], "chain_steps": int(st["steps_per_chain"]) * Cm,
                    "status_word": st["status_word"], "clocks": clocks}

        def run_mh():
            """The MH baseline (Section 8): l = --mh-large-step, burn-in --mh-burn-in
            (Section 9: 0.3 and 10^4), --mh-chains chains; the burn-in runs on
            the clock; checkpoints after it, off the clock (no tours to drain)."""
            Cm = args.mh_chains or C
            ch = jr.Chains(g, side, side, sc.depth, Cm, seed=7, flags=jr.JR_FLAG_MH, large_step=args.mh_large_step,
                           burn_in=args.mh_burn_in, stream=stream)
            ch.set_execution("wave")
            sampler = ClockSampler(torch.cuda.current_device())
            sampler.start()
            clock, curve, e, done = 0.0, [], 0, 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while done < args.mh_burn_in:            # the burn-in: no estimate yet
                k = min(args.epoch_max, args.mh_burn_in - done)
                ch.advance(k, stream=stream)
                done += k
            torch.cuda.synchronize()
            clock = time.perf_counter() - t0
            t_burn = clock
            while clock < tmax:
                n_ep = min(int(round(epoch * args.epoch_growth ** e)), args.epoch_max)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ch.advance(n_ep, stream=stream)
                torch.cuda.synchronize()
                clock += time.perf_counter() - t0
                img = torch.zeros((side, side, 3), dtype=torch.float32, device="cuda")
                ch.resolve(out=img, stream=stream)
                stream.synchronize()
                curve.append((clock, relmse(img.double(), ref)))
                e += 1
                if curve[-1][1] <= target:
                    break
            clocks = sampler.stop()
            st = ch.stats(stream=stream, check=False)
            hit = next((t for t, r in curve if r <= target), None)
            return {"time_to_target_s": hit, "final_relmse": curve[-1][1] if curve else None, "chains": Cm,
                    "large_step": args.mh_large_step, "burn_in": args.mh_burn_in, "burn_in_s": round(t_burn, 3),
                    "curve": [[round(t, 3), r] for t, r in curve[:: max(1, len(curve) // 40)]],
                    "large_steps": st["regenerations"], "small_steps": st["local_steps"],
                    "accepted": st["accepted"], "b_hat": st["p_sum_large"] / max(1, st["regenerations"]),
                    "chain_steps": int(st["steps_per_chain"]) * Cm, "status_word": st["status_word"],
                    "clocks": clocks}

        companions = []
        if args.batched:   # companion chain sets that share the arm's batched launches
            for q, csc in enumerate(scenes.batched_workload(seed=7, n_scenes=args.batch_companions)):
                cg = jr.Scene(csc, stream=stream)
                companions.append((cg, csc))

        def run(learned, flow_dim=None):
            ch = jr.Chains(g, side, side, sc.depth, C, seed=5 if learned else 6, c_tilde=args.c_tilde, stream=stream)
            ch.set_execution("wave")
            batch, comp_sets = None, []
            if args.batched:
                # the learned + batched form: the arm's chains advance through the
                # batched wavefront (one persistent launch set for every set of the
                # batch, replayed from a CUDA graph), beside the companion sets
                comp_sets = [jr.Chains(cg, csc.width, csc.height, csc.depth, csc.width * csc.height, seed=9,
                                       stream=stream) for cg, csc in companions]
                batch = jr.Batch([ch] + comp_sets, stream=stream)
                batch.set_block(0)

            def adv(n):
                if batch is not None:
                    batch.advance_graph(n, stream=stream)
                else:
                    ch.advance(n, stream=stream)
            sampler = ClockSampler(torch.cuda.current_device())
            sampler.start()
            curve = []
            clock = 0.0
            trainer = render = None
            if learned:
                Df = flow_dim or (min(args.flow_dim, sc.D) if args.flow_dim else sc.D)
                perm, w = init_flow_params(Df, 0)
                trainer = jr.Flow(Df, perm, w, stream=stream)
                render = [jr.Flow(Df, perm, w, stream=stream), jr.Flow(Df, perm, w, stream=stream)]
                buf = jr.ReplayBuffer(sc.D, args.replay)
            e = 0
            parts = {"advance": 0.0, "train": 0.0, "drain_switch": 0.0}
            drain_steps = 0
            diag = []
            split = None
            prev = ch.stats(stream=stream)

            def lap(key, t0):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                parts[key] += t1 - t0
                return t1

            while clock < tmax:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                n_ep = min(int(round(epoch * args.epoch_growth ** e)), args.epoch_max)
                for k in range(0, n_ep, args.snap_every):
                    adv(min(args.snap_every, n_ep - k))
                    if learned:
                        buf.append(ch, stream=stream)
                t1 = lap("advance", t0)
                s0 = ch.stats(stream=stream)["steps_per_chain"]
                t1 = time.perf_counter()
                loss = None
                if learned:
                    iters = args.train_iters0 if e < args.warm_epochs else args.train_iters
                    losses = trainer.train_replay(buf, iters, batch=args.batch, lr=args.lr, seed=e, stream=stream)
                    loss = float(losses[-16:].mean()) if len(losses) else None
                    nxt = render[e % 2]
                    nxt.copy_params_from(trainer, stream=stream)
                    t1 = lap("train", t1)
                    jr.set_flow(ch, nxt, args.beta, stream=stream)   # completes the open tours first
                else:
                    jr.complete_tours(ch, stream=stream)
                t2 = lap("drain_switch", t1)
                clock += t2 - t0
                cur = ch.stats(stream=stream)
                drain_steps += cur["steps_per_chain"] - s0
                if e == args.split_epoch:  # off the clock: device time per kernel class of 16 steps
                    split = ch.advance_timed(16, stream=stream)
                    cur = ch.stats(stream=stream)
                img = torch.zeros((side, side, 3), dtype=torch.float32, device="cuda")
                ch.resolve(out=img, stream=stream)
                stream.synchronize()
                curve.append((clock, relmse(img.double(), ref)))
                dsteps = (cur["steps_per_chain"] - prev["steps_per_chain"]) * C
                if len(diag) < 24:
                    diag.append({"epoch": e, "t": round(clock, 3), "relmse": curve[-1][1], "loss": loss,
                                 "local_frac": (cur["local_steps"] - prev["local_steps"]) / max(dsteps, 1),
                                 "regen_per_step": (cur["regenerations"] - prev["regenerations"]) / max(dsteps, 1),
                                 "replay_rows": buf.rows() if learned else None})
                prev = cur
                e += 1
                if curve[-1][1] <= target:
                    break
            clocks = sampler.stop()
            st = ch.stats(stream=stream, check=False)
            hit = next((t for t, r in curve if r <= target), None)
            # log-log interpolation between the checkpoints around the crossing
            cross = None
            for (t0_, r0_), (t1_, r1_) in zip(curve, curve[1:]):
                if r0_ > target >= r1_:
                    a = (math.log(target) - math.log(r0_)) / (math.log(r1_) - math.log(r0_))
                    cross = math.exp(math.log(t0_) + a * (math.log(t1_) - math.log(t0_)))
                    break
            return {"time_to_target_s": hit, "time_to_target_interp_s": cross, "final_relmse": curve[-1][1],
                    "epochs": len(curve),
                    "curve": [[round(t, 3), r] for t, r in curve[:: max(1, len(curve) // 40)]],
                    "seconds": {k: round(v, 3) for k, v in parts.items()}, "drain_steps": drain_steps, "diag": diag,
                    "split_16_steps": split,
                    "regenerations": st["regenerations"], "local_steps": st["local_steps"],
                    "accepted": st["accepted"], "chain_steps": int(st["steps_per_chain"]) * C,
                    "status_word": st["status_word"], "clocks": clocks}

        plain = run(False) if "plain" in args.arms else None
        learned = run(True) if "learned" in args.arms.split(",") else {}
        # the flow's couplings over all D coordinates (configuration 4's statement)
        learned_full = run(True, flow_dim=sc.D) if "learned_full" in args.arms.split(",") else None
        mh = run_mh() if "mh" in args.arms.split(",") else None
        mala = run_mala(False) if "mala" in args.arms.split(",") else None
        mala_mh = run_mala(True) if "mala_mh" in args.arms.split(",") else None
    line = {"metric": METRIC, "workload": wname, "unit": "s to relMSE 1e-2",
            "relmse_eps": 1e-2, "target": target, "time_limit_s": tmax, "chains": C, "c_tilde": args.c_tilde,
            "batched": ({"companions": len(companions),
                         "companion_chains": sum(csc.width * csc.height for _, csc in companions)}
                        if args.batched else None),
            "epoch_steps": epoch,
            "epoch_growth": args.epoch_growth, "epoch_max": args.epoch_max,
            "reference": {"samples": args.ref_samples, "seconds": round(t_ref, 2), "noise_relmse_est": ref_noise},
            "plain": plain, "mh": mh, "mala": mala, "mala_mh": mala_mh,
            "learned_full_dim": None if learned_full is None else {**learned_full, "flow_dim": sc.D},
            "learned": {**learned, "beta": args.beta, "flow_dim": min(args.flow_dim, sc.D) if args.flow_dim else sc.D,
                                        "train_iters_per_epoch": args.train_iters,
                                        "train_iters_first": args.train_iters0, "warm_epochs": args.warm_epochs,
                                        "batch": args.batch, "snap_every": args.snap_every, "replay": args.replay,
                                        "lr": args.lr, "flow": "6 coupling layers, MLP 2x64, 16 bins, bf16/FP32"},
            "n_tris": sc.n_tris, "data": "synthetic"}
    return line


def default_time_to_relmse(args):
    """Metric 2 for the default line: time to relMSE 1e-2 on the slit caustic
    (1024^2, depth 10, 2^20 chains), plain against learned regeneration, with
    the harness defaults (a 2^36-sample reference, 20 s at most per arm) and a
    clock record per arm; the curves are left out of the line.  Two learned
    arms: the flow over the leading --flow-dim coordinates (the rest uniform),
    and the flow whose couplings transform all 22."""
    import copy
    a = copy.copy(args)
    a.workload, a.arms, a.chains, a.side, a.ref_samples = "caustic", "plain,learned,learned_full", 0, None, None
    a.time_limit, a.split_epoch, a.ref_file, a.c_tilde, a.batched = 20.0, -1, None, 1.0, False
    r = time_to_target(a)
    keep = ("time_to_target_s", "time_to_target_interp_s", "final_relmse", "epochs", "seconds", "clocks",
            "chain_steps", "status_word")
    out = {"workload": r["workload"], "unit": r["unit"], "target": r["target"], "relmse_eps": r["relmse_eps"],
           "chains": r["chains"], "reference": r["reference"],
           "plain": {k: r["plain"].get(k) for k in keep},
           "learned": {**{k: r["learned"].get(k) for k in keep}, "beta": r["learned"]["beta"],
                       "flow_dim": r["learned"]["flow_dim"]}}
    tp, tl = out["plain"]["time_to_target_s"], out["learned"]["time_to_target_s"]
    out["learned_over_plain"] = tl / tp if tp and tl else None   # first checkpoint at or below the target
    ip, il = out["plain"]["time_to_target_interp_s"], out["learned"]["time_to_target_interp_s"]
    out["learned_over_plain_interp"] = il / ip if ip and il else None   # log-log crossing between checkpoints
    lf = r["learned_full_dim"]
    out["learned_full_dim"] = {**{k: lf.get(k) for k in keep}, "beta": r["learned"]["beta"], "flow_dim": lf["flow_dim"]}
    tf, jf = lf["time_to_target_s"], lf["time_to_target_interp_s"]
    out["learned_full_dim_over_plain"] = tf / tp if tp and tf else None
    out["learned_full_dim_over_plain_interp"] = jf / ip if ip and jf else None
    return out


def run_reference(args, sc, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    rates = []
    cores, sample = None, None
    for _ in range(args.warmup):
        cpu_oracle_rate(sc, wl, budget_s=2.0)
    for _ in range(args.steps):
        r, cores, sample = cpu_oracle_rate(sc, wl, budget_s=args.ref_budget)
        rates.append(r)
    v = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wl["chains"] * wl["chain_steps"] / v,
            "ms_per_step_basis": "the sample's rate projected to one full step of the workload",
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}_{sc.width}x{sc.height}_depth{sc.depth}",
                       "image": [sc.width, sc.height], "depth": sc.depth, "n_tris": sc.n_tris,
                       "chains": wl["chains"], "chain_steps_per_step": wl["chain_steps"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cornell_spheres")
    ap.add_argument("--block", type=int, default=0, help="step-kernel block size (0 = library default)")
    ap.add_argument("--exec", default="auto", choices=["auto", "mega", "wave", "warp"], help="execution mode")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-t2t", action="store_true", help="skip the time-to-relMSE object of the default line")
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--chains", type=int, default=0, help="override the chain count (profiling small cases only)")
    ap.add_argument("--chain-steps", type=int, default=0, help="override chain steps per launch (profiling only)")
    ap.add_argument("--side", type=int, default=None, help="caustic/terrain workload: image side")
    ap.add_argument("--time-limit", type=float, default=60.0, help="caustic workload: seconds per arm")
    ap.add_argument("--epoch", type=int, default=128, help="caustic workload: chain steps of the first epoch")
    ap.add_argument("--epoch-growth", type=float, default=1.25, help="caustic workload: epoch length factor")
    ap.add_argument("--epoch-max", type=int, default=1024, help="caustic workload: longest epoch (steps)")
    ap.add_argument("--ref-samples", type=int, default=None,
                    help="caustic / terrain workload: reference PT samples (default 2^36 / 2^37)")
    ap.add_argument("--train-iters", type=int, default=25, help="caustic workload: Adam steps per epoch")
    ap.add_argument("--train-iters0", type=int, default=150, help="caustic workload: Adam steps in the first epochs")
    ap.add_argument("--warm-epochs", type=int, default=2)
    ap.add_argument("--batch", type=int, default=8192, help="caustic workload: training minibatch rows")
    ap.add_argument("--snap-every", type=int, default=16, help="caustic workload: steps between training snapshots")
    ap.add_argument("--replay", type=int, default=1 << 20, help="caustic workload: replay ring rows")
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--ref-file", default=None, help="caustic workload: cache the reference image in this file")
    ap.add_argument("--arms", default="plain,learned", help="caustic workload: arms to run")
    ap.add_argument("--split-epoch", type=int, default=-1, help="caustic workload: time 16 extra steps per kernel class after this epoch (diagnostic)")
    ap.add_argument("--beta", type=float, default=0.15)
    ap.add_argument("--flow-dim", type=int, default=8,
                    help="time-to-target harness: the flow models the first flow-dim coordinates, the rest "
                         "uniform (0 or >= D: all D)")
    ap.add_argument("--c-tilde", type=float, default=1.0, help="time-to-target harness: c~ of the Restore arms")
    ap.add_argument("--batched", action="store_true",
                    help="time-to-target harness: the plain and learned arms advance through a batch (batched wavefront)")
    ap.add_argument("--batch-companions", type=int, default=0,
                    help="with --batched: companion random-box chain sets in the batch (1 chain per pixel)")
    ap.add_argument("--mh-large-step", type=float, default=0.3, help="MH arm: large-step probability l")
    ap.add_argument("--mh-burn-in", type=int, default=10_000, help="MH arm: iterations before the estimate starts")
    ap.add_argument("--mh-chains", type=int, default=0, help="MH arm: chains (0 = the Restore arms' count)")
    ap.add_argument("--mala-chains", type=int, default=0, help="MALA arms: chains (0 = the Restore arms' count)")
    ap.add_argument("--mala-sigma", type=float, default=0.01, help="MALA arms: sigma of the Langevin proposal")
    args = ap.parse_args()
    if args.workload == "batched64" and args.impl == "ours":
        run_batched(args)
        return
    if args.workload in ("caustic", "terrain", "spheres_t2t") and args.impl == "ours":
        run_caustic(args)
        return
    sc, wl = workload(args.workload)
    if args.chains:
        wl["chains"] = args.chains
    if args.chain_steps:
        wl["chain_steps"] = args.chain_steps
    if args.impl == "reference":
        run_reference(args, sc, wl)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2409_07148_gb300 import jr

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    C, K = wl["chains"], wl["chain_steps"]
    from paper_2409_07148_gb300.shard import chain_range
    first, _ = chain_range(rank, ws, C * ws)   # weak scaling: C chains per rank, disjoint id ranges
    with torch.cuda.stream(stream):
        scene = jr.Scene(sc, stream=stream)
        info = scene.info()
        ch = jr.Chains(scene, sc.width, sc.height, sc.depth, C, seed=0, chain_offset=first, stream=stream)
        if args.block:
            ch.set_block_size(args.block)
        ch.set_execution(args.exec)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            ch.advance(K, stream=stream)
        stream.synchronize()
        sampler = ClockSampler(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler.start()
        times = []
        for _ in range(args.steps):
            flush.fill_(1)                      # evict the L2 between timed launches
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ch.advance(K, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        st = ch.stats(stream=stream)
        total = sum(times)
        if ws > 1:
            t = torch.tensor([total], device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total = float(t.item())
        steps_done = ws * C * K * args.steps
        value = steps_done / total
        # algorithmic work of one launch (instrumented variant on a fresh, identical chain set)
        wc = jr.Chains(scene, sc.width, sc.height, sc.depth, C, seed=0, chain_offset=first, stream=stream)
        for _ in range(args.warmup):
            wc.advance(K, stream=stream)
        work = wc.advance_counted(K, stream=stream)
        del wc
        # device time per kernel class for the same K steps of an identical chain set
        wt = jr.Chains(scene, sc.width, sc.height, sc.depth, C, seed=0, chain_offset=first, stream=stream)
        wt.set_execution(args.exec)
        for _ in range(args.warmup):
            wt.advance(K, stream=stream)
        split = wt.advance_timed(K, stream=stream)
        del wt
        flop = FLOP_PER_NODE * work["nodes"] + FLOP_PER_TRI * work["tris"]
        pk, pk_kind = peaks()
        sm_mhz_peak = float(pk.get("sm_max_mhz", 2070.0))
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        nominal_peak = sms * FP32_LANES * 2 * sm_mhz_peak * 1e6 / 1e12
        fma_tflops, fma_ms = jr.fp32_peak(stream=stream)   # measured: our FMA microbenchmark kernel
        alu_peak = fma_tflops
        split_total = sum(v["ms"] for v in split.values())
        dom = max(split, key=lambda k: split[k]["ms"])
        # the library's rule for the single-launch modes: one warp per chain when asked for, or
        # (auto) for a scene of at most 128 triangles with fewer than 32 chains per SM
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        warp = args.exec == "warp" or (args.exec == "auto" and C < 32 * n_sm and sc.n_tris <= 128)
        step_kernel_name = "step_kernel_warp" if warp else "step_kernel"
        if dom == "path":    # the traversal work runs in the path kernel
            achieved = flop / 1e12 / (split["path"]["ms"] / 1e3)
        else:                # one launch does everything (megakernel)
            achieved = flop / 1e12 / (sum(times) / args.steps)
        # end to end through the C ABI with host buffers: scene upload (BVH built on
        # the host from the caller's arrays), chain init, advance, image read back
        e2e_times = []
        h2d = info["device_bytes"] + sc.verts.nbytes + sc.tris.nbytes + sc.tri_mat.nbytes + sc.mats.nbytes
        d2h = sc.width * sc.height * 3 * 4
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = jr.Scene(sc, stream=stream)
            c2 = jr.Chains(s2, sc.width, sc.height, sc.depth, C, seed=1, chain_offset=first, stream=stream)
            c2.advance(K, stream=stream)
            img = c2.resolve(stream=stream)
            e2e_times.append(time.perf_counter() - t0)
            del c2, s2
        e2e = {"value": ws * C * K / (sum(e2e_times) / len(e2e_times)), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    t2t = None
    if not args.no_t2t and ws == 1:
        t2t = default_time_to_relmse(args)
    small = None
    if ws == 1:
        rg1, tg1 = gpu_config1(stream)
        small = {"workload": "cornell_64x64_depth3: the whole 256 chains x 10^4 steps", "value": rg1, "unit": UNIT,
                 "seconds": round(tg1, 4), "kernel": "step_kernel_warp"}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        r, cores, sample = cpu_oracle_rate(sc, wl)
        r1, _, sample1 = cpu_oracle_rate(sc, wl, budget_s=4.0, n_threads=1, max_chains=256)
        rc1, cores1, tc1 = cpu_oracle_config1()
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": r1, "unit": UNIT, "cores": 1, "sample": sample1},
               "config1_full": {"value": rc1, "unit": UNIT, "cores": cores1, "seconds": round(tc1, 3),
                                "sample": "the whole 64x64 Cornell workload: 256 chains x 10^4 steps, depth 3"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}_{sc.width}x{sc.height}_depth{sc.depth}", "model": None,
                   "scene": sc.name, "n_tris": sc.n_tris, "bvh_nodes": info["n_nodes"], "image": [sc.width, sc.height],
                   "depth": sc.depth, "dim": sc.D, "chains_per_gpu": C, "chain_steps_per_step": K, "seed": 0,
                   "c_tilde": 1.0, "sigma": 0.01, "regen": "uniform", "global_batch": ws * C, "seq_len": K,
                   "parallelism": f"chains sharded over {ws} GPU(s)", "l2": "flushed by a 512 MB write between timed launches",
                   "block": args.block or 128, "exec": args.exec},
        "roofline": {"bound": "alu", "kernel": "wf_path_kernel" if dom == "path" else step_kernel_name,
                     "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak,
                     "traffic": path_traffic(args.workload, C) if dom == "path" else None,
                     "traffic_source": PATH_TRAFFIC["summary"],
                     "peak_source": (f"measured: jr_fp32_peak, independent FMA chains on all {sms} SMs "
                                     f"({fma_ms:.2f} ms launch); nominal {sms} SMs x {FP32_LANES} lanes x 2 x "
                                     f"{sm_mhz_peak:.0f} MHz = {nominal_peak:.1f} TFLOP/s"),
                     "peak_nominal": nominal_peak, "sms": sms,
                     "work_per_step": work, "flop_per_step": flop,
                     "launches_per_step": split[dom]["launches"],
                     "avg_launch_us": 1e3 * split[dom]["ms"] / max(1, split[dom]["launches"]),
                     "flop_per_launch": flop / max(1, split[dom]["launches"]),
                     "split_ms": {k: round(v["ms"], 3) for k, v in split.items()},
                     "share": split[dom]["ms"] / split_total if split_total else None},
        "mrays_per_s": work["rays"] / (sum(times) / args.steps) / 1e6,
        "regen_fraction": st["regenerations"] / max(1, st["regenerations"] + st["local_steps"]),
        "accept_rate": st["accepted"] / max(1, st["local_steps"]),
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": args.steps * (sum(v["launches"] for v in split.values()) + 1),  # + the fold
        "cpu_baseline": cpu,
        "small_case": small,
        "time_to_relmse": t2t,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
