#!/usr/bin/env python
"""Benchmark of the Diffusion Restore hot path: Restore chain-steps/s (and
rays/s) on one or more GB300s, one process per GPU.

A timed "step" advances every chain of the workload by one Restore step
(regenerate or LocalDynamics, path contribution with NEE, hold/kill clock,
splat record, adjoint drift for survivors); the records are splatted into the
FP64 image and resolved once at the end of the timed region (inside it).

Default workload: the large procedural scene (fBm terrain + 200 tessellated
spheres/boxes, ~1M triangles, mixed Lambertian / GGX / dielectric), 1280x720,
L = 12 (d = 46), 2^20 chains, adjoint drift; inputs are larger than L2 and
L2 is also flushed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, timed on host cores

Under torchrun each rank runs an independent replica (disjoint seeds, weak
scaling).  The method's two exchanges are all-reduces outside the timed
region: the ranks agree on p_lambda at init (so every rank splats with the
same k0), and the per-rank FP64 images and tour counts are merged at the end.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2605_08916_gb300 import scenes as S  # noqa: E402

METRIC = "Restore chain-steps/s"
UNIT = "chain-steps/s"

WORKLOADS = {
    "procedural-1m-720p": dict(scene=lambda: S.procedural_scene(1, 1280, 720), L=12, chains=1 << 20,
                               drift="adjoint", spp=4, cpu_chains=64),
    "cornell-glossy-256": dict(scene=lambda: S.cornell_box(1, 256, 256, glossy=True), L=8, chains=65536,
                               drift="adjoint", spp=16, cpu_chains=256),
    "caustic-20k-512": dict(scene=lambda: S.caustic_scene(1, 512, 512), L=10, chains=262144, drift="adjoint",
                            spp=16, cpu_chains=128),
    "cornell-64-fd": dict(scene=lambda: S.cornell_box(1, 64, 64), L=4, chains=4096, drift="fd", spp=16,
                          cpu_chains=128),
    # the procedural layout with its 200 objects as instances of two meshes
    # (two-level BVH); the oracle renders its flattening
    "procedural-instanced-1m-720p": dict(scene=lambda: S.procedural_scene_instanced(1, 1280, 720), L=12,
                                         chains=1 << 20, drift="adjoint", spp=4, cpu_chains=64),
}


def flat_of(scene):
    """The flat scene the oracle takes (an instanced scene's flattening)."""
    return scene.flatten() if isinstance(scene, S.InstancedScene) else scene


def upload(r, scene):
    if isinstance(scene, S.InstancedScene):
        r.upload_instanced(scene)
    else:
        r.upload_scene(scene)


def input_bytes(scene):
    """Host bytes an upload copies (the scene arrays)."""
    if isinstance(scene, S.InstancedScene):
        n = sum(a.nbytes for m in scene.meshes for a in (m.verts, m.tris, m.tri_mat) if a is not None)
        n += sum(m.normals.nbytes for m in scene.meshes if m.normals is not None)
        return n + 56 * len(scene.instances) + scene.materials.nbytes + scene.camera.nbytes
    n = sum(a.nbytes for a in (scene.verts, scene.tris, scene.tri_mat, scene.materials, scene.camera))
    return n + (scene.normals.nbytes if scene.normals is not None else 0)


DEFAULT = "procedural-1m-720p"
SEED = 0x5EED


TRAFFIC_SOURCES = ["dr_common.cuh", "dr_trace.cuh", "dr_path.cuh", "dr_step.cuh", "dr_internal.h", "dr_wavefront.cu",
                   "dr_bvh.cu", "dr_bvh4.cu"]


def traversal_traffic(workload, n_chains):
    """DRAM bytes per step of the traversal passes from the committed ncu
    capture for this workload, if the traversal sources are unchanged since
    (their sha256 matches); else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"wf_traverse_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if line.strip() and not line.startswith("#") and ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2605_08916_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != kv.get("source_sha256") or int(kv.get("chains", 0)) != n_chains:
        return None
    return int(kv["dram_read_bytes_per_step"]) + int(kv["dram_write_bytes_per_step"])


def measured_peaks():
    """HBM copy bandwidth (GB/s) measured on this machine's GPUs, else the
    earlier GB300 measurement of 6.8 TB/s, marked "fallback"."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "measured"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line is the only stdout output)."""
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(wl, scene, steps=8, target_s=15.0):
    """The FP64 oracle, as it stands, on this host's cores: a bounded sample
    of the same workload (the first m of its chains for init + `steps`
    steps), sized by a calibration run to about target_s seconds."""
    from oracle import oracle as O
    tgt = O.OracleScene(scene)
    cores = O.num_threads()
    prm = O.make_params(L=wl["L"], drift="exact" if wl["drift"] == "adjoint" else wl["drift"], rb=True, k0=1.0)
    # p_lambda estimate on a uniform sample sets k0 as the GPU run does
    est = O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(4096), n_steps=0, record=False)
    prm.k0 = est["p_init_sum"] / 4096 / (64.0 * 1e-5)
    m = 1024
    while True:
        t0 = time.perf_counter()
        O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(m), n_steps=steps, record=False, accum=False)
        dt = time.perf_counter() - t0
        if dt > 1.0 or m >= wl["chains"]:
            break
        m = min(wl["chains"], m * 4)
    m = int(max(16, min(wl["chains"], m * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(m), n_steps=steps, record=False, accum=False)
    dt = time.perf_counter() - t0
    units = m * (steps + 1)
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} chains x {steps + 1} steps (init + {steps}) of the workload, FP64, OpenMP",
            "seconds": dt}


def run_reference(args, wl, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on this host's
    cores, timing init + args.steps steps of a bounded sample of the
    workload's chains (sized by a calibration run so that the timed run
    takes about ten seconds), after args.warmup untimed one-step runs."""
    if rank != 0:
        return 0
    scene = flat_of(wl["scene"]())
    from oracle import oracle as O
    tgt = O.OracleScene(scene)
    prm = O.make_params(L=wl["L"], drift="exact" if wl["drift"] == "adjoint" else wl["drift"], rb=True, k0=1.0)
    est = O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(4096), n_steps=0, record=False)
    prm.k0 = est["p_init_sum"] / 4096 / (64.0 * 1e-5)
    for _ in range(args.warmup):
        O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(256), n_steps=1, record=False, accum=False)
    m = 1024
    while True:
        t0 = time.perf_counter()
        O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(m), n_steps=args.steps, record=False, accum=False)
        dt = time.perf_counter() - t0
        if dt > 1.0 or m >= wl["chains"]:
            break
        m = min(wl["chains"], m * 4)
    m = int(max(256, min(wl["chains"], m * 10.0 / max(dt, 1e-3))))
    t0 = time.perf_counter()
    O.restore_run(tgt, prm, seed=SEED, chain_ids=np.arange(m), n_steps=args.steps, record=False, accum=False)
    dt = time.perf_counter() - t0
    value = m * (args.steps + 1) / dt
    sample = f"{m} chains x {args.steps + 1} steps (init + {args.steps}) of the workload, FP64 oracle, OpenMP"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / (args.steps + 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "chains": m, "max_path_len": wl["L"], "triangles": scene.n_tris,
                       "image": [scene.width, scene.height], "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, wl, rank, world, local):
    import torch
    from paper_2605_08916_gb300 import renderer as R
    from paper_2605_08916_gb300.replicas import init_chains_agreed, merge_and_resolve, replica_seed

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    scene = wl["scene"]()
    log(f"scene {scene.name}: {scene.n_tris} triangles")
    N = args.chains or wl["chains"]
    F = wl["spp"]                                   # steps per frame (one graph replay)
    params = R.make_params(L=wl["L"], drift=wl["drift"], rb=True, k0=0.0, steps_per_splat=F)
    seed = replica_seed(SEED, rank)
    stream = torch.cuda.Stream(device=dev)          # graph capture needs a created stream
    r = R.Renderer(local, stream)
    r.set_option("work_order", args.work_order)
    r.set_option("wavefront", args.wavefront)
    r.set_option("bvh_width", args.bvh_width)
    r.set_option("ray_order", args.ray_order)
    r.set_option("two_level", args.two_level)
    if args.ploc_radius:
        r.set_bvh_builder("ploc", args.ploc_radius)
    if args.tail_bounce is not None:
        r.set_option("tail_bounce", args.tail_bounce)
    upload(r, scene)
    stream.synchronize()
    t_init = time.perf_counter()
    if world > 1:
        # Alg. 1 with one k0 on every replica: p_lambda over all ranks' samples
        init_chains_agreed(r, N, seed, params, device=dev)
    else:
        r.init_chains(N, seed, params)
    stream.synchronize()
    t_init = time.perf_counter() - t_init
    log(f"init (evaluation + p_lambda estimate + clock) {t_init * 1e3:.1f} ms")
    bvh4 = r.bvh4_info() if args.bvh_width != 2 else None
    bvh8 = r.bvh8_info() if args.bvh_width == 8 else None
    two_level = r.two_level_info() if isinstance(scene, S.InstancedScene) and args.two_level else None
    sah4 = r.bvh4_sah() if bvh4 else None
    log(f"uploaded + init {N} chains; bvh {r.bvh_info()}; 4-wide {bvh4}; 8-wide {bvh8}; two-level {two_level}")
    # traversal statistics (separate kernel instantiation, untimed)
    r.set_stats(True)
    r.step(2)
    ts = r.traversal_stats()
    r.set_stats(False)
    chain_steps_stats = 2 * N
    d = 2 + 4 * (wl["L"] - 1)
    # node size of the BVH the stats pass traversed: 4-wide in the
    # bounce-by-bounce passes unless disabled; the fused kernel (automatic
    # width) walks the binary one
    wf_expected = wl["drift"] == "adjoint" and (args.wavefront == 1 or (args.wavefront == -1 and N >= 1 << 17))
    wide = bool(bvh4)
    # the 8-wide compressed BVH serves the bounce-by-bounce passes only
    node_bytes = 80 if (bvh8 and wf_expected) else 112 if wide else 64
    trav_bytes = (ts["node_visits"] * node_bytes + ts["tri_tests"] * 48) / chain_steps_stats
    state_bytes = 4 * d * 4 + 1 + 1 + 4 + 16   # x and score read+write, killed r+w, logp, record
    log(f"stats pass: {ts}")
    # per-phase device time (events around each pass; untimed) for the roofline
    r.set_option("profile", 1)
    r.profile()
    prof_steps = 4
    r.step(prof_steps)
    bprof = r.bounce_profile(wl["L"])
    prof = r.profile()
    r.set_option("profile", 0)
    wavefront = prof["trace"][1] > 0
    assert wavefront == wf_expected, "execution mode differs from the one the roofline bytes assume"
    if wavefront:
        k_name = ("wf_traverse (two-level BVH traversal passes)" if two_level
                  else "wf_traverse (8-wide compressed BVH traversal passes)" if bvh8
                  else "wf_traverse (4-wide BVH traversal passes)" if wide
                  else "wf_trace + wf_shadow (binary BVH traversal passes)")
        # the persistent tail pass (long paths) traverses too: its node
        # visits are in the statistics, so its time is in the denominator
        # (with its shading, which makes the fraction a lower bound)
        k_ms = (prof["trace"][0] + prof["shadow"][0] + prof["tail"][0]) / prof_steps
        k_bytes = trav_bytes
    else:
        k_name = "step_kernel (fused Restore step)"
        k_ms = (prof["fused_step"][0] + prof["fd_score"][0]) / prof_steps
        k_bytes = trav_bytes + state_bytes
    log(f"profile per step: " + ", ".join(f"{k} {v[0] / prof_steps:.3f} ms" for k, v in prof.items() if v[1]))
    # warm-up frames (also captures the frame graph)
    n_frames = max(1, (args.steps + F - 1) // F)
    steps = n_frames * F
    for _ in range(max(1, (args.warmup + F - 1) // F)):
        r.frame(F)
    stream.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    c0 = r.counters()
    l0 = r.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames + 1)]
    img = torch.empty((scene.height, scene.width, 3), dtype=torch.float32, device=dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(n_frames):
                flush.zero_()
                ev[k][0].record(stream)
                r.frame(F)
                ev[k][1].record(stream)
            flush.zero_()
            ev[-1][0].record(stream)
            r.resolve(img)
            ev[-1][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(times)
    launches = r.launch_count() - l0
    c1 = r.counters()
    rays = c1["rays"] - c0["rays"]
    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
        # the method's one exchange: merge the FP64 images and tour counts
        merge_and_resolve(torch.from_numpy(r.readback_accum()).to(dev), c1["tour_count"], c1["k0"],
                          resolve=R.resolve_accum)
    value = N * steps * world / (t_max / 1e3)
    rays_s = rays * world / (t_max / 1e3)
    peak, peak_kind = measured_peaks()
    achieved = k_bytes * N / (k_ms / 1e3) / 1e9
    clocks = clk.summary()
    if rank == 0:
        log(f"timed {steps} steps in {n_frames} frames: {total_ms:.1f} ms")
        e2e = None if args.no_e2e else run_e2e(R, scene, wl, N, steps, local, stream)
        rel = None if args.no_relmse else run_relmse33(R, scene, wl, local)
        others = None
        if not args.no_other and world == 1:
            others = [measure_workload(R, n, local) for n in OTHER_WORKLOADS if n != args.workload]
            others.append(measure_batch(R, local))
            for o in others:
                log(f"other workload {o['workload']}: {o['value'] / 1e6:.1f} M chain-steps/s, "
                    f"roofline {o['roofline']['frac']:.3f}")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": t_max / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "scene": scene.name, "triangles": scene.n_tris,
                           "image": [scene.width, scene.height], "chains_per_gpu": N, "max_path_len": wl["L"],
                           "pss_dim": d, "drift": wl["drift"], "rb_weight": True, "steps_per_frame": F,
                           "execution": "wavefront" if wavefront else "fused",
                           "bvh_sah": sah4,
                           "bvh": ("two-level (4-wide TLAS over instances, 4-wide BLAS per mesh)" if two_level
                                   else "8-wide compressed" if (bvh8 and wavefront) else "4-wide" if wide
                                   else "binary"),
                           "frame": "CUDA graph of steps_per_frame steps + splat, replayed",
                           "l2": "inputs > L2 (BVH + chain state) and a 512 MB L2 flush between timed frames",
                           "parallelism": f"replicas{world}"},
                "rays_per_s": rays_s, "rays_per_chain_step": rays / max(1, N * steps),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak,
                             "traffic": traversal_traffic(args.workload, N) if wavefront and wide else None,
                             "basis": "per Restore step: all traversal launches of the step (achieved = "
                                      "algorithmic bytes per step / their time; traffic = their DRAM bytes)",
                             "peak_kind": peak_kind, "kernel": k_name, "kernel_ms_per_step": k_ms,
                             "algorithmic_bytes_per_chain_step": k_bytes,
                             "node_visits_per_chain_step": ts["node_visits"] / chain_steps_stats,
                             "tri_tests_per_chain_step": ts["tri_tests"] / chain_steps_stats},
                "phase_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items() if v[1]},
                "bounce_ms_per_step": {k: [round(x / prof_steps, 4) for x in v] for k, v in bprof.items()
                                       if k in ("trace", "shade", "shadow")} if wavefront else None,
                "bounce_rays_per_step": {k: [int(x // prof_steps) for x in v] for k, v in bprof.items()
                                         if k in ("rays", "shadow_rays")}
                if wavefront else None,
                "clocks": clocks, "gpu_launches": launches, "e2e": e2e, "relmse_33ms": rel,
                "other_workloads": others}
        if world == 1 and not args.no_cpu_baseline:
            cb = cpu_baseline(wl, flat_of(scene))
            cb["per_core"] = cb["value"] / max(1, cb["cores"])
            # the oracle traces the same paths (same Philox streams), so its
            # rays per chain-step are the ones counted on the GPU
            cb["rays_per_s"] = cb["value"] * line["rays_per_chain_step"]
            line["cpu_baseline"] = cb
            log("cpu baseline done")
        print(json.dumps(line), flush=True)
    r.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


OTHER_WORKLOADS = ["caustic-20k-512", "cornell-glossy-256", "cornell-64-fd"]


def measure_workload(R, name, local, steps=16, warmup=4):
    """A short measurement of another configuration in the same process:
    chain-steps/s over `steps` steps in graph frames (inputs > L2 or a 512 MB
    L2 flush between frames), the traversal roofline from the statistics
    pass and the profiled phases, as in the main measurement."""
    import torch
    wl = WORKLOADS[name]
    dev = torch.device("cuda", local)
    scene = wl["scene"]()
    N, F = wl["chains"], wl["spp"]
    stream = torch.cuda.Stream(device=dev)
    r = R.Renderer(local, stream)
    upload(r, scene)
    r.init_chains(N, SEED, R.make_params(L=wl["L"], drift=wl["drift"], rb=True, k0=0.0, steps_per_splat=F))
    r.set_stats(True)
    r.step(2)
    ts = r.traversal_stats()
    r.set_stats(False)
    bvh4 = r.bvh4_info()
    r.set_option("profile", 1)
    r.profile()
    r.step(4)
    prof = r.profile()
    r.set_option("profile", 0)
    wavefront = prof["trace"][1] > 0
    d = 2 + 4 * (wl["L"] - 1)
    trav = (ts["node_visits"] * (112 if bvh4 else 64) + ts["tri_tests"] * 48) / (2 * N)
    if wavefront:
        k_ms, k_bytes = (prof["trace"][0] + prof["shadow"][0] + prof["tail"][0]) / 4, trav
    else:
        k_ms = (prof["fused_step"][0] + prof["fd_score"][0]) / 4
        k_bytes = trav + 4 * d * 4 + 1 + 1 + 4 + 16
    n_frames = max(1, steps // F)
    for _ in range(max(1, warmup // F)):
        r.frame(F)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    c0 = r.counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(n_frames):
            flush.zero_()
            ev[k][0].record(stream)
            r.frame(F)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    c1 = r.counters()
    r.close()
    peak, peak_kind = measured_peaks()
    achieved = k_bytes * N / (k_ms / 1e3) / 1e9
    return {"workload": name, "triangles": scene.n_tris, "image": [scene.width, scene.height], "chains": N,
            "max_path_len": wl["L"], "drift": wl["drift"], "execution": "wavefront" if wavefront else "fused",
            "value": N * n_frames * F / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / (n_frames * F),
            "steps": n_frames * F, "rays_per_s": (c1["rays"] - c0["rays"]) / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "kernel_ms_per_step": k_ms,
                         "algorithmic_bytes_per_chain_step": k_bytes}}


def measure_batch(R, local, steps=16, F=4):
    """A short measurement of the 64-scene batch (configuration 5) in the
    same process, with the library's default schedule (the full run,
    `--workload batched-64`, autotunes it and adds the per-scene baseline)."""
    import torch
    dev = torch.device("cuda", local)
    items = S.procedural_batch()
    N = sum(n for _, _, n in items)
    stream = torch.cuda.Stream(device=dev)
    r = R.Renderer(local, stream)
    r.upload_scenes(items)
    r.init_chains(N, SEED, R.make_params(L=16, drift="adjoint", rb=True, k0=0.0, steps_per_splat=F))
    r.set_stats(True)
    r.step(2)
    ts = r.traversal_stats()
    r.set_stats(False)
    r.set_option("profile", 1)
    r.profile()
    r.step(4)
    prof = r.profile()
    r.set_option("profile", 0)
    trav = (ts["node_visits"] * 112 + ts["tri_tests"] * 48) / (2 * N)
    k_ms = (prof["trace"][0] + prof["shadow"][0] + prof["tail"][0]) / 4
    for _ in range(2):
        r.frame(F)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    n_frames = max(1, steps // F)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
    c0 = r.counters()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(n_frames):
            flush.zero_()
            ev[k][0].record(stream)
            r.frame(F)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    c1 = r.counters()
    r.close()
    peak, peak_kind = measured_peaks()
    achieved = trav * N / (k_ms / 1e3) / 1e9
    return {"workload": "batched-64", "scenes": len(items), "triangles": sum(sc.n_tris for sc, _, _ in items),
            "chains": N, "schedule": "library default", "execution": "wavefront (one batch)",
            "value": N * n_frames * F / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / (n_frames * F),
            "steps": n_frames * F, "rays_per_s": (c1["rays"] - c0["rays"]) / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "kernel_ms_per_step": k_ms,
                         "algorithmic_bytes_per_chain_step": trav}}


BUDGET_MS = 1000.0 / 30.0


def relmse(img, ref):
    """mean over pixels and channels of (I - R)^2 / (R^2 + 1e-2)"""
    return float(np.mean((img - ref) ** 2 / (ref ** 2 + 1e-2)))


def bias_variance(imgs, ref):
    """Split of the relMSE over seeds: per seed it is (I - R)^2 / (R^2 + 1e-2)
    averaged over pixels and channels; its mean over seeds is the weighted
    squared bias of the mean image plus the weighted variance.  Returns
    (mean relMSE, its standard deviation over seeds, squared bias,
    variance), the bias corrected for the variance left in the mean of the
    seeds."""
    imgs = np.stack(imgs).astype(np.float64)
    w = 1.0 / (ref ** 2 + 1e-2)
    per = [float(np.mean((im - ref) ** 2 * w)) for im in imgs]
    n = imgs.shape[0]
    mean = imgs.mean(0)
    var = float(np.mean(imgs.var(0, ddof=1) * w))
    bias2 = max(0.0, float(np.mean((mean - ref) ** 2 * w)) - var / n)
    return statistics.mean(per), statistics.stdev(per), bias2, var


def run_relmse33(R, scene, wl, local, seeds=16):
    """Image relMSE after one 33.3 ms frame budget, from scratch (chain init
    with the p_lambda estimate, the steps, the splat and the resolve all
    inside the budget).  Forms:
      plain_fd         finite-difference drift, one launch sequence per step;
      batched_adjoint  adjoint drift, bounce-by-bounce passes, all steps of
                       the frame in one CUDA graph;
      batched_none     the same without a drift (LocalDynamics with a zero
                       score), the ablation of the drift at equal budget;
      graph_fd         finite-difference drift, all steps in one CUDA graph;
      mala_restore     MALA Restore (Sec. 6's comparison method: Metropolis-
                       adjusted Langevin moves, holding rate 1), fused
                       kernel, all steps in one CUDA graph;
      pt               path tracing of the same f (stratified film
                       samples), as many samples per pixel as fit the budget.
    Each Restore form takes the largest chain count (halving from the
    workload's) that fits at least two steps; the steps are calibrated to
    the budget.  Each form reports the mean relMSE over seeds split into the
    squared bias of the seeds' mean image and the variance.  Reference:
    path tracing of the same f with a fixed large sample count."""
    import torch
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    rr = R.Renderer(local, stream)
    upload(rr, scene)
    t0 = time.perf_counter()
    rr.pt_render(wl["L"], 4, seed=99)
    stream.synchronize()
    per_spp = (time.perf_counter() - t0) / 4
    spp_ref = int(max(64, min(4096, 2 ** int(np.log2(max(1.0, 20.0 / max(per_spp, 1e-6)))))))
    t0 = time.perf_counter()
    ref = rr.pt_render(wl["L"], spp_ref, seed=12345).cpu().numpy()
    t_ref = time.perf_counter() - t0
    log(f"relmse: reference PT {spp_ref} spp in {t_ref:.1f} s")
    out = {"budget_ms": BUDGET_MS, "seeds": seeds, "reference": f"path tracing, {spp_ref} spp, same f",
           "metric": "mean over pixels and channels of (I-R)^2/(R^2+1e-2)",
           "split": "relmse_mean = bias2 (squared bias of the mean image over seeds) + variance (per seed)"}
    # path tracing at the same budget: the render of spp samples per pixel
    # from scratch, its result on the device
    def pt_ms(spp, seed):
        stream.synchronize()
        t0 = time.perf_counter()
        img_pt = rr.pt_render(wl["L"], spp, seed=seed)
        stream.synchronize()
        return (time.perf_counter() - t0) * 1e3, img_pt
    pt_ms(1, 5)
    t1 = min(pt_ms(1, 6 + k)[0] for k in range(2))
    t4 = min(pt_ms(4, 8 + k)[0] for k in range(2))
    per = max((t4 - t1) / 3, 1e-3)
    spp = max(1, int((0.97 * BUDGET_MS - (t1 - per)) / per))
    while spp > 1 and min(pt_ms(spp, 10 + k)[0] for k in range(2)) > 0.97 * BUDGET_MS:
        spp -= 1
    imgs, times = [], []
    for k in range(seeds):
        ms, im = pt_ms(spp, 2000 + k)
        times.append(ms)
        imgs.append(im.cpu().numpy())
    rm, sd, b2, var = bias_variance(imgs, ref)
    out["pt"] = {"spp": spp, "frame_ms_mean": statistics.mean(times), "frame_ms_max": max(times),
                 "relmse_mean": rm, "relmse_sd": sd, "bias2": b2, "variance": var}
    log(f"relmse pt: {spp} spp, frame {statistics.mean(times):.1f} ms, relMSE {rm:.4g} (bias2 {b2:.3g}, var {var:.3g})")
    rr.close()
    img = torch.empty((scene.height, scene.width, 3), dtype=torch.float32, device=torch.device("cuda", local))
    forms = {"plain_fd": ("fd", False), "batched_adjoint": ("adjoint", True), "batched_none": ("none", True),
             "graph_fd": ("fd", True), "mala_restore": ("mala", True)}
    for form, (drift, graph) in forms.items():
        r = R.Renderer(local, stream)
        upload(r, scene)
        if drift in ("fd", "mala"):
            r.set_option("wavefront", 0)
        F = wl["spp"]
        # MALA Restore runs with the paper's holding rate 1 (dt = 1)
        prm = R.make_params(L=wl["L"], drift=drift, rb=True, k0=0.0, steps_per_splat=F,
                            dt=1.0 if drift == "mala" else 1e-5)

        def run(n, steps, seed):
            stream.synchronize()
            t0 = time.perf_counter()
            r.init_chains(n, seed, prm)
            if graph:
                r.frame(steps)
            else:
                r.step(steps)
            r.resolve(img)
            stream.synchronize()
            return (time.perf_counter() - t0) * 1e3

        n = wl["chains"]
        while True:
            for steps in (2, 4):            # warm-up (graph capture), then calibration
                run(n, steps, 7)
            ta = min(run(n, 2, 8 + k) for k in range(2))
            tb = min(run(n, 4, 10 + k) for k in range(2))
            t_step = max((tb - ta) / 2, 1e-3)
            t_fixed = ta - 2 * t_step
            steps = int((0.97 * BUDGET_MS - t_fixed) / t_step)
            if steps >= 2 or n <= 4096:
                break
            n //= 2
        steps = max(1, steps)
        run(n, steps, 9)                    # capture at the final step count
        imgs, times = [], []
        for k in range(seeds):
            times.append(run(n, steps, 1000 + k))
            imgs.append(img.cpu().numpy().astype(np.float64))
        r.close()
        rm, sd, b2, var = bias_variance(imgs, ref)
        out[form] = {"drift": drift, "graph": graph, "chains": n, "steps": steps, "ms_per_step": t_step,
                     "ms_fixed": t_fixed, "frame_ms_mean": statistics.mean(times), "frame_ms_max": max(times),
                     "relmse_mean": rm, "relmse_sd": sd, "bias2": b2, "variance": var}
        log(f"relmse {form}: {n} chains x {steps} steps, frame {statistics.mean(times):.1f} ms, "
            f"relMSE {rm:.4g} +- {sd:.2g} (bias2 {b2:.3g}, var {var:.3g})")
    out["ratio_plain_over_batched"] = out["plain_fd"]["relmse_mean"] / out["batched_adjoint"]["relmse_mean"]
    out["ratio_pt_over_batched"] = out["pt"]["relmse_mean"] / out["batched_adjoint"]["relmse_mean"]
    return out


def run_e2e(R, scene, wl, N, steps, local, stream):
    """Same metric through the public API with host buffers: scene arrays
    copied host -> device (upload + BVH build), chain init with the p_lambda
    estimate, the steps, resolve, and the image copied device -> host."""
    import torch
    h2d = input_bytes(scene)
    out = torch.empty((scene.height, scene.width, 3), dtype=torch.float32, device=torch.device("cuda", local))
    host = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = R.Renderer(local, stream)
    upload(r, scene)
    r.init_chains(N, SEED + 1, R.make_params(L=wl["L"], drift=wl["drift"], rb=True, k0=0.0,
                                            steps_per_splat=wl["spp"]))
    F = wl["spp"]
    for _ in range(steps // F):
        r.frame(F)
    r.resolve(out)
    with torch.cuda.stream(stream):
        host.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    r.close()
    d2h = out.numel() * 4
    return {"value": N * steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "seconds": dt, "includes": "scene upload + BVH build + init (p_lambda estimate) + steps + resolve + image D2H"}


def run_batched(args, rank, world, local):
    """The multi-scene workload: 64 procedural variants (1k-200k triangles,
    128^2-512^2 images, L 4-16, 2^21 chains split by pixel count) advanced as
    one batch (every step of every scene in one sequence of bounce-by-bounce
    launches, frames captured as CUDA graphs, schedule chosen by the
    autotuner), against plain per-scene per-step launches (one context per
    scene, each stepped on its own)."""
    import torch
    from paper_2605_08916_gb300 import autotune as AT
    from paper_2605_08916_gb300 import renderer as R
    from paper_2605_08916_gb300.replicas import replica_seed
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    items = S.procedural_batch()
    N = sum(n for _, _, n in items)
    tris = sum(sc.n_tris for sc, _, _ in items)
    pixels = sum(sc.width * sc.height for sc, _, _ in items)
    log(f"batch: {len(items)} scenes, {tris} triangles, {pixels} pixels, {N} chains")
    stream = torch.cuda.Stream(device=dev)
    r = R.Renderer(local, stream)
    r.set_option("ray_order", args.ray_order)
    if args.bvh_width == 8:
        r.set_option("bvh_width", 8)
    if args.tail_bounce is not None:
        r.set_option("tail_bounce", args.tail_bounce)
    r.upload_scenes(items)
    seed = replica_seed(SEED, rank)
    prm = R.make_params(L=16, drift="adjoint", rb=True, k0=0.0, steps_per_splat=8)
    best, table = AT.autotune(r, stream, N, seed, prm)
    F = best["steps_per_frame"]
    log(f"autotuned schedule {best}; top: " +
        ", ".join(f"{ms:.2f} ms {c}" for ms, c in sorted(table, key=lambda t: t[0])[:3]))
    r.init_chains(N, seed, prm)
    r.set_stats(True)
    r.step(2)
    ts = r.traversal_stats()
    r.set_stats(False)
    trav_bytes = (ts["node_visits"] * (80 if args.bvh_width == 8 else 112) + ts["tri_tests"] * 48) / (2 * N)
    r.set_option("profile", 1)
    r.profile()
    prof_steps = 4
    r.step(prof_steps)
    prof = r.profile()
    r.set_option("profile", 0)
    # the tail pass's node visits are counted, so its time is too (it also
    # shades: the fraction is a lower bound when the tail pass runs)
    k_ms = (prof["trace"][0] + prof["shadow"][0] + prof["tail"][0]) / prof_steps
    n_frames = max(1, (args.steps + F - 1) // F)
    steps = n_frames * F
    for _ in range(max(1, (args.warmup + F - 1) // F)):
        r.frame(F)
    stream.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    l0 = r.launch_count()
    c0 = r.counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(n_frames):
                flush.zero_()
                ev[k][0].record(stream)
                r.frame(F)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = r.launch_count() - l0
    rays = r.counters()["rays"] - c0["rays"]
    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    value = N * steps * world / (t_max / 1e3)
    imgs_ok = all(torch.isfinite(r.resolve_scene(s)).all().item() for s in range(len(items)))
    r.close()
    clocks = clk.summary()
    if rank != 0:
        return 0
    # plain per-scene per-step launches
    plain_r = []
    for s_i, (sc, L, n) in enumerate(items):
        rp = R.Renderer(local, stream)
        rp.upload_scene(sc)
        seed_s = (seed & 0xFFFFFFFF) | ((((seed >> 32) + s_i) & 0xFFFFFFFF) << 32)  # the batch's key for scene s_i
        rp.init_chains(n, seed_s, R.make_params(L=L, drift="adjoint", rb=True, k0=0.0, steps_per_splat=8))
        plain_r.append(rp)
    for rp in plain_r:
        rp.step(1)
    stream.synchronize()
    p_steps = 4
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(p_steps):
        for rp in plain_r:
            rp.step(1)
    e1.record(stream)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1)
    for rp in plain_r:
        rp.close()
    plain_value = N * p_steps / (plain_ms / 1e3)
    peak, peak_kind = measured_peaks()
    achieved = trav_bytes * N / (k_ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": t_max / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched-64", "scenes": len(items), "triangles": tris, "pixels": pixels,
                       "chains_per_gpu": N, "max_path_len": [4, 16], "drift": "adjoint", "rb_weight": True,
                       "execution": "one batch: every scene's chains in one sequence of bounce-by-bounce launches",
                       "steps_per_frame": F, "schedule": best, "frame": "CUDA graph, replayed",
                       "l2": "512 MB L2 flush between timed frames", "parallelism": f"replicas{world}"},
            "rays_per_s": rays * world / (t_max / 1e3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": peak_kind, "kernel": "wf_traverse (batch instantiation)",
                         "kernel_ms_per_step": k_ms, "algorithmic_bytes_per_chain_step": trav_bytes},
            "phase_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items() if v[1]},
            "plain_per_scene": {"value": plain_value, "unit": UNIT, "steps": p_steps, "ms_per_step": plain_ms / p_steps,
                                "execution": "64 contexts, each stepped with its own launches (dr_step per scene)"},
            "speedup_vs_plain": value / plain_value, "images_finite": imgs_ok,
            "autotune": [{"ms_per_step": round(ms, 4), **c} for ms, c in sorted(table, key=lambda t: t[0])],
            "clocks": clocks, "gpu_launches": launches, "e2e": None}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + ["batched-64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run (profiling cases)")
    ap.add_argument("--no-relmse", action="store_true", help="skip the 33 ms image relMSE comparison")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the short measurements of the other configurations (caustic, Cornell)")
    ap.add_argument("--chains", type=int, default=0, help="override the workload's chain count (profiling cases)")
    ap.add_argument("--wavefront", type=int, default=-1, choices=[-1, 0, 1],
                    help="bounce-by-bounce execution over compacted path queues: 1 on, 0 fused kernel, "
                         "-1 (default) by chain count")
    ap.add_argument("--tail-bounce", type=int, default=None,
                    help="run the bounces from this one on as one persistent pass (0 off; default: library's choice)")
    ap.add_argument("--ray-order", type=int, default=-1, choices=[-1, 0, 1],
                    help="sort camera rays by pixel before the first traversal (-1: by triangle count)")
    ap.add_argument("--ploc-radius", type=int, default=0,
                    help="PLOC search radius of the BVH build (0: the library default, 16)")
    ap.add_argument("--two-level", type=int, default=0, choices=[0, 1],
                    help="instanced workloads: walk the two-level BVH (1) or the flattened one (0)")
    ap.add_argument("--bvh-width", type=int, default=0, choices=[0, 2, 4, 8],
                    help="BVH the rays traverse: 4-wide (0, the default, or 4) or binary (2)")
    ap.add_argument("--work-order", type=int, default=0, choices=[0, 1],
                    help="fused kernel only: order chains by expected path cost (default 0)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    wl = WORKLOADS.get(args.workload)
    if args.workload == "batched-64":
        if args.impl == "reference":
            wl = WORKLOADS[DEFAULT]
            return run_reference(args, wl, rank, world)
        return run_batched(args, rank, world, local)
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    return run_ours(args, wl, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
