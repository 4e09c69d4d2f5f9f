#!/usr/bin/env python
"""Benchmark: RGB-D frames/s of the sensor-rendering hot path on one B300.

Default workload (N=1): the 1M-triangle synthetic house with a 4096^2 RGBA8
atlas, 64 agents at random navigable poses, 256x256 RGB + depth — one step
renders all 64 views in one batched launch. `--mode plain` renders the same
views one agent per launch. The batched step is one replay of a
graph-captured persistent batch (hsr_batch_render). The default run (one
GPU) adds sub-records for the rest of the metric: the 128^2 batching
workload (8 scenes, 1,024 agents), the 2M-triangle 512^2 workload, and
serving at 10k and 50k requests/s with p50/p99 latency (`--no-sub` skips
them). `--impl reference` times the CPU oracle (the reference arm: there is
no runnable code of the paper) on the view sequence cpu_baseline renders.

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas (the
path has no exchange step); value is the sum of all ranks' frames over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RGB-D frames/sec (batched vs plain)"
# kernels per render call: cull, 3 raster phases, 2 hierarchical-z builds, shade
def kernels_per_call(n_phases: int) -> int:
    """Kernels one render call launches: cull (with the z-buffer clear), per
    occlusion phase a raster and a large-triangle raster, before every phase
    after the first a tile-z build, its pyramid and the occlusion test, shade."""
    P = max(1, int(n_phases))
    return 1 + 2 * P + 3 * (P - 1) + 1
UNIT = "frames/s"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6400.0

KERNEL_SOURCES = ["paper_1904_01201_b300/csrc/render.cu", "paper_1904_01201_b300/csrc/hsr_internal.h",
                  "paper_1904_01201_b300/csrc/kernels/transform.cuh", "paper_1904_01201_b300/csrc/kernels/setup.cuh",
                  "paper_1904_01201_b300/csrc/kernels/bin.cuh", "paper_1904_01201_b300/csrc/kernels/raster.cuh",
                  "paper_1904_01201_b300/csrc/kernels/shade.cuh", "paper_1904_01201_b300/csrc/kernels/bulk.cuh"]


def d2h_link_gbs(dev, nbytes: int = 256 << 20) -> float:
    """Device -> page-locked host copy bandwidth (GB/s), best of three."""
    import torch
    src = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dst = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    best = 0.0
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        best = max(best, nbytes / (time.perf_counter() - t) / 1e9)
    del src, dst
    return best


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------- workloads
def make_workload(name: str, seed: int = 0):
    from paper_1904_01201_b300 import workloads as wl
    if name == "house":
        sc = wl.make_house(seed, 1_000_000, 4096)
        poses = wl.random_poses(sc, 64, seed)
        return dict(name="house-1M-atlas4096-64x256", scenes=[sc], soa=np.zeros(64, np.uint32), poses=poses,
                    W=256, H=256, ids=False, intr=wl.pinhole_90(256, 256))
    if name == "room":
        sc = wl.make_room(seed)
        poses = wl.random_poses(sc, 16, seed)
        return dict(name="room-10k-vcolor-16x128", scenes=[sc], soa=np.zeros(16, np.uint32), poses=poses,
                    W=128, H=128, ids=False, intr=wl.pinhole_90(128, 128))
    if name == "batching":
        scenes = wl.batching_scenes(seed)
        split = wl.dirichlet_split(1024, len(scenes), 0.5, seed)
        soa = np.repeat(np.arange(len(scenes)), split).astype(np.uint32)
        poses = np.concatenate([wl.random_poses(s, int(k), seed + i) for i, (s, k) in enumerate(zip(scenes, split))])
        return dict(name="batching-8scenes-1024x128", scenes=scenes, soa=soa, poses=poses, W=128, H=128, ids=False,
                    intr=wl.pinhole_90(128, 128))
    if name == "large":
        sc = wl.make_house(seed + 5, 2_000_000, 8192, semantic=True)
        poses = wl.random_poses(sc, 256, seed)
        return dict(name="large-2M-atlas8192-256x512-ids", scenes=[sc], soa=np.zeros(256, np.uint32), poses=poses,
                    W=512, H=512, ids=True, intr=wl.pinhole_90(512, 512))
    raise ValueError(name)


def algorithmic_bytes_per_view(scene, W, H, ids) -> float:
    """Per-view algorithmic bytes: the whole mesh is read once per view
    (indices 12 B/triangle; xyz + uv 20 B/vertex, or xyz + rgb8 15 B), the
    framebuffer written once (3 B RGB + 4 B depth (+4 B id) per pixel), and
    one bilinear quad of RGBA8 texels (16 B) per pixel when textured."""
    T, V = scene.n_tris, scene.n_verts
    textured = scene.uv is not None and scene.atlas is not None
    b = 12.0 * T + (20.0 if textured else 15.0) * V + 7.0 * W * H
    if ids:
        b += 4.0 * W * H
    if textured:
        b += 16.0 * W * H
    return b


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def load_peaks_field(key: str):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            v = json.load(f).get(key)
        return None if v is None else float(v)
    return None


def raster_bytes_per_view(scene) -> float:
    """Algorithmic bytes of the raster stage per view: the mesh read once
    (a 12-byte index triple per triangle, 12 bytes of xyz per vertex)."""
    return 12.0 * scene.n_tris + 12.0 * scene.n_verts


def recorded_profile(workload_name: str, key: str):
    """A per-launch figure (dram_bytes_per_launch, warp_instructions_per_launch)
    of the raster stage from a committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"raster_kernel_{workload_name}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != kernel_source_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def recorded_traffic(workload_name: str):
    return recorded_profile(workload_name, "dram_bytes_per_launch")


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's timed-region length (every rank calls it; a single
    rank gets its own)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(frames_per_rank: int, world: int, ms_max: float) -> float:
    """Frames/s of the whole job: every rank's frames over the slowest rank's time."""
    return frames_per_rank * world / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo), or the platform's."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def cpu_chunks(wk, size: int):
    """The view sequence the CPU legs render: the workload's views in order,
    cycling, in chunks of up to `size` consecutive views of one scene (one
    oracle call each)."""
    soa = wk["soa"]
    i = 0
    while True:
        s = int(soa[i])
        sel = [j for j in range(i, min(i + size, len(soa))) if soa[j] == s]
        yield s, sel
        i = (sel[-1] + 1) % len(soa)


def cpu_baseline(wk, n_frames: int, min_seconds: float = 10.0, seconds_cap: float = 30.0,
                 single_seconds: float = 3.0):
    """The oracle, as it stands, on a bounded sample of the workload's views
    (the sequence of cpu_chunks, as the reference arm renders it): at least
    n_frames views and min_seconds of CPU work on every host core, at most
    seconds_cap; then one view at a time on one thread for single_seconds."""
    import oracle
    cores = os.cpu_count() or 1
    poses = wk["poses"]
    done, t0 = 0, time.perf_counter()
    for s, sel in cpu_chunks(wk, cores):
        oracle.render(wk["scenes"][s], poses[sel], wk["intr"], wk["W"], wk["H"], nthreads=cores, ids=wk["ids"])
        done += len(sel)
        el = time.perf_counter() - t0
        if el >= seconds_cap or (done >= n_frames and el >= min_seconds):
            break
    dt = time.perf_counter() - t0
    one, t1 = 0, time.perf_counter()
    for s, sel in cpu_chunks(wk, 1):
        oracle.render(wk["scenes"][s], poses[sel], wk["intr"], wk["W"], wk["H"], nthreads=1, ids=wk["ids"])
        one += 1
        if time.perf_counter() - t1 >= single_seconds:
            break
    dt1 = time.perf_counter() - t1
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{done} of the workload's views, in order from the first, rendered by the CPU oracle on "
                      f"{cores} threads in {dt:.1f} s",
            "single_thread": {"value": one / dt1, "unit": UNIT, "threads": 1,
                              "sample": f"{one} views, in order from the first, on one thread in {dt1:.1f} s"}}


# ----------------------------------------------------------------- arms
def run_reference(args, wk):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.render(wk["scenes"][int(wk["soa"][0])], wk["poses"][:1], wk["intr"], wk["W"], wk["H"], nthreads=1,
                      ids=wk["ids"])
    # each step: the next chunk of the view sequence cpu_baseline renders
    chunks = cpu_chunks(wk, cores)
    t0 = time.perf_counter()
    frames = 0
    for k in range(args.steps):
        s, sel = next(chunks)
        oracle.render(wk["scenes"][s], wk["poses"][sel], wk["intr"], wk["W"], wk["H"], nthreads=cores, ids=wk["ids"])
        frames += len(sel)
    dt = time.perf_counter() - t0
    v = frames / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/int", "data": "synthetic",
            "config": {"workload": wk["name"], "sample_views_per_step": int(cores), "mode": "cpu-oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"{frames} of the workload's views, in order from the first (up to {cores} "
                                       f"per step, as cpu_baseline renders them), on {cores} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_other(args):
    """The reference arm of the serving workload: the oracle's rate over the
    request mix (cpu_serving). The transfer and semantic workloads time GPU
    copy paths and a GPU sensor pair that have no CPU counterpart."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    if args.workload != "serving":
        return {"impl": "reference", "unavailable": f"the {args.workload} workload times GPU-side paths with no "
                                                    "CPU counterpart; the oracle arm covers house, room, batching, "
                                                    "large and serving"}
    from paper_1904_01201_b300 import workloads as wl
    cpu = cpu_serving(wl.batching_scenes(args.seed), args)
    return {"impl": "reference", "metric": "served RGB-D frames/sec with p50/p99 request latency",
            "value": cpu["value"], "unit": UNIT, "n_gpus": world, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/int", "data": "synthetic",
            "config": {"workload": "serving-8scenes-1024agents-mix64-512", "mode": "cpu-oracle"},
            "cpu_baseline": cpu, "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}


def run_gpu(args, wk):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")
    from paper_1904_01201_b300 import hsr

    handles = [hsr.SceneHandle(s) for s in wk["scenes"]]
    n, W, H = len(wk["soa"]), wk["W"], wk["H"]
    out = hsr.alloc_outputs(n, W, H, ids=wk["ids"], device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    poses, soa = wk["poses"], wk["soa"]
    multi = len(handles) > 1

    def step_oneshot():
        if multi:
            st = hsr.hsr_render_batch([h.handle for h in handles], soa, poses, wk["intr"], W, H, out["rgb"],
                                      out["depth"], out.get("ids"), stream)
        else:
            st = hsr.hsr_render(handles[0].handle, poses, wk["intr"], W, H, out["rgb"], out["depth"],
                                out.get("ids"), stream)
        if st != 0:
            raise hsr.HsrError(st, "render")
        return 1

    graph = None

    def step_batched():
        # one replay of the graph-captured persistent batch
        st = hsr.hsr_batch_render(graph, soa if multi else None, poses, None, stream)
        if st != 0:
            raise hsr.HsrError(st, "hsr_batch_render")
        return 1

    intr_c = hsr.as_intrinsics(wk["intr"])      # converted once, as a caller looping over agents would
    # each agent's C-ABI arguments (scene, pose, output addresses) prepared
    # once, as a caller looping over its agents would hold them, so that the
    # loop times the library's calls rather than the binding's conversions
    import ctypes
    lib = hsr.library()
    poses_c = np.ascontiguousarray(poses, dtype=np.float32)
    px = W * H
    sptr = ctypes.c_void_p(stream.cuda_stream)
    plain_args = []
    for i in range(n):
        ids_p = None if out.get("ids") is None else ctypes.c_void_p(out["ids"].data_ptr() + 4 * px * i)
        plain_args.append((ctypes.c_void_p(handles[int(soa[i])].handle),
                           ctypes.c_void_p(poses_c.ctypes.data + 28 * i), 1, ctypes.byref(intr_c), W, H,
                           ctypes.c_void_p(out["rgb"].data_ptr() + 3 * px * i),
                           ctypes.c_void_p(out["depth"].data_ptr() + 4 * px * i), ids_p, sptr))
    render_c = lib.hsr_render

    def step_plain():
        for a in plain_args:
            st = render_c(*a)
            if st != 0:
                raise hsr.HsrError(st, "render")
        return n

    step = step_plain if args.mode == "plain" else step_batched

    # autotuned launch configuration for this workload (untimed; cached per GPU)
    tuned = None
    if not args.no_tune:
        from paper_1904_01201_b300 import tuning
        cfg, source = tuning.ensure_tuned(wk["scenes"], handles, soa, poses, wk["intr"], W, H, out, stream,
                                          use_cache=not args.retune)
        tuned = dict(cfg, source=source)
    launch_phases = tuned["n_phases"] if tuned else hsr.hsr_config_default().n_phases
    graph = hsr.hsr_batch_create([h.handle for h in handles], n, wk["intr"], W, H, out["rgb"], out["depth"],
                                 out.get("ids"))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(stepfn, steps, sampler=None):
        for _ in range(args.warmup):
            stepfn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches = 0
        clk = ClockSampler(sampler) if sampler is not False else None
        for s, e in evs:
            flush.zero_()
            s.record(stream)
            launches += stepfn()
            e.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop() if clk else None
        barrier()
        ms = sum(s.elapsed_time(e) for s, e in evs)
        return ms, launches, clocks

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None

    ms, launches, clocks = timed(step, args.steps, uuid)
    local_ms = ms
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_value(n * args.steps, world, ms)

    # per-stage device times (CUDA events recorded by the library around each
    # kernel on this stream), over separate steps after the timed region
    hsr.hsr_set_stage_timing(True)
    stage_steps = max(3, min(args.steps, 20))
    acc = {"cull": 0.0, "raster": 0.0, "shade": 0.0, "total": 0.0}
    for _ in range(stage_steps):
        flush.zero_()
        step_oneshot() if args.mode == "batched" else step_plain()   # same kernels as the graph replay
        t = hsr.hsr_get_stage_timing()
        for k in acc:
            acc[k] += t[k]
    hsr.hsr_set_stage_timing(False)
    stages = {k: v / stage_steps for k, v in acc.items()}

    # one-shot calls (per-call scratch allocation, no graph) on the same views
    oneshot = None
    if args.mode == "batched":
        osteps = max(3, args.steps // 5)
        oms, _, _ = timed(step_oneshot, osteps, False)
        oneshot = {"value": n * osteps / (oms / 1e3), "ms_per_step": oms / osteps}

    # plain one-agent-per-launch path on the same views, for comparison: its
    # rate (CUDA events around each step of n calls), the host's time to
    # issue one call, and one call's device time (stage timing: first kernel
    # start to last kernel end). The host time is wall clock over bursts of
    # at most as many calls as the library has page-locked staging slots,
    # each burst started on an idle device, so that no call waits for a slot
    # (a longer unsynchronised run would time the device instead).
    plain = None
    if args.mode == "batched" and not args.no_plain:
        psteps = max(3, args.steps // 10)
        pms, _, _ = timed(step_plain, psteps, False)
        burst = 4
        host_s, host_calls = 0.0, 0
        for k in range(0, min(n, 256), burst):
            torch.cuda.synchronize()
            th = time.perf_counter()
            for a in plain_args[k:k + burst]:
                st = render_c(*a)
                if st != 0:
                    raise hsr.HsrError(st, "render")
            host_s += time.perf_counter() - th
            host_calls += len(plain_args[k:k + burst])
        host_ms = host_s * 1e3 / host_calls
        torch.cuda.synchronize()
        hsr.hsr_set_stage_timing(True)
        dev_ms = []
        for a in plain_args[:64]:
            st = render_c(*a)
            if st != 0:
                raise hsr.HsrError(st, "render")
            dev_ms.append(hsr.hsr_get_stage_timing()["total"])
        hsr.hsr_set_stage_timing(False)
        plain = {"value": n * psteps / (pms / 1e3), "ms_per_step": pms / psteps, "launches_per_step": n,
                 "host_ms_per_call": host_ms, "device_ms_per_call": statistics.mean(dev_ms),
                 "device_bound_value": 1e3 / statistics.mean(dev_ms)}

    # end to end through the C-ABI with host buffers: every step renders from
    # host poses (the view descriptors go up inside the call) and copies its
    # outputs to page-locked host memory (hsr_batch_render_host); two batches
    # on two streams alternate so that one step's copies overlap the next
    # step's render, and a step's host buffers are waited for before reuse
    def host_like(o):
        return {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in o.items() if v is not None}

    e2e_steps = max(20, args.steps // 4)      # enough steps for the two pipes to reach steady state
    if args.mode == "batched":
        out2 = hsr.alloc_outputs(n, W, H, ids=wk["ids"], device=dev)
        graph2 = hsr.hsr_batch_create([h.handle for h in handles], n, wk["intr"], W, H, out2["rgb"],
                                      out2["depth"], out2.get("ids"))
        pipes = [(graph, torch.cuda.Stream(dev), host_like(out)), (graph2, torch.cuda.Stream(dev), host_like(out2))]
        h2d_step = [0]

        def e2e_step(i):
            b, s, hb = pipes[i % 2]
            s.synchronize()                      # this pipe's previous frames are in host memory
            st, h2d_step[0] = hsr.hsr_batch_render_host(b, soa if multi else None, poses, W, H, hb["rgb"],
                                                        hb["depth"], hb.get("ids"), s)
            if st != 0:
                raise hsr.HsrError(st, "hsr_batch_render_host")

        for i in range(args.warmup):
            e2e_step(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            e2e_step(i)
        for _, s, _ in pipes:
            s.synchronize()
        e2e_dt = time.perf_counter() - t0
        hsr.hsr_batch_destroy(graph2)
        h2d_bytes = h2d_step[0]
        d2h_bytes = sum(v.numel() * v.element_size() for v in pipes[0][2].values())
    else:
        hb = host_like(out)
        for _ in range(args.warmup):
            step()
            for k, v in hb.items():
                v.copy_(out[k], non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            step()
            for k, v in hb.items():
                v.copy_(out[k], non_blocking=True)
            torch.cuda.current_stream().synchronize()
        e2e_dt = time.perf_counter() - t0
        h2d_bytes = int(poses.nbytes)
        d2h_bytes = sum(v.numel() * v.element_size() for v in hb.values())
    e2e = {"value": n * e2e_steps / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d_bytes),
           "d2h_bytes_per_step": int(d2h_bytes)}
    # the device->host link these frames cross, measured the same way (one
    # 256 MiB copy to page-locked memory, best of three, untimed): the e2e
    # frame traffic against it
    link = d2h_link_gbs(dev)
    e2e["d2h_gbs"] = e2e["value"] * d2h_bytes / n / 1e9
    e2e["link_gbs"] = link
    e2e["link_frac"] = e2e["d2h_gbs"] / link if link else None

    if rank != 0:
        return None
    peak, peak_kind = load_peaks()
    bview = sum(algorithmic_bytes_per_view(wk["scenes"][int(s)], W, H, wk["ids"]) for s in soa) / n
    views_per_launch = n * args.steps / launches
    kernel_ms_per_launch = local_ms / launches
    path_achieved = bview * views_per_launch / (kernel_ms_per_launch / 1e3) / 1e9
    # dominant kernel: the raster stage (one launch per render call; in plain
    # mode the stage timing covers the last single-view call)
    rview = sum(raster_bytes_per_view(wk["scenes"][int(s)]) for s in soa) / n
    raster_views = n if args.mode == "batched" else 1
    raster_achieved = rview * raster_views / (stages["raster"] / 1e3) / 1e9
    traffic = recorded_traffic(wk["name"]) if args.mode == "batched" else None
    # the same stage against the instruction-issue roofline: its kernels' warp
    # instructions per call (ncu, committed summary) over its live time,
    # against one warp instruction per clock on each SM sub-partition
    winst = recorded_profile(wk["name"], "warp_instructions_per_launch") if args.mode == "batched" else None
    issue = None
    if winst:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_mhz") or load_peaks_field("sm_max_mhz") or 2032.0
        ipeak = sms * 4 * mhz * 1e6 / 1e9
        iach = winst / (stages["raster"] / 1e3) / 1e9
        issue = {"bound": "alu", "achieved": iach, "peak": ipeak, "unit": "G warp instructions/s", "frac": iach / ipeak,
                 "warp_instructions_per_launch": winst, "sms": sms, "sm_mhz": mhz,
                 "what": "raster stage (all its kernels, one render call) over its live time"}
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/int", "data": "synthetic",
        "config": {"workload": wk["name"], "scenes": len(handles), "tris": [int(s.n_tris) for s in wk["scenes"]],
                   "agents": n, "width": W, "height": H, "outputs": "rgb+depth" + ("+ids" if wk["ids"] else ""),
                   "mode": args.mode, "l2": "flushed before every step (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}", "launch_config": tuned or "default"},
        "roofline": {"bound": "hbm", "achieved": raster_achieved, "peak": peak, "unit": "GB/s",
                     "frac": raster_achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "raster stage (raster_kernel and big_raster_kernel per phase, tile z, pyramid, "
                               "occlusion)", "kernel_ms_per_launch": stages["raster"],
                     "algorithmic_bytes_per_view": rview, "views_per_launch": raster_views,
                     "dram_gbs": None if traffic is None else traffic / (stages["raster"] / 1e3) / 1e9,
                     "dram_frac": None if traffic is None else traffic / (stages["raster"] / 1e3) / 1e9 / peak},
        "roofline_issue": issue,
        "roofline_path": {"bound": "hbm", "achieved": path_achieved, "peak": peak, "unit": "GB/s",
                          "frac": path_achieved / peak, "peak_kind": peak_kind,
                          "what": "whole render call (cull + raster + shade) per step",
                          "algorithmic_bytes_per_view": bview, "views_per_launch": views_per_launch,
                          "ms_per_launch": kernel_ms_per_launch},
        "stages_ms": stages,
        "e2e": e2e,
        "gpu_launches": kernels_per_call(launch_phases) * launches,
        "render_calls": launches,
        "clocks": clocks,
        "kernel_sha": kernel_source_hash(),
    }
    if oneshot:
        res["oneshot"] = oneshot
    if plain:
        res["plain"] = plain
        res["batched_over_plain"] = value / plain["value"]
    if world == 1 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(wk, args.cpu_frames, min_seconds=args.cpu_seconds,
                                           seconds_cap=3 * args.cpu_seconds,
                                           single_seconds=max(2.0, args.cpu_seconds / 3))
    return res


def run_subrecords(args):
    """The rest of the metric in the default run, each with its own clocks:
    the 10k-triangle room at 128^2, the 128^2 batching workload (8 scenes,
    1,024 agents), the 2M-triangle 512^2 workload with ids (each batched vs
    plain, with the oracle's rate on a shorter sample of the same views),
    serving at 10k and 50k requests/s (p50 / p99 latency; the oracle's rate
    over the request mix), the frame-transfer strategies (the whole table
    and resolution sweep, on shorter measurement windows), the semantic
    sensor from the separate 3M-triangle mesh, and agents stepped on the
    device with and without depth noise."""
    import copy
    out = {}
    for name in ("room", "batching", "large"):
        a = copy.copy(args)
        a.workload, a.cpu_seconds = name, min(args.cpu_seconds, 5.0)
        r = run_gpu(a, make_workload(name, args.seed))
        if r is not None:
            out[name] = r
    a = copy.copy(args)
    a.rates, a.cpu_seconds = "10000,50000", min(args.cpu_seconds, 5.0)
    out["serving"] = run_serving(a)
    out["transfer"] = run_transfer(args, quick=True)
    out["semantic"] = run_semantic(args)
    out["steps"] = run_steps(args)
    return out


def run_serving(args):
    """Serving configuration: the batching scenes resident, requests from 1024
    random-walking agents at resolutions 64/128/256/512 (weights
    0.2/0.4/0.3/0.1), Poisson arrivals swept over rates; frames/s and
    p50/p99 latency per rate."""
    import torch
    from paper_1904_01201_b300 import hsr, serve
    from paper_1904_01201_b300 import workloads as wl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    scenes = wl.batching_scenes(args.seed)
    handles = [hsr.SceneHandle(s) for s in scenes]
    srv = serve.Server(handles, res=(64, 128, 256, 512), weights=(0.2, 0.4, 0.3, 0.1), fb_bytes=4 << 30,
                       max_batch=args.serve_batch, n_streams=args.serve_streams, max_wait_us=args.serve_wait_us)
    actions = args.serve_requests == "action"
    agents = None
    if actions:
        agents, _ = serve.make_agents(scenes, handles, 1024, seed=args.seed)
        srv.attach_agents(agents)
    rates = [float(r) for r in args.rates.split(",")]
    rows = []
    clk = ClockSampler()
    batches0 = 0
    for k, rate in enumerate(rates):
        n = int(max(4000, min(22000, rate * 4)))
        if actions:
            req = serve.make_action_requests(n, 1024, seed=args.seed + k)
        else:
            req = serve.make_requests(scenes, n, seed=args.seed + k)
        row = serve.run_load(srv, req, rate, warmup=min(2000, n // 10), seed=args.seed + k)
        row["batches"] = row["stats"]["batches"] - batches0
        batches0 = row["stats"]["batches"]
        rows.append(row)
    clocks = clk.stop()
    srv.close()
    if agents is not None:
        agents.close()
    best = max(rows, key=lambda r: r["frames_per_s"])
    cpu = cpu_serving(scenes, args) if world == 1 and rank == 0 and not args.no_cpu else None
    return {"metric": "served RGB-D frames/sec with p50/p99 request latency", "value": best["frames_per_s"],
            "unit": UNIT, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/int", "data": "synthetic",
            "config": {"workload": "serving-8scenes-1024agents-mix64-512", "tris": [int(s.n_tris) for s in scenes],
                       "requests": args.serve_requests, "max_batch": args.serve_batch,
                       "streams": args.serve_streams, "max_wait_us": args.serve_wait_us, "fb_bytes": 4 << 30},
            "per_rate": [{k: v for k, v in r.items() if k != "stats"} for r in rows],
            "clocks": clocks, **({"cpu_baseline": cpu} if cpu else {})}


def cpu_serving(scenes, args):
    """The oracle's rate over the serving request mix: requests of random-
    walking agents (resolutions 64/128/256/512 at weights 0.2/0.4/0.3/0.1)
    in arrival order, taken in windows of `window` requests whose requests of
    one scene and resolution are rendered by one oracle call, on every host
    core for at least cpu_seconds (at most three times that); then one
    request at a time on one thread."""
    import oracle
    from paper_1904_01201_b300 import serve
    from paper_1904_01201_b300 import workloads as wl
    cores = os.cpu_count() or 1
    req = serve.make_requests(scenes, 4000, seed=args.seed)

    def chunks(window):
        for i in range(0, len(req), window):
            w = req[i:i + window]
            for key in sorted({(int(q["scene"]), int(q["res"])) for q in w}):
                sel = (w["scene"] == key[0]) & (w["res"] == key[1])
                yield key[0], key[1], w["pose"][sel]

    def run(window, nthreads, seconds):
        done, t0 = 0, time.perf_counter()
        for s, r, poses in chunks(window):
            oracle.render(scenes[s], poses, wl.pinhole_90(r, r), r, r, nthreads=nthreads, ids=False)
            done += len(poses)
            if time.perf_counter() - t0 >= seconds:
                break
        return done, time.perf_counter() - t0

    window = 8 * cores
    done, dt = run(window, cores, args.cpu_seconds)
    one, dt1 = run(1, 1, max(2.0, args.cpu_seconds / 3))
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{done} requests of the serving mix from its first windows of {window} (arrival order), "
                      f"by the CPU oracle on {cores} threads in {dt:.1f} s (throughput; no arrival process)",
            "single_thread": {"value": one / dt1, "unit": UNIT, "threads": 1,
                              "sample": f"the first {one} requests on one thread in {dt1:.1f} s"}}


def run_semantic(args):
    """Semantic sensor from a separate, denser mesh (Table 2, third row and
    footnote): 64 agents at 128x128 in a 1M-triangle textured house, colour +
    depth from it, semantic ids from the same layout tessellated to 3M
    triangles; frames/s of RGB-D alone and of RGB-D + semantics, both as one
    graph-replayed batch per step (CUDA events, L2 flushed between steps)."""
    import torch
    from paper_1904_01201_b300 import hsr
    from paper_1904_01201_b300 import workloads as wl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    col = wl.make_house(args.seed, 1_000_000, 4096)
    sem = wl.make_semantic_mesh(args.seed, 3_000_000)
    hs = [hsr.SceneHandle(col), hsr.SceneHandle(sem)]
    n, W = 64, 128
    intr = wl.pinhole_90(W, W)
    poses = wl.random_poses(col, n, args.seed)
    f = np.arange(n, dtype=np.uint32)
    rgbd = hsr.make_views(poses, 0, f, hsr.HSR_OUT_RGB | hsr.HSR_OUT_DEPTH)
    both = np.concatenate([rgbd, hsr.make_views(poses, 1, f, hsr.HSR_OUT_IDS)])
    b = hsr.Batch(hs, 2 * n, intr, W, W)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(views):
        for _ in range(max(3, args.warmup)):
            assert hsr.hsr_batch_render_views(b.handle, views, stream=stream) == hsr.HSR_OK
        ts = []
        for _ in range(max(5, min(args.steps, 50))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            assert hsr.hsr_batch_render_views(b.handle, views, stream=stream) == hsr.HSR_OK
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return n / (statistics.median(ts) * 1e-3)

    clk = ClockSampler()
    fps_rgbd = timed(rgbd)
    fps_sem = timed(both)
    clocks = clk.stop()
    b.close()
    return {"metric": "RGB-D + semantic frames/sec (semantic ids from a separate denser mesh)", "value": fps_sem,
            "unit": UNIT, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/int", "data": "synthetic",
            "config": {"workload": "semantic-house-1M-atlas4096+sem-3M-64x128", "tris": int(col.n_tris),
                       "sem_tris": int(sem.n_tris), "agents": n, "res": W, "l2": "flushed between steps"},
            "rgbd_frames_per_s": fps_rgbd, "semantic_slowdown": fps_rgbd / fps_sem, "clocks": clocks}


def run_steps(args):
    """Agents stepped on the device (Sec. 4 action space: move forward 0.25 m,
    turn 10 degrees, no sliding) and rendered in one batched call per step:
    the 1M-triangle house at 256x256, 64 agents on its navigability grid taking
    uniform random actions, RGB-D; with and without the Appendix C depth noise
    (sigma 0.4 in inverse depth). Beside them the same batch rendering the
    agents' current poses from the host. Frames/s from the median of CUDA
    events around each call, L2 flushed before each."""
    import torch
    from paper_1904_01201_b300 import hsr
    from paper_1904_01201_b300 import workloads as wl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    sc = wl.make_house(args.seed, 1_000_000, 4096)
    nav = wl.navmap(sc, 0.05)
    n, W = 64, 256
    intr = wl.pinhole_90(W, W)
    h = hsr.SceneHandle(sc)
    ag = hsr.Agents([h], [nav], wl.navigable_poses(sc, nav, n, args.seed + 3))
    b = hsr.Batch([h], n, intr, W, W, ids=False)
    idx = np.arange(n, dtype=np.uint32)
    rng = np.random.default_rng(args.seed + 11)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(call):
        for i in range(max(3, args.warmup)):
            call(i)
        ts = []
        for i in range(max(5, min(args.steps, 50))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(i)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        return n / (ms * 1e-3), ms

    def step(sigma):
        def call(i):
            b.step(ag, idx, rng.integers(hsr.HSR_ACTION_MOVE_FORWARD, hsr.HSR_ACTION_TURN_RIGHT + 1, n).astype(np.uint8),
                   stream=stream, noise_sigma=sigma, noise_seed=7 + i)
        return call

    clk = ClockSampler()
    fps, ms = timed(step(None))
    fps_noise, ms_noise = timed(step(0.4))
    now = ag.poses(stream)
    fps_pose, ms_pose = timed(lambda i: b.render(now, stream=stream))
    clocks = clk.stop()
    b.close()
    ag.close()
    h.close()
    return {"metric": "RGB-D frames/sec of agents stepped on the device", "value": fps, "unit": UNIT,
            "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/int",
            "data": "synthetic",
            "config": {"workload": "steps-house-1M-atlas4096-64x256", "tris": int(sc.n_tris), "agents": n, "res": W,
                       "actions": "uniform move_forward / turn_left / turn_right", "l2": "flushed between steps",
                       "timing": "median of per-call CUDA events"},
            "ms_per_step": ms, "noisy_depth": {"sigma": 0.4, "value": fps_noise, "ms_per_step": ms_noise},
            "pose_render": {"value": fps_pose, "ms_per_step": ms_pose,
                            "what": "the same batch rendering the agents' current poses sent from the host"},
            "clocks": clocks}


def run_transfer(args, quick: bool = False):
    """Frame-transfer strategies (Table 2 and the resolution figure beside it):
    frames stay in device memory for a device consumer (GPU->GPU), are copied
    to pinned host memory (GPU->CPU), or copied to the host and back into a
    separate device buffer (GPU->CPU->GPU); for colour, colour + depth, and
    colour + depth + semantic ids; with 1, 3 or 5 concurrent renderers (CUDA
    streams, each with its own graph-captured batch) in place of the paper's
    simulator processes, each rendering 1 agent per launch (as a simulator
    process does) or 64. Copies are queued on each renderer's stream after
    its render; frames/s over all renderers, wall clock, synchronised on both
    sides. `quick` measures every cell over a shorter window (0.1 s instead
    of 0.25 s)."""
    import torch
    from paper_1904_01201_b300 import hsr
    from paper_1904_01201_b300 import workloads as wl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    sc = wl.make_house(args.seed, 1_000_000, 4096, semantic=True)
    h = hsr.SceneHandle(sc)
    sensors = {"rgb": (False, False), "rgbd": (True, False), "rgbds": (True, True)}
    pool = wl.random_poses(sc, 512, args.seed + 7)

    def measure(res, sensor, strategy, n_streams, per_launch):
        depth, ids = sensors[sensor]
        intr = wl.pinhole_90(res, res)
        streams = [torch.cuda.Stream() for _ in range(n_streams)]
        batches = [hsr.Batch([h], per_launch, intr, res, res, ids=ids, depth=depth) for _ in streams]
        host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in b.out.items() if v is not None}
                for b in batches]
        back = [{k: torch.empty_like(v) for k, v in b.out.items() if v is not None} for b in batches] \
            if strategy == "gpu-cpu-gpu" else None
        n_pose = len(pool) // per_launch

        def step(i):
            for j, (b, s) in enumerate(zip(batches, streams)):
                k0 = ((i * n_streams + j) % n_pose) * per_launch
                b.render(pool[k0:k0 + per_launch], stream=s)
                if strategy == "gpu-gpu":
                    continue
                with torch.cuda.stream(s):
                    for key, dst in host[j].items():
                        dst.copy_(b.out[key], non_blocking=True)
                    if back is not None:
                        for key, dst in back[j].items():
                            dst.copy_(host[j][key], non_blocking=True)

        for i in range(3):
            step(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(3)
        torch.cuda.synchronize()
        steps = int(min(400, max(5, window / max(1e-6, time.perf_counter() - t0))))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            step(4 + i)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for b in batches:
            b.close()
        return n_streams * per_launch * steps / dt

    window = 0.1 if quick else 0.25
    clk = ClockSampler()
    table = []
    for per_launch in (1, 64):
        for sensor in ("rgb", "rgbd", "rgbds"):
            for strategy in ("gpu-cpu-gpu", "gpu-cpu", "gpu-gpu"):
                for n_streams in (1, 3, 5):
                    table.append({"res": 128, "sensors": sensor, "transfer": strategy, "renderers": n_streams,
                                  "agents_per_launch": per_launch,
                                  "frames_per_s": measure(128, sensor, strategy, n_streams, per_launch)})
    sweep = []
    for per_launch in (1, 64):
        for res in (64, 128, 256, 512):
            for strategy in ("gpu-cpu-gpu", "gpu-cpu", "gpu-gpu"):
                sweep.append({"res": res, "sensors": "rgbd", "transfer": strategy, "renderers": 1,
                              "agents_per_launch": per_launch,
                              "frames_per_s": measure(res, "rgbd", strategy, 1, per_launch)})
    clocks = clk.stop()
    head = [r for r in table if r["sensors"] == "rgbd" and r["transfer"] == "gpu-gpu" and r["renderers"] == 1
            and r["agents_per_launch"] == 64][0]
    return {"metric": "RGB-D frames/sec by frame-transfer strategy", "value": head["frames_per_s"], "unit": UNIT,
            "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/int",
            "data": "synthetic",
            "config": {"workload": "transfer-house-1M-atlas4096-sem", "tris": int(sc.n_tris),
                       "value_is": "gpu-gpu, rgbd, 128x128, 1 renderer, 64 agents per launch",
                       "window_s": window},
            "table": table, "resolution_sweep": sweep, "clocks": clocks}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hsr", choices=["hsr", "reference"])
    ap.add_argument("--workload", default="house",
                    choices=["house", "room", "batching", "large", "serving", "transfer", "semantic", "steps"])
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000,50000", help="serving: request rates (1/s)")
    ap.add_argument("--serve-batch", type=int, default=64)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-wait-us", type=int, default=50)
    ap.add_argument("--serve-requests", default="action", choices=["action", "pose"],
                    help="serving: requests carry an action of a device-resident agent, or a host pose")
    ap.add_argument("--mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="house: skip the room, batching, large, serving, transfer, semantic and steps sub-records of "
                         "the default run")
    ap.add_argument("--cpu-frames", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="least CPU time of the oracle's all-core sample (at most three times that)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--agents", type=int, default=0, help="render only the first N agents (profiling)")
    ap.add_argument("--no-tune", action="store_true", help="use the default launch configuration")
    ap.add_argument("--retune", action="store_true", help="ignore the tuning cache")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference" and args.workload in ("serving", "transfer", "semantic", "steps"):
        res = run_reference_other(args)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if args.workload in ("serving", "transfer", "semantic", "steps"):
        res = {"serving": run_serving, "transfer": run_transfer, "semantic": run_semantic,
               "steps": run_steps}[args.workload](args)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    wk = make_workload(args.workload, args.seed)
    if args.agents:
        k = min(args.agents, len(wk["soa"]))
        wk["soa"], wk["poses"] = wk["soa"][:k], wk["poses"][:k]
        wk["name"] += f"-first{k}"
    res = run_reference(args, wk) if args.impl == "reference" else run_gpu(args, wk)
    if res is not None and args.impl != "reference" and args.workload == "house" and not args.agents \
            and not args.no_sub and dist_env()[1] == 1:
        res["sub"] = run_subrecords(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
