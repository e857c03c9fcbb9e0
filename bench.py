"""Mapping-iteration throughput of the GB300 3DGS rasteriser.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

One step = one whole mapping iteration on one batch of synthetic input:
project -> bin/sort -> forward composite -> L1+SSIM loss -> backward ->
Adam, all in libgs_gb300.so.  Default workload: 1M Gaussians (SH degree 3)
in a seeded synthetic room, one 1200x680 view (the Replica-sized stand-in),
target rendered from a perturbed copy of the map.  Inputs are resident in HBM
for `value`; `e2e` adds, per step, the pinned-host -> device copy of the
step's target image and pose and the device -> host read of the loss.

The timed region replays one CUDA graph of the whole iteration per step, with
CUDA events around the K steps on the launching stream; the per-stage times
come from a separate pass that replays one graph per stage with events
between them.  The working set (map,
gradients, Adam moments: ~0.95 GB, plus the workspace) is far larger than the
129 MB L2, so no explicit flush is needed between steps.

With torchrun (N > 1) every rank runs an independent replica of the same
workload (the path shards over keyframes only through a gradient all-reduce,
which this single-GPU build does not implement: replicas only); `value` is
the sum of the ranks' iterations over the max-over-ranks time.
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

METRIC = ("mapping iters/s (fwd+bwd+Adam) @1M Gaussians 1200×680; batched vs per-view; "
          "%roofline")
WORKLOAD = "room1M_1200x680"
# Algorithmic FP32 operations per evaluated (pixel, Gaussian) pair, an FMA
# counting 2, independent of how a kernel is written: forward ~20 (offset 2,
# power as 6 FMA-equivalents, alpha 2, transmittance 2, colour 6, the exp on
# the SFU), adjoint ~60 (the forward's recomputation, the transmittance and
# colour-behind recursion, the alpha, power, mean, conic, opacity and colour
# terms, and the sum over the pixels).  The kernels as written execute a few
# more (the blend tests, the negations of the packed forms); the fractions
# use the algorithmic counts.
PAIR_FLOPS_FWD = 20.0
PAIR_FLOPS_BWD = 60.0

# DRAM bytes (read + write) of one k_render_bwd launch on the 1M 1200x680
# workload stored in Z-order, from one single-pass ncu capture per launch
# shape (tile, backward batch, backward pixels per thread) and tile-rect mode
# of the kernel as committed; other shapes and modes report null.  The
# capture's command and its other counters are kept with the launch-list
# profile of this workload.
RENDER_BWD_TRAFFIC = {
    ("room1M_1200x680", "8x8", 64, 2, "tight"): 54.52e6 + 0.02e6,
}


def iteration_roofline(n, sh_degree, n_views, n_values, n_pixels, instances, pairs, tiles,
                       passes, n_floats, ms, peaks):
    """Per-iteration roofline: the sum over the stages of max(algorithmic
    bytes / HBM peak, algorithmic FLOPs / FP32 peak), with the quantities the
    iteration itself produced (instances, counted pairs), against the
    measured iteration time."""
    K = (sh_degree + 1) ** 2
    pb = 4 * (11 + 3 * K)  # parameter bytes per Gaussian
    bw = peaks["hbm_gbs"] * 1e9
    fl = fp32_peak_tflops(peaks["sm_max_mhz"], peaks["sms"]) * 1e12
    vn = n_views * n
    stages = dict(
        project=((n_views + 3) // 4 * n * pb + vn * 72) / bw,
        bin_sort=(vn * (4 * 16 + 12) + instances * (8 + 16 * passes + 4) + tiles * 8) / bw,
        render_fwd=max(pairs * PAIR_FLOPS_FWD / fl, (instances * 48 + n_pixels * 20) / bw),
        loss_l1_ssim=n_values * 44 / bw,
        render_bwd=max(pairs * PAIR_FLOPS_BWD / fl, (instances * 48 + n_pixels * 16) / bw),
        project_bwd=(vn * (36 + 24 + 4) + 2 * n * pb) / bw,
        adam=n_floats * 28 / bw,
    )
    t = sum(stages.values()) * 1e3
    return dict(ms_roof=t, ms=ms, frac=t / ms,
                stages_ms_roof={k: v * 1e3 for k, v in stages.items()},
                basis="sum over stages of max(bytes / measured HBM copy, FLOPs / FP32 peak)")


def load_peaks(sms=None):
    """Measured HBM copy bandwidth and maximum SM clock, and the SM count of
    the device (sms: given, or read from the current CUDA device)."""
    sms = int(sms) if sms is not None else device_sms()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    sms=sms, source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, sms=sms, source="fallback")


def fp32_peak_tflops(sm_mhz, sms):
    # SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def device_sms():
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons around a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"], samples=0)

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = [num(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=reasons,
                    samples=len(rows), power_w_max=max(num(r[3]) for r in rows))


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x, ws):
    """Max of a float over the ranks of the default process group."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(local_ms, steps, ws):
    """Whole-job iterations/s of `ws` independent replicas, each timing `steps`
    iterations in `local_ms`: all ranks' iterations over the slowest rank's
    time.  Returns (value, max_ms)."""
    max_ms = reduce_max(local_ms, ws)
    return ws * steps / (max_ms / 1e3), max_ms


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------
# The CPU oracle (reference arm and cpu_baseline).
# ----------------------------------------------------------------------------
def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_iteration_seconds(p, view, target, lam, tile=(8, 8), threads=1):
    """Wall time of one whole FP64 oracle iteration (project, bin, render,
    loss, adjoint, Adam) of one view on `threads` host threads."""
    import oracle
    oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        L, g, _ = oracle.iteration(p, [view], [target], lam, tile[0], tile[1])
        flat_p = np.concatenate([np.asarray(p[k], np.float64).ravel()
                                 for k in oracle.PARAM_GROUPS])
        flat_g = np.concatenate([g[k].ravel() for k in oracle.PARAM_GROUPS])
        m, v = np.zeros_like(flat_p), np.zeros_like(flat_p)
        oracle.adam(flat_p, flat_g, m, v, 1e-3, 1)
        return time.perf_counter() - t0
    finally:
        oracle.set_threads(1)


WORKLOADS = {
    # name: (n Gaussians, seed offset, width, height, focal, sh degree)
    "room1M_1200x680": (1_000_000, 3, 1200, 680, 600.0, 3),
    "room200k_640x480": (200_000, 2, 640, 480, 525.0, 3),
}


def make_workload(name=WORKLOAD):
    from paper_2409_13055_gb300 import scenes
    n, so, w, h, f, deg = WORKLOADS[name]
    p = scenes.room_scene(n, seed=scenes.SEED_BASE + so, sh_degree=deg)
    view = scenes.camera(w, h, f, f)
    return p, view


def z_ordered(p):
    from paper_2409_13055_gb300 import scenes
    return scenes.z_ordered(p)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2409_13055_gb300 import scenes
    p, view = make_workload(args.workload)
    target = scenes.random_target(view, scenes.SEED_BASE + 13)
    cores = host_cores()
    times = []
    for _ in range(args.warmup if args.reference_warmup else 0):
        oracle_iteration_seconds(p, view, target, 0.2, threads=cores)
    for _ in range(args.steps):
        times.append(oracle_iteration_seconds(p, view, target, 0.2, threads=cores))
    t = float(np.mean(times))
    v = 1.0 / t
    out = dict(metric=METRIC, value=v, unit="iters/s", impl="reference", n_gpus=0,
               steps=args.steps, warmup=0, ms_per_step=1e3 * t, higher_is_better=True,
               scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
               config=dict(workload=args.workload, gaussians=int(p["means"].shape[0]),
                           width=view["width"], height=view["height"], sh_degree=3, views=1,
                           lam=0.2, tile="8x8"),
               cpu_baseline=dict(value=v, unit="iters/s", cores=cores, kind="oracle",
                                 sample="one full FP64 mapping iteration of the workload per step "
                                        "(target: seeded noise image), OpenMP on every host "
                                        "core of the process"),
               e2e=dict(value=v, unit="iters/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------
# The GPU arm.
# ----------------------------------------------------------------------------
def tile_passes(total_tiles):
    bits = max(1, math.ceil(math.log2(max(2, total_tiles))))
    return (bits + 7) // 8


def run_batched(args, ws):
    """The 16-keyframe form: one batched iteration over 6 x 640x480 RGB,
    6 x 752x480 gray and 4 x 1200x680 RGB views of a shared 500k SH-3 map,
    against the loop of 16 single-view iterations with one Adam step; each
    captured as one CUDA graph and timed with CUDA events."""
    import torch
    from paper_2409_13055_gb300 import mapping, scenes

    p = scenes.room_scene(500_000, seed=scenes.SEED_BASE + 4)
    if args.map_order == "zorder":
        p = z_ordered(p)
    views = scenes.views_mixed16()
    lam = 0.2
    cfg = dict(tile=(args.tile_w, args.tile_h), smem_batch=args.batch,
               pixels_per_thread=args.ppt, smem_batch_bwd=args.batch_bwd,
               pixels_per_thread_bwd=args.ppt_bwd)
    gt = mapping.GaussianMap(scenes.perturbed(p, scenes.SEED_BASE + 24))
    r = mapping.fit_instance_capacity(views, gt)
    r.forward(gt.gs_map())
    targets = [r.view_slice(r.images, v).cpu().numpy() for v in range(len(views))]
    del gt, r
    K = max(10, min(args.steps, 100))
    result = {}
    stream = torch.cuda.current_stream()
    for mode in ("batched", "recompute", "per_view"):
        gm = mapping.GaussianMap(p)
        if mode in ("batched", "recompute"):
            # recompute: the checkpointing plan, the projection and binning
            # of 4 views in the workspace, the 16 views in 4 passes
            rast = mapping.fit_instance_capacity(views, gm, headroom=1.5,
                                                 recompute=4 if mode == "recompute" else 0,
                                                 **cfg)
            it = mapping.MappingStep(gm, rast, rast.pack(targets), lam)
        else:
            it = mapping.PerViewLoop(gm, views, targets, lam, **cfg)
        it.capture(warmup=max(3, args.warmup))
        for _ in range(3):
            it()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        e0.record(stream)
        for _ in range(K):
            it()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), ws) / K
        result[mode] = dict(iters_per_s=ws * 1e3 / ms, ms_per_iter=ms)
        if mode != "per_view":
            result[mode]["workspace_bytes"] = int(rast.workspace_bytes)
        if mode == "batched":
            inst = int(rast.counters().n_instances)
            pairs = int(rast.last_idx.to(torch.int64).sum().item())
            px = sum(v["width"] * v["height"] for v in views)
            result[mode]["iteration_roofline"] = iteration_roofline(
                gm.n, gm.degree, len(views), rast.total_values, px, inst, pairs,
                rast.total_tiles, tile_passes(rast.total_tiles), gm.total, ms, load_peaks())
        del it, gm
        rast = None
        torch.cuda.empty_cache()
    result["speedup_batched_over_per_view"] = (result["batched"]["iters_per_s"] /
                                               result["per_view"]["iters_per_s"])
    result["config"] = dict(gaussians=500_000, views="6x640x480x3 + 6x752x480x1 + 4x1200x680x3",
                            steps=K, tile=f"{args.tile_w}x{args.tile_h}", smem_batch=args.batch,
                            pixels_per_thread=args.ppt, smem_batch_bwd=args.batch_bwd,
                            pixels_per_thread_bwd=args.ppt_bwd, cuda_graph="whole iteration")
    return result


def run_streaming(args, ws):
    """The streaming form: 752x480 grayscale keyframes on a 5 m drone loop,
    each inserting 20k Gaussians from its DSO-like point set (ray-cast
    textured room, inverse-depth noise 0.01), then 30 batched iterations over
    a sliding window of 8 keyframes with the checkpointed backward; the map
    grows to kfs x 20k Gaussians.  Keyframe images and points are drawn
    before the timed loop; insertion, re-planning and graph capture are
    inside it (host clock), the iterations alone are also timed with CUDA
    events."""
    import time

    import torch
    from paper_2409_13055_gb300 import mapping, scenes
    from paper_2409_13055_gb300.streaming import StreamingMapper

    kfs = list(scenes.streaming_keyframes(args.streaming_kfs, 20_000, device="cuda"))
    cfg = dict(tile=(args.tile_w, args.tile_h), smem_batch=args.batch,
               pixels_per_thread=args.ppt, smem_batch_bwd=args.batch_bwd,
               pixels_per_thread_bwd=args.ppt_bwd)
    mapper = StreamingMapper(window=8, iters=30, lam=0.2, recompute=4,
                             capacity=1 << 20, **cfg)
    stream = torch.cuda.current_stream()
    it_ms = 0.0
    last_kf_ms = 0.0
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for view, tgt, new in kfs:
        mapper.insert_keyframe(view, tgt, new)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mapper.iterate(mapper.iters)
        e1.record(stream)
        e1.synchronize()
        last_kf_ms = e0.elapsed_time(e1)
        it_ms += last_kf_ms
    torch.cuda.synchronize()
    wall = reduce_max(time.perf_counter() - t0, ws)
    it_ms = reduce_max(it_ms, ws)
    status = int(mapper.status().status)
    n_it = mapper.iterations
    # the window's workspace, and what a plan keeping every view's
    # projection (no recompute) would need for the same window and map, its
    # instance capacity covering all views
    final = mapper.steps[0].rast
    ws_keep = mapping.plan_workspace_bytes(
        final.views, final.n_capacity, final.instance_capacity * len(final.views),
        recompute=False, **cfg)
    return dict(iters_per_s=ws * n_it / (it_ms * 1e-3), keyframes_per_s=ws * len(kfs) / wall,
                iterations=n_it, keyframes=len(kfs), final_gaussians=int(mapper.gmap.n),
                ms_per_iter_final_map=last_kf_ms / mapper.iters, wall_s=wall,
                replans=mapper.replans, device_status=status,
                workspace_bytes=int(final.workspace_bytes),
                workspace_bytes_without_recompute=int(ws_keep),
                config=dict(views="752x480x1 window of 8", points_per_keyframe=20_000,
                            iterations_per_keyframe=30, recompute="4 views per pass",
                            cuda_graph="one per keyframe (first iteration eager)",
                            tile=f"{args.tile_w}x{args.tile_h}", smem_batch=args.batch,
                            pixels_per_thread=args.ppt, smem_batch_bwd=args.batch_bwd,
                            pixels_per_thread_bwd=args.ppt_bwd))


def run_autograd(args, ws, p, view, target, lam, K):
    """The headline iteration written as a PyTorch user would: the map's
    parameter groups as autograd leaves, images = GSRender.apply(...),
    loss = L1SSIMLoss.apply(...), loss.backward(), the gradients copied into
    the packed buffer and one Adam step; with the recompute rasteriser
    (forward keeps only final_T and last_idx, the backward repeats the
    projection and binning) and with the one that keeps the projection.
    Eager (no graph), CUDA events around K iterations."""
    import torch
    from paper_2409_13055_gb300 import mapping

    gm = mapping.GaussianMap(p)
    names = ("means", "log_scales", "quats", "opacity_logits", "sh")
    P, G = gm.params(), gm.grads()
    leaves = [P[k].detach().requires_grad_(True) for k in names]  # share gm's storage
    launch = dict(tile=(args.tile_w, args.tile_h), smem_batch=args.batch,
                  pixels_per_thread=args.ppt, smem_batch_bwd=args.batch_bwd,
                  pixels_per_thread_bwd=args.ppt_bwd)
    out = {}
    stream = torch.cuda.current_stream()
    for rec in (False, True):
        rast = mapping.fit_instance_capacity([view], gm, recompute=rec, **launch)
        tgt = target.reshape(-1)

        def iteration():
            for leaf in leaves:
                leaf.grad = None
            img = mapping.GSRender.apply(*leaves, rast)
            loss = mapping.L1SSIMLoss.apply(img, tgt, rast, lam)
            loss.backward()
            for k, leaf in zip(names, leaves):
                G[k].copy_(leaf.grad)
            gm.adam_step()

        for _ in range(max(args.warmup, 3)):
            iteration()
        torch.cuda.synchronize()
        barrier(ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            iteration()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), ws) / K
        assert rast.counters().status == 0
        out["recompute_on" if rec else "recompute_off"] = dict(
            iters_per_s=ws * 1e3 / ms, ms_per_iter=ms, workspace_bytes=int(rast.workspace_bytes))
        del rast
    out["config"] = dict(iterations=K, path="GSRender + L1SSIMLoss autograd Functions, "
                                             "loss.backward(), gradient copy, Adam; eager")
    return out


def run_density(args, ws, p, view, target):
    """Adaptive density control on the headline workload: K whole-iteration
    graph replays that also accumulate the AbsGS statistic (pixel adjoint
    with the homodirectional sums + gs_densify_stats), then one density
    control step (count, one host read of the new size, apply) timed on the
    host clock around a synchronised region."""
    import time

    import torch
    from paper_2409_13055_gb300 import mapping

    gm = mapping.GaussianMap(p)
    rast = mapping.fit_instance_capacity([view], gm, headroom=1.5, tile=(args.tile_w, args.tile_h),
                                         smem_batch=args.batch, pixels_per_thread=args.ppt,
                                         smem_batch_bwd=args.batch_bwd,
                                         pixels_per_thread_bwd=args.ppt_bwd, density_stats=True)
    accum = torch.zeros(gm.n, device="cuda")
    denom = torch.zeros(gm.n, device="cuda")
    step = mapping.MappingStep(gm, rast, target, 0.2, stats=(accum, denom))
    step.capture(warmup=max(3, args.warmup))
    K = max(10, min(args.steps, 100))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    it_ms = reduce_max(e0.elapsed_time(e1), ws) / K
    samples = torch.randn(gm.n, 2, 3, device="cuda",
                          generator=torch.Generator(device="cuda").manual_seed(2409_13055))
    n0 = gm.n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kept, cloned, split = gm.densify(accum, denom, samples, extent=1.0)
    torch.cuda.synchronize()
    dens_ms = (time.perf_counter() - t0) * 1e3
    return dict(iters_per_s_with_stats=ws * 1e3 / it_ms, ms_per_iter_with_stats=it_ms,
                densify_ms=dens_ms, gaussians_before=n0, gaussians_after=gm.n, kept=kept,
                cloned=cloned, split=split, pruned=n0 - kept - split,
                config=dict(statistic_iterations=K + max(3, args.warmup) + 1,
                            grad_threshold=0.0004, percent_dense=0.01, min_opacity=0.005,
                            extent=1.0, cuda_graph="whole iteration",
                            densify="count + one host read + apply, host clock"))


def run_pyramid(args, ws, p, view, target):
    """Gaussian-pyramid training (paper Sec. III-B) on the headline workload:
    the time to build a 3-level target pyramid, and the mapping iteration at
    each level (whole-iteration graph, CUDA events)."""
    import torch
    from paper_2409_13055_gb300 import mapping, pyramid

    stream = torch.cuda.current_stream()
    img = target.reshape(3, view["height"], view["width"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        pyramid.pyramid(img, 3)
    e0.record(stream)
    for _ in range(10):
        levels = pyramid.pyramid(img, 3)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1) / 10
    out = dict(pyramid_build_ms=build_ms, levels=[])
    K = max(10, min(args.steps, 100))
    for level in range(3):
        v = pyramid.level_view(view, level)
        gm = mapping.GaussianMap(p)
        rast = mapping.fit_instance_capacity([v], gm, headroom=1.5, tile=(args.tile_w, args.tile_h),
                                             smem_batch=args.batch, pixels_per_thread=args.ppt,
                                             smem_batch_bwd=args.batch_bwd,
                                             pixels_per_thread_bwd=args.ppt_bwd)
        step = mapping.MappingStep(gm, rast, levels[level].reshape(-1).contiguous(), 0.2)
        step.capture(warmup=max(3, args.warmup))
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), ws) / K
        out["levels"].append(dict(level=level, width=v["width"], height=v["height"],
                                  iters_per_s=ws * 1e3 / ms, ms_per_iter=ms))
        del step, rast, gm
        torch.cuda.empty_cache()
    return out


def run_pointcloud(args, ws):
    """Point-cloud densification of a keyframe (paper Sec. III-A) at the
    EuRoC-like 752x480: GPU selection, host Delaunay of the selected pixels,
    GPU mean-depth interpolation and the new Gaussians, on 10 ray-cast
    keyframes of the drone loop (host clock, synchronised; the ray cast is
    input generation and not timed)."""
    import time

    import torch
    from paper_2409_13055_gb300 import pointcloud, scenes

    views = scenes.drone_loop(10)
    faces, tex = scenes.room_textures()
    frames = [scenes.ray_cast(v, faces, tex, device="cuda") for v in views]
    rows = []
    for it, (v, (depth, gray)) in enumerate(zip(views, frames)):
        D = torch.tensor(depth, device="cuda")
        G = torch.tensor(gray, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        px, py, z = pointcloud.keyframe_points(G, lambda x, y: D[y, x])
        new = pointcloud.gaussians_from_points(v, px, py, z, G)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        n_sel = int(torch.count_nonzero(pointcloud.select_pixels(G)[1]).item())
        if it > 0:  # the first keyframe warms up
            rows.append((ms, n_sel, int(px.numel()) - n_sel, new["means"].shape[0]))
    a = np.array(rows, float)
    return dict(ms_per_keyframe=float(a[:, 0].mean()), selected_per_keyframe=float(a[:, 1].mean()),
                interpolated_per_keyframe=float(a[:, 2].mean()),
                config=dict(image="752x480x1", block=4, passes=3,
                            thresholds_sq=list(pointcloud.DEFAULT_THRESHOLDS_SQ), grid=4,
                            keyframes=len(rows), clock="host, synchronised"))


def run_gpu(args, ws, rank, local):
    import torch
    from paper_2409_13055_gb300 import binding as B
    from paper_2409_13055_gb300 import build as gsbuild
    from paper_2409_13055_gb300 import mapping, scenes

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gsbuild.build()
    peaks = load_peaks()

    p, view = make_workload(args.workload)
    if args.map_order == "zorder":
        p = z_ordered(p)
    lam = 0.2
    # target: render of a perturbed copy of the map (set-up, untimed)
    pert = scenes.perturbed(p, scenes.SEED_BASE + 23)
    gt_map = mapping.GaussianMap(pert)
    rast = mapping.fit_instance_capacity([view], gt_map)
    rast.forward(gt_map.gs_map())
    target = rast.images.clone()
    del gt_map
    gm = mapping.GaussianMap(p)
    tuned = None
    if None in (args.tile_w, args.tile_h, args.batch, args.ppt):
        from paper_2409_13055_gb300 import autotune
        tuned = autotune.autotune([view], gm, target, lam, use_cache=False,
                                  tight_rect=not args.square_rects)
        args.tile_w = args.tile_w or tuned["tile"][0]
        args.tile_h = args.tile_h or tuned["tile"][1]
        args.batch = args.batch or tuned["smem_batch"]
        args.ppt = args.ppt or tuned["pixels_per_thread"]
        args.batch_bwd = args.batch_bwd or tuned["smem_batch_bwd"]
        args.ppt_bwd = args.ppt_bwd or tuned["pixels_per_thread_bwd"]
    args.batch_bwd = args.batch_bwd or args.batch
    args.ppt_bwd = args.ppt_bwd or args.ppt
    rast = mapping.fit_instance_capacity([view], gm, headroom=1.5, tile=(args.tile_w, args.tile_h),
                                         smem_batch=args.batch, pixels_per_thread=args.ppt,
                                         smem_batch_bwd=args.batch_bwd,
                                         pixels_per_thread_bwd=args.ppt_bwd,
                                         deterministic=args.deterministic,
                                         tight_rect=not args.square_rects)
    step = mapping.MappingStep(gm, rast, target, lam, fused=args.adam == "fused",
                               sparse_adam=args.adam == "sparse")
    m, g = gm.gs_map(), gm.gs_map_grad()
    stages = [
        ("project", lambda: rast.project(m)),
        ("bin_sort", lambda: rast.bin_sort(gm.n)),
        ("render_fwd", lambda: rast.render_fwd()),
        ("loss_l1_ssim", lambda: rast.loss_l1_ssim(step.targets, lam)),
        ("render_bwd", lambda: rast.render_bwd_pixels()),
    ]
    if args.adam == "fused":
        stages.append(("project_bwd_adam", lambda: rast.project_bwd_adam(gm)))
    elif args.adam == "sparse":
        vis = torch.zeros(gm.n, dtype=torch.uint8, device="cuda")
        stages += [("project_bwd", lambda: rast.project_bwd(m, g)),
                   ("adam_sparse", lambda: (rast.visibility(gm.n, vis),
                                            gm.adam_step(visible=vis)))]
    else:
        # as MappingStep runs it: the gradient of groups of 32 Gaussians that
        # touch no tile is neither written nor read (same update)
        gvis = torch.zeros((gm.n + B.GS_GRAD_GROUP - 1) // B.GS_GRAD_GROUP, dtype=torch.uint8,
                           device="cuda")
        stages += [("project_bwd", lambda: rast.project_bwd_groups(m, g, gvis)),
                   ("adam", lambda: gm.adam_step(group_vis=gvis))]
    # warm-up (eager), then capture one graph per stage
    for _ in range(max(args.warmup, 3)):
        for _, f in stages:
            f()
    torch.cuda.synchronize()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    graphs = []
    with torch.cuda.stream(cs):
        for name, f in stages:
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=cs):
                f()
            graphs.append((name, gr))
    torch.cuda.current_stream().wait_stream(cs)
    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 3)):
        for _, gr in graphs:
            gr.replay()
    torch.cuda.synchronize()

    # algorithmic counts of this workload (one probe, untimed)
    c = rast.counters()
    instances = int(c.n_instances)
    pairs_bwd = int(rast.last_idx.to(torch.int64).sum().item())

    # one graph of the whole iteration: the stages back to back, as
    # MappingStep.capture records them
    whole = torch.cuda.CUDAGraph()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        with torch.cuda.graph(whole, stream=cs):
            for _, f in stages:
                f()
    torch.cuda.current_stream().wait_stream(cs)
    for _ in range(max(args.warmup, 3)):
        whole.replay()
    torch.cuda.synchronize()

    # --- timed region: K replays of the whole-iteration graph --------------
    K = args.steps
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(K):
        whole.replay()
    t1.record(stream)
    barrier(ws)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    value, total_ms = replica_throughput(total_ms, K, ws)
    ms_step = total_ms / K

    # --- stage breakdown (not the headline): the per-stage graphs with CUDA
    # events between them, a separate pass of up to 50 steps -------------
    KS = max(1, min(K, 50))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(graphs) + 1)]
          for _ in range(KS)]
    torch.cuda.synchronize()
    for k in range(KS):
        ev[k][0].record(stream)
        for j, (_, gr) in enumerate(graphs):
            gr.replay()
            ev[k][j + 1].record(stream)
    torch.cuda.synchronize()
    stage_ms = {name: float(np.mean([ev[k][j].elapsed_time(ev[k][j + 1]) for k in range(KS)]))
                for j, (name, _) in enumerate(graphs)}
    status = rast.counters()
    assert status.status == 0, f"device status {status.status}"

    # --- end to end through mapping.HostPipeline: per step, pinned H2D of the
    # target and the poses, the iteration, D2H of its loss (copies overlapped
    # with the previous / current iteration's compute) -
    host_tgt = target.cpu().pin_memory()
    host_views = rast.views_dev.cpu().pin_memory()
    pipe = mapping.HostPipeline(step)
    E = max(1, min(K, 50))
    for _ in range(3):
        pipe.submit(host_tgt, host_views)
    pipe.drain()
    barrier(ws)
    torch.cuda.synchronize()
    # host clock around the E submissions and the read of the last loss:
    # the copies, the host-side submission and the final D2H are all inside
    t_wall = time.perf_counter()
    for _ in range(E):
        pipe.submit(host_tgt, host_views)
    last_loss = pipe.drain()
    t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    e2e_ms = reduce_max(t_wall * 1e3, ws) / E
    h2d = host_tgt.numel() * 4 + host_views.numel()
    assert last_loss is not None and math.isfinite(last_loss)

    # --- roofline of the dominant kernel ----------------------------------
    n = gm.n
    K_sh = (gm.degree + 1) ** 2
    algo_bytes = dict(
        project=n * (4 * (11 + 3 * K_sh)) + n * 72,
        bin_sort=n * 4 * 16 + n * 12 + instances * 8 + tile_passes(rast.total_tiles) * instances * 16
        + instances * 4 + rast.total_tiles * 8,
        loss_l1_ssim=rast.total_values * 44,
        # parameters read (44 + 12K B), gradients written (same), screen-space
        # gradient 36 B, colour gradient 24 B, tiles touched 4 B
        project_bwd=n * 2 * (4 * (11 + 3 * K_sh)) + n * (36 + 24 + 4),
        adam=gm.total * 28,
        # every parameter read once with its two moments and written back
        # with them (24 B per float), plus the screen-space and colour
        # gradients, tiles touched and the deferred mean gradient
        project_bwd_adam=gm.total * 24 + n * (36 + 24 + 4 + 24),
    )
    dominant = max(stage_ms, key=stage_ms.get)
    if dominant in algo_bytes:
        achieved = algo_bytes[dominant] / (stage_ms[dominant] * 1e-3) / 1e9
        roof = dict(bound="hbm", kernel=dominant, achieved=achieved, peak=peaks["hbm_gbs"],
                    unit="GB/s", frac=achieved / peaks["hbm_gbs"],
                    traffic=None, algorithmic=algo_bytes[dominant],
                    peak_source=peaks["source"])
    else:
        per_pair = PAIR_FLOPS_BWD if dominant == "render_bwd" else PAIR_FLOPS_FWD
        flops = pairs_bwd * per_pair
        peak = fp32_peak_tflops(peaks["sm_max_mhz"], peaks["sms"])
        achieved = flops / (stage_ms[dominant] * 1e-3) / 1e12
        traffic = None
        if dominant == "render_bwd" and args.map_order == "zorder" and not args.deterministic:
            traffic = RENDER_BWD_TRAFFIC.get((args.workload, f"{args.tile_w}x{args.tile_h}",
                                              args.batch_bwd, args.ppt_bwd,
                                              "square" if args.square_rects else "tight"))
        roof = dict(bound="alu", kernel=dominant, achieved=achieved, peak=peak, unit="TFLOP/s",
                    frac=achieved / peak, traffic=traffic, algorithmic=flops,
                    flops_per_pair=per_pair, pairs=pairs_bwd,
                    peak_source="%d SMs (device) x 128 FP32 lanes x 2 x sm_max_mhz (%s)" % (
                        peaks["sms"], peaks["source"]))

    # project 1, bin_sort 18 + 3 per tile-id pass, render_fwd 1, loss 2,
    # render_bwd 1, then the projection adjoint (one kernel for one view) +
    # step counter + adam (+ the visibility kernel for sparse), or step
    # counter + the fused adjoint kernel
    launches_per_step = 1 + (18 + 3 * tile_passes(rast.total_tiles)) + 1 + 2 + 1 + \
        {"fused": 2, "separate": 3, "sparse": 4}[args.adam]

    out = dict(metric=METRIC, value=value, unit="iters/s", n_gpus=ws, steps=K, warmup=args.warmup,
               ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None,
               dtype="f32", data="synthetic",
               config=dict(workload=args.workload, gaussians=n, width=view["width"],
                           height=view["height"], sh_degree=3,
                           views=1, lam=0.2, tile=f"{args.tile_w}x{args.tile_h}",
                           smem_batch=args.batch, pixels_per_thread=args.ppt,
                           smem_batch_bwd=args.batch_bwd, pixels_per_thread_bwd=args.ppt_bwd,
                           autotuned=tuned is not None,
                           cuda_graph="one graph per iteration (stage times: a separate pass "
                                      "of one graph per stage)",
                           adam=args.adam, map_order=args.map_order,
                           deterministic=bool(args.deterministic),
                           tile_rects="square" if args.square_rects else "tight",
                           l2="working set ~1.2 GB > 129 MB L2, no flush",
                           instances=instances, pairs_bwd=pairs_bwd,
                           workspace_bytes=int(rast.workspace_bytes),
                           workspace_bytes_recompute=int(mapping.plan_workspace_bytes(
                               [view], gm.n, rast.instance_capacity, recompute=True,
                               tile=(args.tile_w, args.tile_h), smem_batch=args.batch,
                               pixels_per_thread=args.ppt, smem_batch_bwd=args.batch_bwd,
                               pixels_per_thread_bwd=args.ppt_bwd))),
               stages_ms=stage_ms, roofline=roof,
               iteration_roofline=iteration_roofline(
                   n, gm.degree, 1, rast.total_values, view["width"] * view["height"], instances,
                   pairs_bwd, rast.total_tiles, tile_passes(rast.total_tiles), gm.total, ms_step,
                   peaks),
               e2e=dict(value=1e3 / e2e_ms * ws, unit="iters/s", h2d_bytes_per_step=int(h2d),
                        d2h_bytes_per_step=4),
               clocks=clocks, gpu_launches=launches_per_step * K)

    if tuned is not None:
        out["autotune"] = [dict(t, ms=round(t["ms"], 4), fwd_ms=round(t["fwd_ms"], 4),
                                bwd_ms=round(t["bwd_ms"], 4)) for t in tuned["timings"]]
    if not args.no_batched:
        del rast, step, graphs
        gm = None
        torch.cuda.empty_cache()
        out["batched16"] = run_batched(args, ws)
    if args.streaming_kfs > 0:
        torch.cuda.empty_cache()
        out["streaming"] = run_streaming(args, ws)
    if not args.no_autograd:
        torch.cuda.empty_cache()
        out["autograd"] = run_autograd(args, ws, p, view, target, lam, max(1, min(K, 100)))
    if not args.no_density:
        torch.cuda.empty_cache()
        out["density_control"] = run_density(args, ws, p, view, target)
    if not args.no_pyramid:
        torch.cuda.empty_cache()
        out["pyramid"] = run_pyramid(args, ws, p, view, target)
    if not args.no_pointcloud:
        out["pointcloud"] = run_pointcloud(args, ws)

    if rank == 0 and not args.no_cpu_baseline:
        from paper_2409_13055_gb300 import scenes as sc
        tgt = sc.random_target(view, sc.SEED_BASE + 13)
        tile = (args.tile_w, args.tile_h)
        cores = host_cores()
        t_all = oracle_iteration_seconds(p, view, tgt, lam, tile, threads=cores)
        t_one = oracle_iteration_seconds(p, view, tgt, lam, tile, threads=1)
        out["cpu_baseline"] = dict(value=1.0 / t_all, unit="iters/s", cores=cores, kind="oracle",
                                   sample="one full FP64 mapping iteration of the workload "
                                          "(target: seeded noise image) at the GPU arm's tile "
                                          "shape, OpenMP on every host core of the process",
                                   one_core=dict(value=1.0 / t_one, unit="iters/s", cores=1))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="room1M_1200x680 is the headline; room200k_640x480 a smaller "
                         "case of the same shape for profiling")
    ap.add_argument("--tile-w", type=int, default=None, help="fix the tile width (else autotuned)")
    ap.add_argument("--tile-h", type=int, default=None)
    ap.add_argument("--batch", type=int, default=None, help="Gaussians per shared-memory batch")
    ap.add_argument("--ppt", type=int, default=None, help="pixels per thread")
    ap.add_argument("--batch-bwd", type=int, default=None, help="backward smem batch")
    ap.add_argument("--ppt-bwd", type=int, default=None, help="backward pixels per thread")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 16-keyframe batched vs per-view measurement")
    ap.add_argument("--adam", default="separate", choices=["fused", "separate", "sparse"],
                    help="Adam as its own pass over the gradient buffer (measured faster at "
                         "1M: 0.44 vs 0.56 ms), inside the projection adjoint, or the "
                         "visibility-masked variant (changes the optimiser: not the headline)")
    ap.add_argument("--square-rects", action="store_true",
                    help="plain 3-sigma square tile rects instead of the opacity-aware tight "
                         "ones (same images and gradients, more (Gaussian, tile) instances)")
    ap.add_argument("--deterministic", action="store_true",
                    help="bit-reproducible pixel adjoint (partial sums per (Gaussian, tile) "
                         "reduced in a fixed order instead of float atomics)")
    ap.add_argument("--map-order", default="zorder", choices=["zorder", "generated"],
                    help="storage order of the map's Gaussians (the same set either way)")
    ap.add_argument("--streaming-kfs", type=int, default=100,
                    help="keyframes of the streaming measurement (0 skips it)")
    ap.add_argument("--no-pointcloud", action="store_true",
                    help="skip the keyframe point-cloud densification measurement")
    ap.add_argument("--no-pyramid", action="store_true",
                    help="skip the Gaussian-pyramid level measurement")
    ap.add_argument("--no-density", action="store_true",
                    help="skip the adaptive density control measurement")
    ap.add_argument("--no-autograd", action="store_true",
                    help="skip the autograd-Function iterations (recompute on and off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-warmup", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        if args.steps > 10:
            args.steps = 10  # each oracle step is a full FP64 iteration (~1-2 s on 16 cores)
        run_reference(args, ws, rank)
        return
    run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    main()
