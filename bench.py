#!/usr/bin/env python
"""Benchmark of the MIRReS stage-2 hot path on one GB300 (or N independent replicas).

One step = one pass of the whole path over the workload: LBVH build (Morton codes, radix
sort, hierarchy, boxes) and env sampling tables, the forward render of every view, the L2
image loss against reference images and the adjoint (PRIMARY mode) into the gradients of
textures, env map and vertices. Metric: forward+backward path samples per second (one path
sample = one pixel sample of one view), for the batched launch (every view in one
graph-captured wavefront: the headline value), the plain per-view wavefront launch and the
single persistent kernel; Mrays/s alongside. The same step with the FULL-mode adjoint
(gradients through every vertex) is reported as `full_adjoint` when its tape fits, the step with
spatial reservoir reuse as `spatial_reuse`, and the denoiser as `denoiser`.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload config3|config5|config2]
  python bench.py --impl reference ...   (the CPU oracle on the host cores, bounded sample)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd path-samples/s (batched launch; plain per-view launch and Mrays/s alongside)"
# denoiser sigmas (colour, normal, position) of the EAWT arm, and the measured HBM copy rate
EAWT_SIGMAS = (0.5, 0.3, 0.2)
# spatial reuse arm: neighbours merged per pixel and the radius they are drawn from
REUSE = (4, 8)
# timed calls of the demodulated-lighting kernel for its roofline
DEMOD_REPS = 5


# DRAM bytes per unit of the three stage kernels (closest-hit ray, RIS candidate, shadow ray),
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the first render's
# launches on config 3 reduced to 2 views, divided by that render's unit counts; the 1-view
# capture gives per-unit figures within 2%, so traffic is taken to grow in proportion and is
# scaled to the bench's launches by their unit counts. Valid only for the kernel sources they
# were measured on (SHA-256 prefix of wave.cu, device.cuh, path.cuh, bvh.cu, env.cu); otherwise
# null.
TRAFFIC_SOURCES = ("wave.cu", "device.cuh", "path.cuh", "bvh.cu", "env.cu")
TRAFFIC_SHA = "618e3614140c8c45"
TRAFFIC_PER_UNIT = {"closest": 81.75, "shade": 12.09, "shadow": 125.11}


def _traffic_valid():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2406_16360_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16] == TRAFFIC_SHA


def _hbm_peak():
    try:
        return float(json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                 "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0  # fallback figure when the measured peaks are absent


HBM_PEAK = _hbm_peak()
UNIT = "path-samples/s"


def make_workload(name, views=None):
    from paper_2406_16360_gb300 import synth
    if name == "config3":
        return synth.config3() if views is None else synth.config3(n_views=views)
    if name == "config2":
        return synth.config2()
    if name == "config5":
        return synth.config5() if views is None else synth.config5(n_scenes=views)
    raise SystemExit(f"unknown workload {name}")


def workload_config(w, name):
    sc = w.scenes[0]
    v = w.views[0]
    cfg = {"workload": w.name, "views": len(w.views), "scenes": len(w.scenes),
           "triangles": int(sum(s.n_tris for s in w.scenes)), "ris_m": w.ris_m,
           "samples_per_step": int(w.samples)}
    if name != "config5":
        cfg.update({"resolution": f"{v.width}x{v.height}", "spp": v.spp, "bounces": v.bounces,
                    "texture": f"{sc.albedo.shape[1]}x{sc.albedo.shape[0]}",
                    "env": f"{sc.env.shape[1]}x{sc.env.shape[0]}"})
    return cfg


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------------------
def oracle_sample(w, target_seconds, threads):
    """fwd+bwd of the oracle on a bounded set of pixels of view 0 (all spp, all bounces)."""
    import numpy as np
    from oracle import oracle as O
    v = w.views[0]
    osc = O.OracleScene(w.scenes[v.scene])
    rng = np.random.Generator(np.random.PCG64(77))
    n_all = v.width * v.height

    def run(npix):
        pix = np.sort(rng.choice(n_all, size=npix, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        r = O.render(osc, v, 0, w.ris_m, seed=w.seed, pixels=pix, threads=threads, margins=False)
        g = O.backward(osc, v, 0, w.ris_m, np.ones((npix, 3)), seed=w.seed, pixels=pix, threads=threads,
                       want_abs=False)
        dt = time.perf_counter() - t0
        return dt, r["counts"], npix * v.spp

    probe = min(n_all, threads * 32)
    dt, _, _ = run(probe)
    per_px = dt / probe
    npix = int(min(n_all, max(threads * 4, target_seconds / max(per_px, 1e-9))))
    return osc, run, npix


def cpu_baseline(w, seconds=15.0):
    threads = os.cpu_count() or 1
    osc, run, npix = oracle_sample(w, seconds, threads)
    dt, counts, samples = run(npix)
    v = w.views[0]
    return {"value": samples / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"fwd+bwd of {npix} random pixels of view 0 ({v.width}x{v.height}, {v.spp} spp, "
                      f"{v.bounces} bounces, M={w.ris_m}), {samples} path samples in {dt:.1f} s"}, counts, samples


def run_reference(args):
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    w = make_workload(args.workload, args.views)
    threads = os.cpu_count() or 1
    osc, run, npix = oracle_sample(w, args.ref_seconds, threads)
    for _ in range(args.warmup):
        run(npix)
    tot_t, tot_s = 0.0, 0
    for _ in range(args.steps):
        dt, _, s = run(npix)
        tot_t += dt
        tot_s += s
    value = tot_s / tot_t
    v = w.views[0]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: fwd+bwd of {npix} random pixels of view 0 "
                                       f"({v.width}x{v.height}, {v.spp} spp)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _unique_edges(tris):
    """number of unique undirected edges of a triangle list (for the regulariser byte count)"""
    import numpy as np
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), axis=1)
    e = e[e[:, 0] != e[:, 1]]
    return int(np.unique(e[:, 0] << 32 | e[:, 1]).size)


def reduce_max(x, device):
    """max of a per-rank number over all ranks (the slowest replica sets the time)"""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([float(x)], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="config3", choices=["config3", "config5", "config2"])
    ap.add_argument("--views", type=int, default=None, help="override the view / scene count (smaller runs)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-launch arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-full", action="store_true", help="skip the FULL-mode adjoint arm")
    ap.add_argument("--no-eawt", action="store_true", help="skip the denoiser arm")
    ap.add_argument("--no-regularizers", action="store_true", help="skip the mesh regulariser arm")
    ap.add_argument("--no-reuse", action="store_true", help="skip the spatial-reuse arm")
    ap.add_argument("--bvh", default="lbvh", choices=["lbvh", "ploc"],
                    help="hierarchy builder run every step: Karras LBVH (the paper's) or PLOC clustering")
    ap.add_argument("--traversal", default="binary", choices=["binary", "wide"],
                    help="ray traversal through the binary tree (default) or the 8-wide BVH collapsed from it")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--bin", action="store_true",
                    help="batched launch: bin continuation rays by origin cell and direction octant")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mine":
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    BIN_FLAG = 8 if args.bin else 0
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_16360_gb300 import mirres as M
    from paper_2406_16360_gb300.renderer import GpuWorkload

    # the roofline denominators, measured on this device before the workload is set up: the FP32
    # FMA rate of the SMs (the stages' arithmetic) and the bandwidth of loads served by L2 (where
    # the traversal's node and triangle loads hit)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_clk = ClockSampler(local)
    peak_clk.start()
    fp32_flops, fp32_ms = M.mirres_peak_fp32()
    l2_bps, l2_ms = M.mirres_peak_l2()
    peak_clocks = peak_clk.stop()
    peaks = {"fp32_tflops": fp32_flops / 1e12, "fp32_basis": "FMA microbenchmark (mirres_peak_fp32): 16 independent "
             f"chains per thread, {sm_count} SMs x 8 blocks of 256, {fp32_ms:.1f} ms timed launch",
             "l2_gbs": l2_bps / 1e9, "l2_basis": "32 MiB L2-resident buffer, 400 passes of 16-byte ld.global.cg "
             f"loads over all SMs (mirres_peak_l2), {l2_ms:.1f} ms timed launch",
             "sm_count": sm_count, "nominal_fp32_tflops_at_max_clock": sm_count * 128 * 2 * 2.070e9 / 1e12,
             "clocks_during_peaks": peak_clocks}

    w = make_workload(args.workload, args.views)
    builder = M.MIRRES_BVH_PLOC if args.bvh == "ploc" else M.MIRRES_BVH_LBVH
    traversal = M.MIRRES_TRAVERSAL_WIDE if args.traversal == "wide" else M.MIRRES_TRAVERSAL_BINARY
    gw = GpuWorkload(w, local, builder=builder, traversal=traversal)
    samples = w.samples
    stream = torch.cuda.current_stream()
    scenes = [s.handle for s in gw.scenes]
    # views of one size render into one [N][H][W][3] stack (the denoiser then takes the stack
    # in one launch per level)
    sizes = {(v.width, v.height) for v in gw.views}
    uniform = len(sizes) == 1
    if uniform:
        (W0, H0), = sizes
        img_stack = torch.empty((len(gw.views), H0, W0, 3), device=dev)
        images = list(img_stack.unbind(0))
    else:
        images = gw.new_images()
    # one tape for every arm: FULL-mode size when it fits (a FULL tape also serves PRIMARY mode),
    # leaving room for the wavefront queues and the workspace
    full_bytes = M.mirres_tape_bytes_mode(gw.views, M.GRAD_FULL)
    free_bytes, _ = torch.cuda.mem_get_info(dev)
    want_full = (not args.no_full) and full_bytes + (24 << 30) < free_bytes
    tape = gw.new_tape(M.GRAD_FULL if want_full else M.GRAD_PRIMARY)
    grads = gw.zero_grads()
    tuned = None
    if not args.block:
        t0 = time.perf_counter()
        tuned = gw.autotune(tape=tape, budget=min(samples, 32_000_000))
        tuned["tuning_s"] = time.perf_counter() - t0
    # reference images: the same scene rendered with another seed
    refs, _ = gw.render(launch=1, seed=w.seed + 1, tape=tape)
    refs = [r.clone() for r in refs]
    if uniform:
        d_stack = torch.empty_like(img_stack)
        d_images = list(d_stack.unbind(0))
    else:
        d_images = [torch.empty_like(r) for r in refs]
    loss = torch.zeros(1, device=dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    history = None

    def step(launch, ev_render=None, ev_bwd=None, grad_mode=0, reuse=(0, 0), temporal=0, before_loss=None):
        for s in gw.scenes:
            M.mirres_bvh_build(s.handle)
        if ev_render is not None:
            ev_render[0].record()
        # the batched wavefront records stage events (graph event nodes) for the roofline
        M.mirres_render(gw.ctx, scenes, gw.views, gw.params(launch, block=args.block, blocks_per_sm=args.blocks_per_sm,
                                                            flags=(1 | BIN_FLAG) if launch == 1 else 0,
                                                            grad_mode=grad_mode, reuse=reuse, temporal=temporal,
                                                            history=history),
                        images, tape)
        if ev_render is not None:
            ev_render[1].record()
        if before_loss is not None:
            before_loss()
        for img, ref, d in zip(images, refs, d_images):
            M.mirres_l2_loss(img, ref, d, loss)
        if ev_bwd is not None:
            ev_bwd[0].record()
        M.mirres_backward(gw.ctx, scenes, gw.views, gw.params(launch, grad_mode=grad_mode, reuse=reuse), d_images,
                          tape, grads)
        if ev_bwd is not None:
            ev_bwd[1].record()

    def zero():
        for g in grads:
            for t in g.values():
                t.zero_()
        loss.zero_()

    def timed(launch, steps, warmup, grad_mode=0, reuse=(0, 0), temporal=0):
        for k in range(warmup):
            zero()
            step(launch, grad_mode=grad_mode, reuse=reuse, temporal=1 if (temporal and k == 0) else temporal)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        c0 = M.mirres_get_counters(gw.ctx)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))  # evict L2 between timed steps (outside the timed window)
            zero()
            evs[i][0].record()
            step(launch, evr[i], evg[i], grad_mode=grad_mode, reuse=reuse, temporal=temporal)
            evs[i][1].record()
        torch.cuda.synchronize()
        barrier()
        c1 = M.mirres_get_counters(gw.ctx)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        ms_render = sum(a.elapsed_time(b) for a, b in evr)
        timed.backward_ms = sum(a.elapsed_time(b) for a, b in evg) / steps
        rays = (c1[0] - c0[0]) + (c1[1] - c0[1]) + (c1[2] - c0[2])
        launches = c1[6] - c0[6]
        return ms, ms_render, rays, launches, [c1[k] - c0[k] for k in range(8)]

    def max_over_ranks(x):
        return reduce_max(x, dev)

    clocks = ClockSampler(local)
    clocks.start()
    ms_b, msr_b, rays_b, launches_b, cnt_b = timed(1, args.steps, args.warmup)
    clk = clocks.stop()
    backward_ms = timed.backward_ms
    stages = M.mirres_stage_times(gw.ctx)  # stage times of the last timed batched render
    by_bounce = {}
    for name, b, ms in M.mirres_stage_trace(gw.ctx):
        if b >= 0:
            by_bounce.setdefault(name, {}).setdefault(b, 0.0)
            by_bounce[name][b] += ms
    ms_b = max_over_ranks(ms_b)
    # traversal work of one render, counted outside the timed region by the separately compiled
    # counting variant of the traversal kernels (deterministic: the same rays visit the same
    # nodes in every render)
    w0 = M.mirres_get_work_counters(gw.ctx)
    M.mirres_render(gw.ctx, scenes, gw.views, gw.params(1, flags=2), images, tape)
    work = [b - a for a, b in zip(w0, M.mirres_get_work_counters(gw.ctx))]
    # per-launch stage times for the rooflines: with concurrent wave chains (branches > 1) the
    # launches of different chains overlap and each one's event span includes the other's work,
    # so the stages are re-timed in an untimed render whose chains run one at a time
    shape = M.mirres_get_wave_shape(gw.ctx)
    stages_roof, roof_basis = stages, "stage events of the last timed render"
    if shape.get("branches", 1) > 1:
        M.mirres_set_wave_shape(gw.ctx, dict(shape, branches=1))
        for _ in range(2):  # the first render captures the graph
            M.mirres_render(gw.ctx, scenes, gw.views, gw.params(1, flags=1), images, tape)
        torch.cuda.synchronize()
        stages_roof = M.mirres_stage_times(gw.ctx)
        roof_basis = ("stage events of an untimed render with the same shape but one wave chain (branches = 1): "
                      "the timed render's concurrent chains overlap their launches")
        M.mirres_set_wave_shape(gw.ctx, shape)

    def arm(launch):
        ms, msr, rays, launches, _ = timed(launch, args.steps, args.warmup)
        ms = max_over_ranks(ms)
        return {"value": world * samples * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                "mrays_per_s": world * rays / (ms / 1e3) / 1e6, "render_ms_per_step": msr / args.steps,
                "gpu_launches": launches}

    plain = None if args.no_plain else arm(0)
    persistent = None if args.no_plain else dict(arm(2), launch_shape=tuned)

    # end to end: host parameters and reference images in pinned memory, copies in the timed region
    host_params = [{k: t.detach().cpu().pin_memory() for k, t in s.params().items()} for s in gw.scenes]
    host_refs = [r.cpu().pin_memory() for r in refs]
    host_grads = [{k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in g.items()} for g in grads]
    host_loss = torch.empty(1).pin_memory()
    h2d = sum(t.numel() * t.element_size() for hp in host_params for t in hp.values()) + \
        sum(t.numel() * t.element_size() for t in host_refs)
    d2h = sum(t.numel() * t.element_size() for hg in host_grads for t in hg.values()) + 4

    copy_stream = torch.cuda.Stream(device=dev)

    def e2e_step():
        # this step's inputs from pinned host memory: the scene parameters before the render on
        # the compute stream, the reference images (the bulk) on a copy stream that overlaps the
        # render and is waited for before the loss
        for s, hp in zip(gw.scenes, host_params):
            for k, t in s.params().items():
                t.copy_(hp[k], non_blocking=True)
        copy_stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(copy_stream):
            for r, hr in zip(refs, host_refs):
                r.copy_(hr, non_blocking=True)
        refs_ready = torch.cuda.Event()
        refs_ready.record(copy_stream)
        zero()
        step(1, before_loss=lambda: torch.cuda.current_stream().wait_event(refs_ready))
        for g, hg in zip(grads, host_grads):
            for k in g:
                hg[k].copy_(g[k], non_blocking=True)
        host_loss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for _ in range(1):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    # the denoiser between image and loss (EAWT, Appendix A), every view: G-buffer, forward and
    # adjoint; HBM-bound stencils (taps hit L1/L2). Algorithmic bytes per pixel: forward 108 (pack
    # image, normal, position: 36 in, 48 out) + 3 levels x (48 in, 20 out) - 4 (the last level
    # writes 12-byte colour), adjoint 28 (pack the gradient) + 3 levels x (52 in, 16 out) - 4
    eawt = None
    if not args.no_eawt:
        ep = M.EawtParams(EAWT_SIGMAS[0], EAWT_SIGMAS[1], EAWT_SIGMAS[2], 3)
        if uniform:  # the whole stack per level
            gbn_s, gbx_s, out_s, grad_s = (torch.empty_like(img_stack) for _ in range(4))
            gbn, gbx = list(gbn_s.unbind(0)), list(gbx_s.unbind(0))
            rec_s = torch.empty(len(gw.views) * M.mirres_eawt_record_bytes(W0, H0, 3) // 4, device=dev)
        else:
            gbn = [torch.empty_like(im) for im in images]
            gbx = [torch.empty_like(im) for im in images]
            dn_out = [torch.empty_like(im) for im in images]
            dn_grad = [torch.empty_like(im) for im in images]
            recs = [torch.empty(M.mirres_eawt_record_bytes(v.width, v.height, 3) // 4, device=dev) for v in gw.views]

        def eawt_pass(ev=None):
            for vi, v in enumerate(gw.views):
                M.mirres_gbuffer(gw.ctx, gw.scenes[v.scene].handle, v, gbn[vi], gbx[vi])
            if ev is not None:
                ev[0].record()
            if uniform:
                M.mirres_eawt_batch(gw.ctx, img_stack, gbn_s, gbx_s, ep, out_s, rec_s)
                M.mirres_eawt_batch_backward(gw.ctx, d_stack, gbn_s, gbx_s, ep, rec_s, grad_s)
            else:
                for vi in range(len(gw.views)):
                    M.mirres_eawt(gw.ctx, images[vi], gbn[vi], gbx[vi], ep, dn_out[vi], recs[vi])
                for vi in range(len(gw.views)):
                    M.mirres_eawt_backward(gw.ctx, d_images[vi], gbn[vi], gbx[vi], ep, recs[vi], dn_grad[vi])
            if ev is not None:
                ev[1].record()

        for _ in range(args.warmup):
            eawt_pass()
        torch.cuda.synchronize()
        e_all = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e_dn = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e_all[0].record()
        for _ in range(args.steps):
            eawt_pass(e_dn)
        e_all[1].record()
        torch.cuda.synchronize()
        pix = sum(v.width * v.height for v in gw.views)
        ms_all = e_all[0].elapsed_time(e_all[1]) / args.steps
        ms_dn = e_dn[0].elapsed_time(e_dn[1])  # the last pass
        bytes_px = (84 + 3 * 68 - 4) + (28 + 3 * 68 - 4)
        ach = pix * bytes_px / (ms_dn / 1e3) / 1e9
        eawt = {"mpix_per_s": pix / (ms_all / 1e3) / 1e6, "ms_per_step": ms_all,
                "ms_denoise_fwd_bwd": ms_dn, "pixels": pix, "levels": 3, "sigmas": list(EAWT_SIGMAS),
                "roofline": {"bound": "hbm", "achieved": ach, "peak": HBM_PEAK, "unit": "GB/s",
                             "frac": ach / HBM_PEAK, "traffic": None, "bytes_per_pixel": bytes_px,
                             "kernel": "k_eawt_level + k_eawt_level_adjoint",
                             "launches_per_level": 1 if uniform else len(gw.views),
                             "peak_basis": "hbm_gbs of MEASURED_PEAKS.json"}}

    # mesh regularisers added to the loss (L_smooth + L_offset, Appendix A) on every scene: one
    # call per scene. Algorithmic bytes: per vertex 12 (position) + 12 (rest position) + 4 (1 /
    # neighbour count) + 24 (gradient read and written), per unique edge 8 (its two indices)
    regs = None
    if not args.no_regularizers:
        rests = [s.verts.clone() for s in gw.scenes]
        rl = torch.zeros(1, device=dev)
        rg = [torch.zeros_like(s.verts) for s in gw.scenes]

        def reg_pass():
            for si, s in enumerate(gw.scenes):
                M.mirres_mesh_regularizers(gw.ctx, s.handle, rests[si], 0.1, 0.01, rl, rg[si])

        for _ in range(max(args.warmup, 3)):
            reg_pass()
        torch.cuda.synchronize()
        e_rg = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e_rg[0].record()
        for _ in range(args.steps):
            reg_pass()
        e_rg[1].record()
        torch.cuda.synchronize()
        ms_rg = e_rg[0].elapsed_time(e_rg[1]) / args.steps
        nv = sum(int(s.verts.shape[0]) for s in gw.scenes)
        ne = sum(_unique_edges(sc.tris) for sc in w.scenes)
        bytes_rg = nv * 52 + 8 * ne
        ach = bytes_rg / (ms_rg / 1e3) / 1e9
        regs = {"ms_per_step": ms_rg, "vertices": nv, "edges": ne, "weights": [0.1, 0.01],
                "roofline": {"bound": "hbm", "achieved": ach, "peak": HBM_PEAK, "unit": "GB/s", "frac": ach / HBM_PEAK,
                             "traffic": None, "kernel": "k_smooth + k_offset",
                             "bytes_note": "52 B per vertex + 8 B per unique edge; the mesh is L2-resident",
                             "peak_basis": "hbm_gbs of MEASURED_PEAKS.json"}}
        # material smoothness L_k over every view's pixel-centre hits (one closest-hit ray per
        # pixel, then the albedo / roughness lookup differences and their scattered gradient)
        lkp = M.LkParams(0.01, 0.1, 0.1, 0, 0)
        lk_l = torch.zeros(1, device=dev)
        lk_ga = [torch.zeros_like(s.albedo) for s in gw.scenes]
        lk_gr = [torch.zeros_like(s.roughness) for s in gw.scenes]

        def lk_pass():
            for vi, v in enumerate(gw.views):
                sc_i = v.scene
                M.mirres_material_smoothness(gw.ctx, gw.scenes[sc_i].handle, v, vi, lkp, lk_l, lk_ga[sc_i],
                                             lk_gr[sc_i])

        for _ in range(max(args.warmup, 3)):
            lk_pass()
        torch.cuda.synchronize()
        e_lk = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e_lk[0].record()
        for _ in range(args.steps):
            lk_pass()
        e_lk[1].record()
        torch.cuda.synchronize()
        ms_lk = e_lk[0].elapsed_time(e_lk[1]) / args.steps
        pix = sum(v.width * v.height for v in gw.views)
        regs["material_smoothness"] = {"ms_per_step": ms_lk, "pixels": pix, "mpix_per_s": pix / (ms_lk / 1e3) / 1e6,
                                       "sigma": 0.01, "kernel": "k_lk_hits + k_lk_apply"}
        rests = rg = lk_ga = lk_gr = None
        # monochrome light regulariser L_light over every view, from the tape of the last render:
        # the demodulated lighting per pixel (the primary vertex replayed for each sample), the
        # loss against the reference images and its seed, and the adjoint (replayed again)
        lp = gw.params(1)
        ll_c = [torch.empty((v.height, v.width, 4), device=dev) for v in gw.views]
        ll_d = [torch.empty((v.height, v.width, 3), device=dev) for v in gw.views]
        ll_l = torch.zeros(1, device=dev)
        ll_g = gw.zero_grads()

        def light_pass():
            M.mirres_light_demod(gw.ctx, scenes, gw.views, lp, tape, ll_c)
            M.mirres_light_loss(gw.ctx, gw.views, ll_c, refs, 0.1, ll_l, ll_d)
            M.mirres_light_backward(gw.ctx, scenes, gw.views, lp, ll_d, tape, ll_g)

        for _ in range(max(args.warmup, 3)):
            light_pass()
        torch.cuda.synchronize()
        e_ll = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e_ll[0].record()
        for _ in range(args.steps):
            light_pass()
        e_ll[1].record()
        torch.cuda.synchronize()
        ms_ll = e_ll[0].elapsed_time(e_ll[1]) / args.steps
        # the demodulated-lighting kernel alone: a stream over the tape's primary words (4 B for
        # a sample whose primary ray escaped, 56 B for one that hit) plus 16 B written per pixel;
        # the hit count is exact from the coverage channel
        # timed over DEMOD_REPS calls, one event pair each (the call's table uploads are a few
        # hundred bytes); mean and spread reported
        e_dm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(DEMOD_REPS)]
        for a, b in e_dm:
            a.record()
            M.mirres_light_demod(gw.ctx, scenes, gw.views, lp, tape, ll_c)
            b.record()
        torch.cuda.synchronize()
        ms_all = [a.elapsed_time(b) for a, b in e_dm]
        ms_dm = sum(ms_all) / len(ms_all)
        hits = int(round(sum(float((c[..., 3].double() * v.spp).sum()) for c, v in zip(ll_c, gw.views))))
        bytes_dm = 56 * hits + 4 * (samples - hits) + 16 * pix
        ach_dm = bytes_dm / (ms_dm / 1e3) / 1e9
        regs["light"] = {"ms_per_step": ms_ll, "pixels": pix, "samples": samples,
                         "mpix_per_s": pix / (ms_ll / 1e3) / 1e6,
                         "msamples_per_s": samples / (ms_ll / 1e3) / 1e6, "weight": 0.1,
                         "kernel": "k_light_demod + k_light_count + k_light_apply + k_backward<DEMOD>",
                         "demod_ms": ms_dm, "demod_ms_min": min(ms_all), "demod_ms_max": max(ms_all),
                         "demod_repeats": len(ms_all), "demod_hit_samples": hits,
                         "roofline": {"bound": "hbm", "achieved": ach_dm, "peak": HBM_PEAK, "unit": "GB/s",
                                      "frac": ach_dm / HBM_PEAK, "traffic": None, "bytes": bytes_dm,
                                      "kernel": "k_light_demod",
                                      "bytes_note": "56 B per hit sample, 4 B per escaped sample, 16 B per pixel",
                                      "peak_basis": "hbm_gbs of MEASURED_PEAKS.json"}}
        ll_c = ll_d = ll_g = None

    # FULL-mode adjoint (gradients through every vertex): the same step with grad_mode 1
    full = None
    if want_full:
        ms_f, msr_f, _, launches_f, _ = timed(1, args.steps, args.warmup, grad_mode=M.GRAD_FULL)
        ms_f = max_over_ranks(ms_f)
        full = {"value": world * samples * args.steps / (ms_f / 1e3), "ms_per_step": ms_f / args.steps,
                "render_ms_per_step": msr_f / args.steps, "backward_ms_per_step": timed.backward_ms,
                "tape_bytes": full_bytes, "gpu_launches": launches_f}
    elif not args.no_full:
        full = {"skipped": f"FULL tape of {full_bytes / 2**30:.1f} GiB does not fit next to the workload"}

    # spatial reservoir reuse at the primary vertex (Appendix A), REUSE neighbours in a square of
    # radius REUSE_RADIUS: the same step
    reuse_arm = None
    if not args.no_reuse:
        ms_r, msr_r, _, launches_r, _ = timed(1, args.steps, args.warmup, reuse=REUSE)
        ms_r = max_over_ranks(ms_r)
        reuse_arm = {"value": world * samples * args.steps / (ms_r / 1e3), "ms_per_step": ms_r / args.steps,
                     "render_ms_per_step": msr_r / args.steps, "backward_ms_per_step": timed.backward_ms,
                     "neighbours": REUSE[0], "radius": REUSE[1], "gpu_launches": launches_r}
        # spatial and temporal reuse: each step merges the reservoir history the previous one left
        history = gw.new_history()
        ms_t, msr_t, _, launches_t, _ = timed(1, args.steps, args.warmup, reuse=REUSE, temporal=2)
        ms_t = max_over_ranks(ms_t)
        reuse_arm["spatial_temporal"] = {"value": world * samples * args.steps / (ms_t / 1e3),
                                         "ms_per_step": ms_t / args.steps, "render_ms_per_step": msr_t / args.steps,
                                         "temporal_cap": 20, "gpu_launches": launches_t}
        history = None

    value = world * samples * args.steps / (ms_b / 1e3)
    mrays = world * rays_b / (ms_b / 1e3) / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(w, args.workload), parallelism=f"replicas{world}", bvh=args.bvh,
                           traversal=args.traversal,
                           l2="flushed between timed steps (512 MiB write) and each step writes > 40 GB"),
            "mrays_per_s": mrays, "render_ms_per_step": msr_b / args.steps, "backward_ms_per_step": backward_ms,
            "batched": {"value": value, "ms_per_step": ms_b / args.steps, "mrays_per_s": mrays,
                        "launch": "batched wavefront, one CUDA graph per forward",
                        "launch_shape": M.mirres_get_wave_shape(gw.ctx),
                        "binned_continuation_rays": bool(args.bin),
                        "launch_shape_stages": list(M.WAVE_STAGES),
                        "stage_ms_per_render": {k: v[0] for k, v in stages.items()},
                        "stage_ms_by_bounce": {k: [v[b] for b in sorted(v)] for k, v in by_bounce.items()},
                        "stage_launches_per_render": {k: v[1] for k, v in stages.items()},
                        "stage_ms_per_render_one_chain": {k: v[0] for k, v in stages_roof.items()}},
            "plain": plain,
            "persistent": persistent,
            "full_adjoint": full,
            "denoiser": eawt,
            "mesh_regularizers": regs,
            "spatial_reuse": reuse_arm,
            "speedup_batched_over_plain": (value / plain["value"]) if plain else None,
            "counters_per_step": {"primary_rays": cnt_b[0] // args.steps, "continuation_rays": cnt_b[1] // args.steps,
                                  "shadow_rays": cnt_b[2] // args.steps, "ris_candidates": cnt_b[5] // args.steps,
                                  "samples_differentiated": cnt_b[4] // args.steps},
            "gpu_launches": launches_b,
            "clocks": clk,
            "peaks": peaks,
            "e2e": {"value": world * samples * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}

    # roofline of the dominant stage kernel of the batched forward. All three are bound by FP32
    # arithmetic (their data is L2-resident, no tensor-core work); algorithmic FLOPs per unit:
    # shade (k_wshade): per RIS candidate 60 (BRDF luminance and cosine) + 2 log2(env texels)
    # (the two CDF inversions); closest hit and shadow rays (k_wclosest / k_wclosest_refill,
    # k_wshadow_refill): 12 per box
    # test (slab) + 27 per triangle test. Candidates and box / triangle tests are counted by the
    # library; times come from the stage events captured in the graph.
    env_texels = sum(s.env.shape[0] * s.env.shape[1] for s in w.scenes) / len(w.scenes)
    per_cand = 60 + 2 * math.log2(env_texels)
    cand_per_render = cnt_b[5] / args.steps
    peak = peaks["fp32_tflops"]
    total_stage_ms = max(sum(v[0] for v in stages_roof.values()), 1e-9)
    stage_flops = {"shade": cand_per_render * per_cand,
                   "closest": 12.0 * work[0] + 27.0 * work[1],
                   "shadow": 12.0 * work[2] + 27.0 * work[3]}
    names = {"shade": "k_wshade (shade + RIS stage)",
             "closest": "k_wclosest + k_wclosest_refill (closest-hit stage: primary, then continuation rays)",
             "shadow": "k_wshadow (shadow-ray stage)"}
    units_per_render = {"closest": (cnt_b[0] + cnt_b[1]) / args.steps, "shade": cand_per_render,
                        "shadow": cnt_b[2] / args.steps}
    traffic_ok = _traffic_valid()
    roofs = {}
    for k in ("closest", "shade", "shadow"):
        ms_k, launches_k = stages_roof[k]
        achieved = stage_flops[k] / (ms_k / 1e3) / 1e12
        traffic = (TRAFFIC_PER_UNIT[k] * units_per_render[k] / max(launches_k, 1)) if traffic_ok else None
        roofs[k] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": traffic, "traffic_unit": "bytes per launch",
                    "traffic_basis": "ncu DRAM bytes per unit on a 2-view capture x units per launch",
                    "kernel": names[k], "kernel_ms_per_launch": ms_k / max(launches_k, 1),
                    "kernel_share_of_render": ms_k / total_stage_ms, "flops_per_render": stage_flops[k],
                    "timing_basis": roof_basis,
                    "peak_basis": "measured FP32 FMA rate of this device (peaks.fp32_basis), non-tensor"}
        if k in ("closest", "shadow"):
            # the memory side: the traversal's algorithmic bytes (32 B per box test, i.e. per
            # child box, + 36 B per triangle test) over the time, against the measured L2 load
            # bandwidth (the nodes and triangles are L2-resident)
            box, tri = (work[0], work[1]) if k == "closest" else (work[2], work[3])
            nbytes = 32.0 * box + 36.0 * tri
            ach = nbytes / (ms_k / 1e3) / 1e9
            roofs[k]["memory"] = {"bound": "l2", "achieved": ach, "peak": peaks["l2_gbs"], "unit": "GB/s",
                                  "frac": ach / peaks["l2_gbs"], "bytes_per_render": nbytes,
                                  "peak_basis": "measured L2 load bandwidth (peaks.l2_basis)"}
    roofs["shade"].update(flops_per_candidate=per_cand, candidates_per_render=cand_per_render)
    roofs["closest"].update(box_tests_per_render=work[0], triangle_tests_per_render=work[1])
    roofs["shadow"].update(box_tests_per_render=work[2], triangle_tests_per_render=work[3])
    dominant = max(("closest", "shade", "shadow"), key=lambda k: stages_roof[k][0])
    line["roofline"] = dict(roofs[dominant])
    line["stage_rooflines"] = roofs
    if rank == 0 and not args.no_cpu:
        cb, counts, osamples = cpu_baseline(w)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    gw.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
