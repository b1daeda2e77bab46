"""Benchmark: forward + backward Monte Carlo direct-illumination shading.

A step is one pass of the hot path over one synthetic batch: probe sampling
tables, LBVH over this iteration's mesh, rasterised G-buffer, forward MIS
estimator with shadow rays, the U-Net denoiser on c_d and c_s, its input
gradient, and the shading adjoint (Sec. 3-4 of the paper).  The
workload is the 512 x 512, 16 spp (8 light / 4 cosine / 4 GGX) view of the
~198k-triangle sphere-union mesh with 1024^2 textures and a 512 x 256
three-lobe probe.  The metric is shaded samples per second (covered pixels x
spp, forward + backward), with the dominant kernel's HBM roofline fraction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mcdi|reference]

N > 1 runs under torchrun, one independent replica per GPU (weak scaling; the
path has no data exchange that this single-GPU build performs).  The
``reference`` arm times the FP64 CPU oracle on a bounded pixel sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd MC shading Msamples/s & %HBM roofline at 512² 16spp"
# DRAM bytes (read + write) per launch at the headline size, from one ncu capture of the kernel as it
# stands (profiles/); an entry is removed when its kernels change.
MEASURED_TRAFFIC = {"wave_trace_kernel": 41.83e6, "shade_fwd": 109.7e6, "shade_bwd": 24.9e6}
UNIT = "Msamples/s"
L2_FLUSH_BYTES = 512 << 20
# serving: requests of fewer than 2M samples in one lane, the rest in another (measured against 1M - 3M
# bounds and against one shared queue on 2-4 streams: the lanes gain at twice the offered rate and tie at it)
SERVING_LANES = (2e6,)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def tensor_peak():
    """BF16 dense peak for a kernel timed inside a long step: the sustained figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops_sustained" in d:
            return d["bf16_tflops_sustained"], "measured (sustained)"
        if "bf16_tflops" in d:
            return d["bf16_tflops"], "measured (burst)"
    return 1700.0, "fallback (sustained)"


# ------------------------------------------------------------------ distributed harness
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def init_dist(backend):
    import torch.distributed as dist

    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, world


def replica_seed(base: int, rank: int, world: int) -> int:
    """Seed of a replica's synthetic workload: each rank renders its own scene (weak scaling)."""
    return base + 1000 * rank if world > 1 else base


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(", ") for r in self.out.strip().splitlines() if r.strip()]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4) if r[5 + k].strip() == "Active"})
        busy = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}



# ------------------------------------------------------------------ algorithmic bytes
def tracer_structure_bytes(bvh) -> int:
    """Bytes of the traversal structure the shadow-ray tracer reads: the four-wide nodes of the
    built tree (64 B each) and the 48-byte triangle records."""
    from paper_2206_03380_gb300 import mcdi

    return mcdi.tracer_structure_bytes(bvh)


def algorithmic_bytes(P: int, spp: int, structure: int, probe, env) -> dict:
    """Algorithmic HBM bytes per launch of the shading stages at P pixels (all pixels of the views):

    forward   per pixel: G-buffer payload in 48 B (position, normal, k_d, k_orm: 12 B each), outputs
              c_d / k_d,out / c_s 36 B, visibility spp/8 B; once: the traversal structure, the probe
              (16 B per texel as stored) and its tables
    tracer    the traversal structure once and the visibility bits (spp/8 B per pixel)
    backward  per pixel: upstream gradients 36 B, G-buffer payload 48 B, visibility spp/8 B, gradients
              of k_d, k_orm and N 36 B; once: probe and tables, probe gradient written (12 B per texel)
    """
    vis = spp / 8.0
    probe_bytes = env.nbytes + probe.cond.numel() * 4 + probe.marg.numel() * 4
    texels = env.shape[0] * env.shape[1]
    return {"shade_fwd": P * (48 + 36 + vis) + structure + probe_bytes,
            "wave_trace": structure + P * vis,
            "shade_bwd": P * (36 + 48 + vis + 36) + probe_bytes + 12 * texels}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world):
    import torch

    from paper_2206_03380_gb300 import mcdi, scenes
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    local = dist_env()[2]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.sphere_union_scene(seed=replica_seed(scenes.BASE_SEED + 2, rank, world))
    den_params = mcdi.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3))
    pipe = ShadingPipeline(sc, device=dev, denoiser_params=den_params)
    N, H, W = pipe.N, pipe.H, pipe.W
    rng = np.random.default_rng(3)
    # the step is driven by the paper's image loss against a synthetic reference image (positive radiance)
    ref = torch.from_numpy(np.abs(rng.lognormal(-0.5, 1.0, size=(N, H, W, 4))).astype(np.float32)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    stages = ["probe_cdf", "bvh_build", "primary_cast", "shade_fwd", "denoise_fwd", "loss", "denoise_bwd",
              "shade_bwd"]
    # the library's kernels per step at this size (the level-0 and level-1 max-pools run inside the
    # convolutions' epilogues, the level-2 one as its own kernel; the G-buffer is rasterised: depth-buffer
    # clear, raster, resolve)
    n_launch = {"probe_cdf": 2, "bvh_build": mcdi.bvh_build_launches(sc.tris.shape[0]), "primary_cast": 3,
                "shade_fwd": 4, "denoise_fwd": 1 + 15 + 1, "loss": 2, "denoise_bwd": 1 + 15 + 3,
                "shade_bwd": 1}

    def one_step(ev=None):
        calls = [pipe.build_probe, pipe.build_bvh, pipe.primary, pipe.forward, pipe.denoise,
                 lambda: pipe.image_loss(ref),
                 lambda: pipe.denoise_backward(pipe.g_loss_terms),
                 lambda: pipe.backward(pipe.g_terms[:N], pipe.g_loss_kdout, pipe.g_terms[N:])]
        for k, f in enumerate(calls):
            if ev is not None:
                ev[k].record(stream)
            f()
        if ev is not None:
            ev[len(calls)].record(stream)

    clk = ClockSampler(local)
    clk.__enter__()  # samples clocks from the warm-up (at least 1 s of load) through the timed region
    t_w = time.perf_counter()
    k = 0
    while k < args.warmup or time.perf_counter() - t_w < 1.0:
        flush.zero_()
        one_step()
        torch.cuda.synchronize()
        k += 1
    covered = pipe.covered_pixels()
    samples_per_step = covered * sc.spp

    # (1) eager launches with an event between stages: the per-stage breakdown
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for _ in range(4):
        flush.zero_()  # a queue of device work so that the first timed launch does not wait for the host
    for s in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        one_step(evs[s])
    torch.cuda.synchronize()
    stage_ms = {st: [evs[s][k].elapsed_time(evs[s][k + 1]) for s in range(args.steps)] for k, st in enumerate(stages)}
    eager_ms = max_over_ranks(float(np.mean([evs[s][0].elapsed_time(evs[s][-1]) for s in range(args.steps)])), dev)
    total_samples = sum_over_ranks(float(samples_per_step), dev)

    # (2) the headline: the same step captured once in a CUDA graph and replayed, one host launch per
    # step; warm-up replays, then exactly `steps` timed replays, each bracketed by CUDA events on the
    # launching stream, the L2 flushed between them (outside the events)
    pipe.capture_loss_step(ref)
    for _ in range(args.warmup):
        flush.zero_()
        pipe.replay()
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for _ in range(4):
        flush.zero_()
    t0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        gev[s][0].record(stream)
        pipe.replay()
        gev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk.__exit__(None, None, None)
    dev_ms_max = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in gev])), dev)
    value = total_samples / (dev_ms_max * 1e-3) / 1e6

    # e2e: host inputs -> device -> the step -> host outputs, every step.  The step's own host I/O
    # overlaps its compute (pipeline.loss_step_io: uploads in the order the stages first read them, each
    # stage waiting only for its inputs, outputs read back as soon as their producer has run), all of it
    # in one captured graph; nothing of a later step is copied early.  The same step with the copies
    # serialised around the graph replay is timed beside it (e2e.serial_ms).
    # the material textures as RGB / ORM triples (the device copy pads them to float4; the 4th channel
    # carries nothing)
    host_in = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in
               [("verts", sc.verts), ("vnrm", sc.vnrm), ("tris", sc.tris), ("env", sc.env),
                ("tex_kd", sc.tex_kd[..., :3]), ("tex_korm", sc.tex_korm[..., :3])]}
    host_ref = ref.cpu().pin_memory()
    outs_dev = [pipe.loss, pipe.color, pipe.g_kd, pipe.g_korm, pipe.g_nrm, pipe.g_env]
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs_dev]
    h2d = sum(t.numel() * t.element_size() for t in list(host_in.values()) + [host_ref])
    d2h = sum(t.numel() * t.element_size() for t in host_out)

    pipe.capture_loss_step_io(ref, host_in, host_ref, list(zip(outs_dev, host_out)))

    def e2e_serial_step():
        pipe.verts.copy_(host_in["verts"], non_blocking=True)
        pipe.vnrm.copy_(host_in["vnrm"], non_blocking=True)
        pipe.tris.copy_(host_in["tris"], non_blocking=True)
        pipe.env.copy_(host_in["env"], non_blocking=True)
        pipe.tex_kd[..., :3].copy_(host_in["tex_kd"], non_blocking=True)
        pipe.tex_korm[..., :3].copy_(host_in["tex_korm"], non_blocking=True)
        ref.copy_(host_ref, non_blocking=True)
        pipe.replay()
        for h, d in zip(host_out, outs_dev):
            h.copy_(d, non_blocking=True)

    def time_e2e(step_fn):
        for _ in range(2):
            step_fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step_fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)

    e2e_serial_ms = time_e2e(e2e_serial_step)
    e2e_ms = time_e2e(pipe.replay_io)
    e2e_value = total_samples / (e2e_ms * 1e-3) / 1e6

    # rooflines: algorithmic bytes (or FLOPs) per launch / CUDA-event time
    avg = {st: float(np.mean(v)) for st, v in stage_ms.items()}
    P = N * H * W
    algo = algorithmic_bytes(P, sc.spp, tracer_structure_bytes(pipe.bvh), pipe.probe, sc.env)
    # denoiser: algorithmic tensor FLOPs (2 * 9 * c_in * c_out per output pixel and conv, unpadded)
    conv_flops = 0
    for name, ci, co in scenes.UNET_SHAPES:
        lvl = {"enc1": 0, "enc2": 1, "enc3": 2, "bot_": 3, "dec3": 2, "dec2": 1, "dec1": 0, "out": 0}[name[:4]]
        conv_flops += 2 * 9 * ci * co * (2 * N) * (H >> lvl) * (W >> lvl)
    flops = {"denoise_fwd": conv_flops, "denoise_bwd": conv_flops}  # input-gradient convs: same shapes
    peak, peak_kind = peaks()
    rays = shadow_ray_figures(pipe, flush, stream, args.steps, samples_per_step)
    # the dominant kernel of the step (largest share of the launch list): the shadow-ray tracer, timed
    # alone with CUDA events on its launching stream (L2 flushed before each launch)
    t_trace = rays["ms"]
    achieved = algo["wave_trace"] / (t_trace * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "wave_trace_kernel", "achieved": round(achieved, 2), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 5), "traffic": MEASURED_TRAFFIC.get("wave_trace_kernel"),
            "peak_source": peak_kind, "algorithmic_bytes": int(algo["wave_trace"]), "ms": round(t_trace, 4),
            "note": "algorithmic bytes: the traversal structure read once (nodes + triangle records) and the "
                    "visibility bits written; the kernel is bound by L1 wavefronts of incoherent node fetches, "
                    "see shadow_rays"}
    stage_roof = {}
    for st in ("shade_fwd", "shade_bwd"):
        a = algo[st] / (avg[st] * 1e-3) / 1e9
        stage_roof[st] = {"achieved": round(a, 2), "peak": peak, "unit": "GB/s", "frac": round(a / peak, 5),
                          "algorithmic_bytes": int(algo[st]), "ms": round(avg[st], 4),
                          "traffic": MEASURED_TRAFFIC.get(st)}
    for st in ("denoise_fwd", "denoise_bwd"):
        tpeak, tkind = tensor_peak()
        a = flops[st] / (avg[st] * 1e-3) / 1e12
        stage_roof[st] = {"achieved": round(a, 2), "peak": tpeak, "unit": "TFLOP/s", "frac": round(a / tpeak, 5),
                          "algorithmic_flops": int(flops[st]), "ms": round(avg[st], 4), "peak_source": tkind}
    whole = sum(algo[st] for st in ("shade_fwd", "shade_bwd"))
    stage_roof["shading_fwd_bwd"] = {"algorithmic_bytes": int(whole),
                                     "frac_of_step": round(whole / (dev_ms_max * 1e-3) / 1e9 / peak, 5),
                                     "note": "forward + backward shading bytes over the whole graph-replayed step"}
    den_tf = {k: round(flops[k] / (avg[k] * 1e-3) / 1e12, 2) for k in flops}
    clocks = clk.summary()
    launches = args.steps * sum(n_launch.values())
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_ms_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded sphere-union SDF mesh, value-noise "
                                                   "textures, log-normal probe with sun lobes)",
        "config": {"workload": sc.name, "views": N, "width": W, "height": H, "spp": sc.spp,
                   "split": [sc.n_light, sc.n_cos, sc.n_ggx], "triangles": int(sc.tris.shape[0]),
                   "probe": [int(sc.env.shape[1]), int(sc.env.shape[0])], "texture": int(sc.tex_kd.shape[0]),
                   "pixels_covered": covered, "samples_per_step": samples_per_step,
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "launch": "the step captured once in a CUDA graph, one replay per timed step",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "stage_ms": {k: round(v, 4) for k, v in avg.items()},  # eager launches (events between stages)
        "wall_s": round(wall, 3),
        "roofline": roof,
        "stage_roofline": stage_roof,
        "denoiser_tflops": den_tf,
        "clocks": clocks,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 4),
                "serial_ms": round(e2e_serial_ms, 4),
                "note": "each step's own uploads and read-backs overlap its compute inside one graph "
                        "(pipeline.loss_step_io); serial_ms: the same copies serialised around the replay"},
        "gpu_launches": launches,
        "eager": {"ms_per_step": round(eager_ms, 4), "value": round(total_samples / (eager_ms * 1e-3) / 1e6, 2),
                  "unit": UNIT, "note": "the same step launched kernel by kernel from the host, with events between "
                                        "stages (the source of stage_ms)"},
    }
    result["denoiser_wgrad"] = time_denoiser_wgrad(pipe.denoiser, conv_flops, flush, stream, args.steps)
    result["denoiser_e4m3"] = time_denoiser_e4m3(pipe, den_params, conv_flops, flush, stream, args.steps)
    result["denoiser_bilateral"] = time_bilateral(pipe, flush, stream, args.steps)
    result["shadow_rays"] = rays
    result["bvh"] = time_bvh_refit(pipe, flush, stream, args.steps)
    result["shadow_edge_grad"] = time_shadow_edge_grad(pipe, flush, stream, args.steps)
    if world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(sc, n_pix=args.cpu_pixels)
    if args.batch_steps > 0:
        del pipe
        torch.cuda.empty_cache()
        result["step_batch"] = run_step_batch(args.batch_steps, flush, dev, rank, world)
    if args.serving_requests > 0:
        del flush
        torch.cuda.empty_cache()
        result["serving"] = run_serving(args.serving_requests, args.serving_rate, dev, rank)
    return result


def run_step_batch(steps, flush, dev, rank, world):
    """The optimisation-step batch: 8 of 200 views at 800^2, 32 spp, on the union of
    32 spheres and 32 boxes (256^3 grid, ~1.3M triangles), 2048^2 textures and a
    1024 x 512 probe; tables, BVH, G-buffer, forward, BF16 denoiser, image loss
    against a synthetic reference, denoiser input gradient and the adjoint,
    captured in one CUDA graph and replayed (L2 flushed before each replay)."""
    import torch

    from paper_2206_03380_gb300 import mcdi, scenes
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = scenes.union_step_scene(seed=replica_seed(scenes.BASE_SEED + 4, rank, world))
    den = mcdi.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3))
    pipe = ShadingPipeline(sc, device=dev, denoiser_params=den)
    rng = np.random.default_rng(5)
    ref = torch.from_numpy(np.abs(rng.lognormal(-0.5, 1.0, size=(pipe.N, pipe.H, pipe.W, 4))).astype(np.float32))
    ref = ref.to(dev)  # the graph reads this buffer: it lives until the replays are done
    pipe.capture_loss_step(ref)
    stream = torch.cuda.current_stream(dev)
    ms = []
    for k in range(steps + 2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pipe.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            ms.append(e0.elapsed_time(e1))
    if pipe.denoiser.err.item() != 0:
        raise RuntimeError("denoiser pipeline wait timed out")
    samples = pipe.covered_pixels() * sc.spp
    t = max_over_ranks(float(np.mean(ms)), dev)
    total = sum_over_ranks(float(samples), dev)
    # the tracer and the BVH at 1.3M triangles, where the BVH (~110 MB) no longer sits in L2
    rays = shadow_ray_figures(pipe, flush, stream, min(steps, 5), samples)
    bvh = time_bvh_refit(pipe, flush, stream, min(steps, 5))
    return {"workload": sc.name, "views": pipe.N, "width": pipe.W, "height": pipe.H, "spp": sc.spp,
            "triangles": int(sc.tris.shape[0]), "samples_per_step": int(samples), "ms_per_step": round(t, 3),
            "value": round(total / (t * 1e-3) / 1e6, 2), "unit": UNIT, "steps": steps,
            "note": "one CUDA graph replay per step", "shadow_rays": rays, "bvh": bvh}


def time_bilateral(pipe, flush, stream, steps, sigma=2.0):
    """The cross-bilateral denoiser (App. B, sigma = 2: 9 x 9 footprint) on the same two
    512^2 terms: forward and colour-adjoint times (CUDA events, L2 flushed before each)."""
    import torch

    from paper_2206_03380_gb300 import mcdi

    y, gx = torch.empty_like(pipe.denoised), torch.empty_like(pipe.denoised)
    g = torch.ones_like(pipe.denoised)
    wsum = torch.empty((pipe.N, pipe.H, pipe.W), device=pipe.device)
    fwd, bwd = [], []
    for k in range(steps + 3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        flush.zero_()
        ev[0].record(stream)
        mcdi.bilateral_fwd(pipe.gb.pos, pipe.gb.nrm, pipe.cams, pipe.terms, sigma, y, wsum, stream=stream)
        ev[1].record(stream)
        mcdi.bilateral_bwd(pipe.gb.pos, pipe.gb.nrm, pipe.cams, wsum, g, sigma, gx, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[1].elapsed_time(ev[2]))
    return {"sigma": sigma, "fwd_ms": round(float(np.mean(fwd)), 4), "bwd_ms": round(float(np.mean(bwd)), 4)}


# per-visit FP32 operations of the traversal, counted from the source: a visit of
# a four-wide node is 3 subtracts + 6 multiplies + 3 fused multiply-adds of
# set-up and per child 6 fused multiply-adds + 3 min/max (two of three operands)
# + 1 compare (52 in all; the byte-to-float moves are integer permutes); a
# two-sided Moller-Trumbore test that runs to the end is 2 cross products (9 ops
# each), 4 dot products (5 each), 1 reciprocal, 3 subtracts, 3 multiplies,
# 1 add and 6 compares (early outs make it shorter: an upper bound)
NODE_OPS, TRI_OPS = 52, 52
NODE_BYTES, TRI_BYTES, RAY_BYTES = 64, 48, 32


def alu_peak_gops():
    """Nominal FP32 lane-operation rate: SMs x 128 lanes x the maximum SM clock."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return sms * 128 * mhz * 1e6 / 1e9


def shadow_ray_figures(pipe, flush, stream, steps, samples):
    """The shadow-ray tracer of the forward pass timed alone (CUDA events, L2
    flushed before each launch) and its counters: node visits (64-byte four-wide
    nodes) and triangle tests per ray, the bytes it requests from the memory
    system (16-byte ray record and its pixel's 16-byte origin, 64-byte nodes,
    48-byte triangle records, one flag byte per blocked ray) against a measured
    L2 read bandwidth, and FP32 operations per sample."""
    import torch

    from paper_2206_03380_gb300 import mcdi

    pipe.forward(stream)
    st = torch.zeros(5, dtype=torch.int64, device=pipe.device)
    mcdi.shadow_ray_stats(pipe.bvh, pipe.N, pipe.H, pipe.W, pipe.params, pipe.workspace, st, stream)
    torch.cuda.synchronize()
    rays, visits, tests, blocked, differ = (int(v) for v in st.cpu())
    ms = []
    for k in range(steps + 3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        flush.zero_()
        ev[0].record(stream)
        mcdi.shadow_ray_retrace(pipe.bvh, pipe.N, pipe.H, pipe.W, pipe.params, pipe.workspace, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            ms.append(ev[0].elapsed_time(ev[1]))
    t = float(np.mean(ms))
    # L2 read bandwidth: 16-byte L1-bypassing loads over buffers that stay in L2, best of sizes and repeats
    sink = torch.zeros(1, dtype=torch.int32, device=pipe.device)
    l2 = 0.0
    for mib in (8, 16, 32):
        buf = torch.zeros(mib << 18, dtype=torch.int32, device=pipe.device)
        passes = 40
        for k in range(4):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            mcdi.read_sweep(buf, 1, sink, stream)  # bring it into L2
            ev[0].record(stream)
            mcdi.read_sweep(buf, passes, sink, stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            l2 = max(l2, (mib << 20) * passes / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e9)
        del buf
    req = rays * RAY_BYTES + visits * NODE_BYTES + tests * TRI_BYTES + blocked
    req_gbs = req / (t * 1e-3) / 1e9
    return {"kernel": "wave_trace_kernel", "ms": round(t, 4), "rays": rays, "disagree_with_forward": differ,
            "node_visits_per_ray": round(visits / max(rays, 1), 2),
            "tri_tests_per_ray": round(tests / max(rays, 1), 2), "blocked_frac": round(blocked / max(rays, 1), 4),
            "requested_bytes": req, "requested_gbs": round(req_gbs, 1), "l2_read_peak_gbs": round(l2, 1),
            "l2_peak_source": "measured (read sweep over 8-32 MiB)",
            "frac_of_l2_read_peak": round(req_gbs / l2, 4) if l2 > 0 else None,
            "traversal_fp32_ops_per_sample": round((visits * NODE_OPS + tests * TRI_OPS) / max(samples, 1), 1),
            "traversal_gops": round((visits * NODE_OPS + tests * TRI_OPS) / (t * 1e-3) / 1e9, 1),
            "alu_peak_gops": round(alu_peak_gops(), 1),
            "alu_peak_source": "derived: SMs x 128 FP32 lanes x max SM clock (one operation per lane per cycle)"}


def time_bvh_refit(pipe, flush, stream, steps):
    """The headline mesh's BVH built from scratch and refitted (bounds only, same
    triangles): CUDA events around each call, L2 flushed before each."""
    import torch

    out = {}
    for name, fn in (("build_ms", lambda: pipe.bvh.build(pipe.verts, pipe.tris, stream)),
                     ("refit_ms", lambda: pipe.bvh.refit(pipe.verts, pipe.tris, stream))):
        ms = []
        for k in range(steps + 3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            flush.zero_()
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                ms.append(ev[0].elapsed_time(ev[1]))
        out[name] = round(float(np.mean(ms)), 4)
    out["note"] = "refit keeps the leaf order and hierarchy of the last build (vertices moved, same triangles)"
    return out


def time_shadow_edge_grad(pipe, flush, stream, steps, samples_per_pixel=16):
    """The shadow-visibility gradient (edge sampling of the blocked set's
    boundary; off in the timed step, as in the paper's main results) on the
    headline G-buffer: the edge-table build and one gradient pass with
    `samples_per_pixel` edge samples, CUDA events around each, L2 flushed
    before each; plus the fraction of edge samples that land on a visible
    silhouette (uniform edge choice over the whole mesh)."""
    import torch

    from paper_2206_03380_gb300 import mcdi

    sc = pipe.scene
    prm = mcdi.make_params(sc.n_light, sc.n_cos, sc.n_ggx, sc.seed, tau=1.0)
    et = mcdi.EdgeTable.allocate(sc.tris.shape[0], pipe.device)
    ones = torch.ones_like(pipe.kd_out)
    g = torch.zeros_like(pipe.verts)
    M = samples_per_pixel
    w = torch.empty(pipe.N * pipe.H * pipe.W, M, device=pipe.device)
    out = {}
    for name, fn in (("edge_table_ms", lambda: et.build(pipe.tris, stream)),
                     ("grad_ms", lambda: mcdi.shadow_edge_grad(pipe.bvh, pipe.verts, et, pipe.probe, pipe.gb,
                                                               pipe.cams, prm, M, ones, ones, g, None,
                                                               stream=stream))):
        ms = []
        for k in range(steps + 3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            flush.zero_()
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                ms.append(ev[0].elapsed_time(ev[1]))
        out[name] = round(float(np.mean(ms)), 4)
    mcdi.shadow_edge_grad(pipe.bvh, pipe.verts, et, pipe.probe, pipe.gb, pipe.cams, prm, M, ones, ones, g, w,
                          stream=stream)
    torch.cuda.synchronize()
    out.update({"edge_samples_per_pixel": M, "edges": int(et.count.item()),
                "contributing_fraction": round(float((w != 0).float().mean().item()), 6),
                "launches": {"edge_table": 6, "grad": 1},
                "note": "not part of the timed step (the paper leaves shadow-visibility gradients off by default)"})
    return out


def time_denoiser_e4m3(pipe, den_params, conv_flops, flush, stream, steps):
    """The FP8 (E4M3, per-tensor scaling) denoiser on the same two 512^2 terms:
    forward and input-gradient times (CUDA events, L2 flushed before each pass);
    its error against the float64 network is a test result, not timed here."""
    import torch

    from paper_2206_03380_gb300 import mcdi

    den = mcdi.Denoiser(den_params, 2 * pipe.N, pipe.H, pipe.W, device=pipe.device, precision=mcdi.E4M3)
    y = torch.empty_like(pipe.denoised)
    gx = torch.empty_like(pipe.denoised)
    g = torch.ones_like(pipe.denoised)
    fwd, bwd = [], []
    for k in range(steps + 3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        flush.zero_()
        ev[0].record(stream)
        den.forward(pipe.terms, pipe.kd_out, pipe.gb.nrm, y, stream)
        ev[1].record(stream)
        den.backward(g, gx, stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[1].elapsed_time(ev[2]))
    if den.err.item() != 0:
        raise RuntimeError("E4M3 denoiser pipeline wait timed out")
    f, b = float(np.mean(fwd)), float(np.mean(bwd))
    peak, how = fp8_peak(stream)
    out = {"fwd_ms": round(f, 4), "bwd_ms": round(b, 4), "fwd_tflops": round(conv_flops / (f * 1e-3) / 1e12, 2),
           "bwd_tflops": round(conv_flops / (b * 1e-3) / 1e12, 2), "e4m3_peak_tflops": peak, "peak_source": how,
           "note": "E4M3 operands with per-tensor scaling (amax folded into each producer, quantised copy before each "
                   "convolution)"}
    if peak:
        out["fwd_frac"] = round(conv_flops / (f * 1e-3) / 1e12 / peak, 4)
        out["bwd_frac"] = round(conv_flops / (b * 1e-3) / 1e12 / peak, 4)
    return out


def time_denoiser_wgrad(den, conv_flops, flush, stream, steps):
    """The denoiser's weight gradient (the live-trained variant, App. B; not part of the timed
    step, whose denoiser weights are locked) after the step's forward and input gradient: 15
    tcgen05 weight-gradient launches and 15 deterministic reductions, CUDA events, L2 flushed
    before each pass.  FLOPs: the forward's (2 * 9 * c_in * c_out per pixel and convolution)."""
    import torch

    gw = den.weight_grad(stream=stream)
    ts = []
    for k in range(steps + 3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        flush.zero_()
        ev[0].record(stream)
        den.weight_grad(gw, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            ts.append(ev[0].elapsed_time(ev[1]))
    if den.err.item() != 0:
        raise RuntimeError("denoiser weight-gradient wait timed out")
    t = float(np.mean(ts))
    tpeak, tkind = tensor_peak()
    tf = conv_flops / (t * 1e-3) / 1e12
    return {"ms": round(t, 4), "tflops": round(tf, 2), "peak": tpeak, "frac": round(tf / tpeak, 4),
            "peak_source": tkind, "launches": 30, "finite": bool(torch.isfinite(gw).all().item()),
            "note": "dW and db of the 15 convolutions for the step's loss; off the timed step (locked weights)"}


def run_wgrad_only(args):
    """Only the denoiser weight gradient at the headline launch (2 images of 512^2, seeded
    synthetic terms and guides): one forward and input gradient, then the timed weight
    gradients.  A profiling entry that skips the rest of the benchmark."""
    import torch

    from paper_2206_03380_gb300 import mcdi, scenes

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(scenes.BASE_SEED + 11)
    H = W = 512
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
    term = t(np.abs(rng.lognormal(0.0, 0.8, size=(2, H, W, 4))))
    kd, nrm = t(rng.uniform(0, 1, size=(1, H, W, 4))), t(rng.normal(size=(1, H, W, 4)))
    den = mcdi.Denoiser(mcdi.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3)), 2, H, W,
                        device=dev)
    y, gx = torch.empty_like(term), torch.empty_like(term)
    den.forward(term, kd, nrm, y)
    den.backward(t(rng.normal(size=(2, H, W, 4))), gx)
    conv_flops = 0
    for name, ci, co in scenes.UNET_SHAPES:
        lvl = {"enc1": 0, "enc2": 1, "enc3": 2, "bot_": 3, "dec3": 2, "dec2": 1, "dec1": 0, "out": 0}[name[:4]]
        conv_flops += 2 * 9 * ci * co * 2 * (H >> lvl) * (W >> lvl)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    out = time_denoiser_wgrad(den, conv_flops, flush, torch.cuda.current_stream(), args.steps)
    print(json.dumps({"denoiser_wgrad": out, "config": {"images": 2, "width": W, "height": H}}))


def fp8_peak(stream, n=8192, reps=10):
    """Dense E4M3 peak measured with the vendor library (torch._scaled_mm, FP32 accumulation,
    per-tensor scales, BF16 output) on an n x n x n product, best of reps: the denominator of the
    E4M3 denoiser's tensor fraction.  A measurement aid only; the denoiser never calls it."""
    import torch

    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return round(2.0 * n ** 3 / (best * 1e-3) / 1e12, 1), f"measured (torch._scaled_mm e4m3 {n}^3, best of {reps})"
    except Exception as e:  # the library path may be missing on some builds
        return None, f"unavailable: {type(e).__name__}: {str(e)[:80]}"


def run_serving(n_requests, rate, dev, rank):
    """Poisson stream of render requests (resolution side uniform over multiples of
    32 in [128, 1024], spp uniform in {4, 8, 16, 32, 64}, 16 resident scenes and 16
    probes) served with continuous batching and one at a time; p50/p99 latency."""
    from paper_2206_03380_gb300 import mcdi, scenes
    from paper_2206_03380_gb300.serving import ServingEngine

    sc = scenes.serving_scenes(n_scenes=16)
    pr = scenes.serving_probes(n_probes=16)
    den = mcdi.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3))
    eng = ServingEngine(sc, pr, den, n_slots=4, hbm_budget=24 << 30, device=dev)
    reqs = scenes.poisson_requests(n_requests, rate, len(sc), len(pr), seed=scenes.BASE_SEED + 7 + rank)
    eng.run(scenes.poisson_requests(64, 1e4, len(sc), len(pr), seed=1), mode="continuous")  # warm-up
    out = {"requests": n_requests, "rate_per_s": rate,
           "triangles": [int(s["tris"].shape[0]) for s in sc[:4]],
           "offered_msamples_per_s": round(rate * float(np.mean([q.res * q.res * q.spp for q in reqs])) / 1e6, 1)}
    keys = ("p50_ms", "p99_ms", "mean_ms", "req_per_s", "msamples_per_s", "wall_s")
    for mode in ("continuous", "serial"):
        r = eng.run(reqs, mode=mode, lanes=SERVING_LANES if mode == "continuous" else None)
        out[mode] = {k: round(r[k], 3) for k in keys}
        out[mode]["admission_waits"] = r["admission_waits"]
    # the same kind of stream arriving twice as fast (half as many requests)
    fast = scenes.poisson_requests(n_requests // 2, 2 * rate, len(sc), len(pr), seed=scenes.BASE_SEED + 7 + rank)
    out["at_2x_rate"] = {mode: {k: round(v, 3) for k, v in
                                eng.run(fast, mode=mode, lanes=SERVING_LANES if mode == "continuous" else None).items()
                                if k in keys} for mode in ("continuous", "serial")}
    out["slots"] = eng.n_slots
    out["lanes"] = list(SERVING_LANES)
    out["design"] = ("two size lanes (fewer than 2M samples / the rest), each FIFO on its own slot, the large-request "
                     "lane's stream at the higher priority; per-slot buffers allocated once at the largest size; the "
                     "denoiser and composite of each request replayed from one CUDA graph per (side, slot) captured "
                     f"at start-up ({len(eng.sides) * eng.n_slots} graphs); raster and shading launched per request "
                     "(scene- and probe-dependent pointers)")
    return out


# ------------------------------------------------------------------ CPU oracle arm
def oracle_step(orc, sc, pix, tables=None):
    """One bounded oracle pass: probe tables, G-buffer rows, forward with records, adjoint."""
    cond, marg, _, tot = orc.envmap_cdf(sc.env)
    c32, m32 = cond.astype(np.float32), marg.astype(np.float32)
    W, H = sc.width, sc.height
    gb = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[0], W, H, pix, sc.tex_kd, sc.tex_korm, sc.uvmap)
    keep = gb[:, 3] > 0
    rows = gb[keep].astype(np.float32)
    p = pix[keep]
    cam = np.tile(sc.cams[0, :3].astype(np.float64), (len(p), 1))
    ctr = np.stack([p, np.zeros(len(p))], 1).astype(np.uint32)
    out, vis, recs = orc.shade_fwd(sc.verts, sc.tris, sc.env, c32, m32, tot, rows, cam, ctr, n_light=sc.n_light,
                                   n_cos=sc.n_cos, n_ggx=sc.n_ggx, seed=sc.seed, tau=1.0)
    g = np.ones((len(p), 9))
    orc.frozen_adjoint(recs, orc.param_rows(rows), cam, out[:, 9].astype(np.int32),
                       sc.env[..., :3].reshape(-1, 3).astype(np.float64), g)
    return len(p) * sc.spp


def oracle_pixel_sample(sc, n_pix, salt=0):
    rng = np.random.default_rng(1234 + salt)
    return np.sort(rng.choice(sc.width * sc.height, size=n_pix, replace=False)).astype(np.int32)


def omp_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(sc, n_pix=8192):
    import oracle

    orc = oracle
    orc.load()
    pix = oracle_pixel_sample(sc, n_pix)
    t0 = time.perf_counter()
    samples = oracle_step(orc, sc, pix)
    dt = time.perf_counter() - t0
    return {"value": round(samples / dt / 1e6, 6), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
            "sample": f"{n_pix} seeded pixels ({samples} covered-pixel samples) of the same view: probe tables, "
                      f"G-buffer rows, forward with brute-force visibility over all {sc.tris.shape[0]} triangles, "
                      f"adjoint", "seconds": round(dt, 2)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle

    from paper_2206_03380_gb300 import scenes

    sc = scenes.sphere_union_scene()
    oracle.load()
    for k in range(args.warmup):
        oracle_step(oracle, sc, oracle_pixel_sample(sc, 8, salt=100 + k))
    times, samples = [], 0
    t_all = time.perf_counter()
    for k in range(args.steps):
        pix = oracle_pixel_sample(sc, args.ref_pixels, salt=k)
        t0 = time.perf_counter()
        samples += oracle_step(oracle, sc, pix)
        times.append(time.perf_counter() - t0)
    total = time.perf_counter() - t_all
    value = samples / sum(times) / 1e6
    cb = {"value": round(value, 6), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
          "sample": f"{args.ref_pixels} seeded pixels per step of the {sc.name} workload (brute-force visibility "
                    f"over all triangles, FP64)"}
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sc.name, "pixels_per_step": args.ref_pixels, "spp": sc.spp,
                       "triangles": int(sc.tris.shape[0])},
            "cpu_baseline": cb, "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}, "wall_s": round(total, 2)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mcdi", choices=["mcdi", "reference"])
    ap.add_argument("--cpu-pixels", type=int, default=8192)
    ap.add_argument("--ref-pixels", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="graph replays of the 8-view 800^2 32-spp step on the ~1.3M-triangle mesh (0: skip)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the optimisation-step batch and print its figures (a profiling aid)")
    ap.add_argument("--wgrad-only", action="store_true",
                    help="run only the denoiser weight gradient at the headline launch (a profiling aid)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.wgrad_only:
        run_wgrad_only(args)
        return
    if args.batch_only:
        import torch

        rank, world = init_dist("nccl" if torch.cuda.is_available() else "gloo")
        torch.cuda.set_device(dist_env()[2])
        dev = torch.device("cuda", dist_env()[2])
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        res = {"step_batch": run_step_batch(max(args.batch_steps, 1), flush, dev, rank, world)}
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    if args.impl == "reference":
        rank, world = init_dist("gloo")
        res = run_reference(args, rank, world)
    else:
        import torch

        rank, world = init_dist("nccl" if torch.cuda.is_available() else "gloo")
        res = run_gpu(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
