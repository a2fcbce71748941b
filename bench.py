#!/usr/bin/env python3
"""fwd+bwd Mpixel/s of the GB300 textured 2D-Gaussian rasterizer.

Workload (default): 1,000,000 splats (80 % on 6 planes, 20 % clutter in a
10^3 box), SH degree 3 and N x N RGB textures stored in FP16, 16 cameras on a
radius-6 sphere at 960x540 / 1280x720 / 1920x1080 (18,086,400 pixels), all
views rendered in one batched forward + backward per step.  Beside it, the
same 16 views one by one on the plain FP32 path (FP32 texture/SH storage).

A step is one forward + backward of all views with inputs resident in HBM
(they exceed the 129 MB L2, so no flush is needed between steps).  Prints one
JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on a
bounded crop of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpixel/s at 1M textured splats, batched vs plain FP32, max err vs FP64"
FP32_PEAK_TFLOPS_AT_MAX = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs, FMA = 2 FLOP, 2070 MHz (no clock sample)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_1m")
    ap.add_argument("--tex-n", type=int, default=4)
    ap.add_argument("--views", type=int, default=0, help="use only the first V cameras (0 = all; profiling)")
    ap.add_argument("--batch", type=int, default=0, help="splats per shared-memory batch (0 = auto)")
    ap.add_argument("--batch-fwd", type=int, default=0,
                    help="the forward's batch depth (0 = --batch, or automatic when that is 0 too)")
    ap.add_argument("--tile", type=int, default=0, help="tile edge 8, 16 or 32 (0 = autotune)")
    ap.add_argument("--ppt", type=int, default=0,
                    help="pixel-parallel backward with 1 or 2 pixels per thread (0 = automatic)")
    ap.add_argument("--bwd-kernel", type=int, default=0,
                    help="backward loop: 0 automatic, 1 pixel-parallel, 2 splat-parallel")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--crop", type=int, default=0, help="oracle crop side in pixels (0 = all of camera 0)")
    ap.add_argument("--mip", type=int, default=0, help="render the grids at this mip level (box filter)")
    ap.add_argument("--tex-sh", type=int, default=0, help="per-texel SH degree of the grids (0 = RGB texels)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations (8x8 grids, persistent launch, training step, multi-scene)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ helpers --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    """Max of x over the ranks (on the GPU under NCCL, on the host under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(pixels_per_rank: int, ms: float, world: int):
    """Whole-job throughput of replicas: every rank renders its own copy of the
    workload (no data-path collective); the job takes the slowest rank's time.
    Returns (ms_max, Mpixel/s over all ranks)."""
    ms_max = allreduce_max(ms, world)
    return ms_max, world * pixels_per_rank / (ms_max / 1e3) / 1e6


def make_workload(args):
    from paper_2412_12734_gb300 import scenes
    wl = scenes.workload(args.workload, seed=0, tex_n=args.tex_n)
    if getattr(args, "mip", 0):
        wl["scenes"] = [dict(sc, mip_level=args.mip) for sc in wl["scenes"]]
    if getattr(args, "tex_sh", 0):
        wl["scenes"] = [scenes.with_texel_sh(sc, args.tex_sh) for sc in wl["scenes"]]
    if args.views:
        for k in ("cams", "cam_scene", "d_rgb"):
            wl[k] = wl[k][:args.views]
    return wl


STORAGE_NAMES = {"f32": "FP32", "f16": "FP16", "bf16": "BF16"}


def workload_label(args, wl) -> str:
    """config.workload of both arms: the workload's name, splats, views and storage."""
    sc = wl["scenes"][0]
    sizes = sorted({(int(c["width"]), int(c["height"])) for c in wl["cams"]}, key=lambda s: s[0] * s[1])
    return (f"{args.workload}: {int(sc['means'].shape[0]):,} splats, {len(wl['cams'])} views "
            f"{'/'.join(f'{w}x{h}' for w, h in sizes)}, {args.tex_n}x{args.tex_n} "
            f"{STORAGE_NAMES[sc.get('tex_dtype', 'f32')]} textures, SH{int(sc['sh_degree'])} "
            f"{STORAGE_NAMES[sc.get('sh_dtype', 'f32')]}")


def crop_window(cam, side):
    W, H = int(cam["width"]), int(cam["height"])
    if side <= 0:
        return (0, 0, W, H)
    w, h = min(side, W), min(side, H)
    return ((W - w) // 2, (H - h) // 2, w, h)


# ------------------------------------------------------------- CPU oracle --

def oracle_sample(wl, crop: int):
    """Oracle fwd+bwd on a centred crop of camera 0: (seconds, pixels, outputs)."""
    import oracle
    sc, cam = wl["scenes"][0], wl["cams"][0]
    win = crop_window(cam, crop)
    x0, y0, w, h = win
    d = wl["d_rgb"][0][y0:y0 + h, x0:x0 + w]
    t0 = time.perf_counter()
    ref = oracle.render(sc, cam, window=win, prefilter=True)
    # upstream gradient zeroed at pixels within 1e-4 of a decision threshold
    d = d * (ref["margin_grad"] > 1e-4)[..., None]
    ref["grads"] = oracle.backward(sc, cam, d, window=win, prefilter=True)
    dt = time.perf_counter() - t0
    ref["d_rgb"] = d
    return dt, w * h, ref, win


# ----------------------------------------------------------- reference arm --

def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    wl = make_workload(args)
    oracle.build()
    times = []
    px = 0
    for i in range(args.warmup + args.steps):
        dt, px, _, win = oracle_sample(wl, args.crop)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = px / (ms / 1e3) / 1e6
    cores = oracle.num_threads()
    sample = (f"{win[2]}x{win[3]} window of camera 0 ({wl['cams'][0]['width']}x{wl['cams'][0]['height']}) "
              f"of the {args.workload} workload, fwd+bwd, bbox-prefiltered FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_label(args, wl), "tex_n": args.tex_n, "crop": args.crop,
                   "mip_level": args.mip, "tex_sh_degree": args.tex_sh},
        "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm --

def run_ours(args, world, rank, local):
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import build as B
    from paper_2412_12734_gb300 import render as R

    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    barrier(world)
    lib = L.load()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    wl = make_workload(args)
    cams = wl["cams"]
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    dev_scene = R.scene_to_device(wl["scenes"][0])
    d_rgb = torch.as_tensor(np.concatenate([d.reshape(-1, 3) for d in wl["d_rgb"]]), device="cuda")
    rast = R.Rasterizer(local)

    # --- tile size and batch depth: explicit, or from the library's autotuner
    tune = None
    if args.tile == 0:
        tune = tune_frame(rast, [dev_scene], cams)
        args.tile, args.batch, args.ppt = tune["tile"], tune["batch"], tune["ppt"]
        args.batch_fwd = tune.get("batch_fwd", 0)
        args.bwd_kernel = tune.get("bwd_kernel", 0)
    opts = {"tile": args.tile, "batch": args.batch, "batch_fwd": args.batch_fwd, "ppt": args.ppt,
            "bwd_kernel": args.bwd_kernel}

    run = BatchedStep(rast, torch, R, L, [dev_scene], cams, None, d_rgb, opts)
    head = run.time(args, world, lib, sample_clocks=local, graph=not args.no_graph)
    ms_max, value = aggregate(P, head["ms"], world)
    phases, pairs = run.phase_times(args)
    dominant = max(phases, key=phases.get)
    roofline = roofline_line(dominant, phases, pairs, head["clocks"], measured_traffic(dominant, args), sms=sms)
    rgb, depth, alpha = run.out

    result = {
        "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(args, wl),
                   "pixels_per_step": P, "tex_n": args.tex_n, "mip_level": args.mip, "tex_sh_degree": args.tex_sh,
                   "storage": "f16", "tile": args.tile,
                   "batch_depth": args.batch, "batch_depth_fwd": args.batch_fwd or args.batch,
                   "pixels_per_thread": args.ppt, "bwd_kernel": args.bwd_kernel, "autotune": tune,
                   "graph": not args.no_graph, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "clocks": head["clocks"], "gpu_launches": int(head["launches"]), "phases_ms": phases,
        "stats": {k: pairs[k] for k in ("visible", "instances", "pairs_fwd", "pairs_bwd", "blended_fwd",
                                        "contributing_bwd", "records")},
        "roofline": roofline,
    }

    # --- the same frame with persistent render blocks (one launch per pass, tiles from a counter)
    if not args.no_extra:
        prun = BatchedStep(rast, torch, R, L, [dev_scene], cams, None, d_rgb, opts, flags=L.GB_FLAG_PERSISTENT)
        pt = prun.time(args, world, lib, graph=not args.no_graph)
        result["persistent"] = {"value": aggregate(P, pt["ms"], world)[1], "unit": "Mpixel/s", "ms_per_step": pt["ms"],
                                "note": "GB_FLAG_PERSISTENT: render blocks pull tiles from a device counter, longest "
                                        "tiles first; same frame and options as the headline"}
        del prun

    # --- plain FP32 path: the same views one by one
    if not args.no_plain:
        result["plain_fp32"] = plain_fp32(args, wl, rast, R, L, torch)

    # --- e2e through host buffers
    if not args.no_e2e:
        result["e2e"] = e2e(args, wl, rast, R, L, torch, cams, P)

    # --- CPU oracle baseline + max error vs FP64 (rank 0)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"], result["max_err_vs_fp64"] = cpu_baseline(args, wl, rgb, alpha, depth, cams,
                                                                          rast, dev_scene)
    del run, dev_scene, d_rgb

    # --- the rest of the benchmark configurations, timed the same way
    if not args.no_extra and args.workload == "batched_1m" and not (args.mip or args.tex_sh or args.views):
        if args.tex_n == 4:
            result["per_tex_n"] = {"8": other_tex_n(args, world, rast, torch, R, L, lib, 8, sms)}
        result["train_3m"] = train_step(args, world, rast, torch, R, L, lib)
        result["multi_scene"] = multi_scene(args, world, rast, torch, R, L, lib)

    if rank == 0:
        print(json.dumps(result), flush=True)
    barrier(world)
    return 0


def tune_frame(rast, scenes, cams, cam_scene=None):
    return rast.autotune(scenes, cams, cam_scene=cam_scene, reps=2,
                         cache=os.path.join(tempfile.gettempdir(), f"gbill_tune_{os.getpid()}.json"))


class BatchedStep:
    """One forward + backward of a frame on a saved state reserved from a
    synchronizing forward, then run without host synchronization; ``post``
    (optional) runs after each backward outside the captured graph (an
    optimiser step whose step count changes)."""

    def __init__(self, rast, torch, R, L, scenes, cams, cam_scene, d_rgb, opts, flags=0, post=None):
        self.rast, self.torch, self.R, self.L = rast, torch, R, L
        self.scenes, self.cams, self.cam_scene = scenes, cams, cam_scene
        self.d_rgb, self.opts, self.flags, self.post = d_rgb, opts, flags, post
        self.P = sum(int(c["width"]) * int(c["height"]) for c in cams)
        self.saved = R.Saved(rast)
        rgb, depth, alpha, _ = rast.forward(scenes, cams, cam_scene=cam_scene, saved=self.saved, flags=flags, **opts)
        st0 = self.saved.stats()
        self.saved.reserve(st0["records"], int(st0["instances"] * 1.1) + 4096, self.P, st0["tiles"])
        self.grads = rast.backward(self.saved, d_rgb)
        self.out = (rgb, depth, alpha)
        self.graph = None
        self.n_post = 0

    def step(self, extra_flags=0):
        L = self.L
        self.rast.forward(self.scenes, self.cams, cam_scene=self.cam_scene, saved=self.saved,
                          flags=self.flags | L.GB_FLAG_NO_SYNC | extra_flags, out=self.out, **self.opts)
        self.rast.backward(self.saved, self.d_rgb, grads=self.grads)

    def replay(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.step()
        if self.post is not None:
            self.n_post += 1
            self.post(self.n_post)

    def time(self, args, world, lib, sample_clocks=None, graph=True):
        """Mean ms per step over args.steps after args.warmup, CUDA events on the
        launch stream, barrier and synchronize on both sides; clocks sampled
        during the timed region when sample_clocks is a device index."""
        torch = self.torch
        for _ in range(args.warmup):
            self.replay()
        torch.cuda.synchronize()
        self.saved.check()
        if graph and self.graph is None:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.step()
            self.graph = g
            self.replay()
            torch.cuda.synchronize()
            self.saved.check()
        per_step = launches_per_step(lib, self.step)
        sampler = ClockSampler(sample_clocks) if sample_clocks is not None else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            self.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clocks = sampler.stop() if sampler else None
        self.saved.check()
        return {"ms": e0.elapsed_time(e1) / args.steps, "clocks": clocks,
                "launches": args.steps * (per_step + (1 if self.post is not None else 0))}

    def phase_times(self, args):
        """Per-phase ms (library events, GB_FLAG_TIMING) over args.steps eager steps, and the counters."""
        acc = {}
        st = None
        for _ in range(args.steps):
            self.step(self.L.GB_FLAG_TIMING)
            for k, v in self.saved.phase_times().items():
                acc.setdefault(k, []).append(v)
            st = self.saved.stats()
        return {k: sum(v) / len(v) for k, v in acc.items()}, st


def other_tex_n(args, world, rast, torch, R, L, lib, tex_n, sms):
    """The headline frame with N x N grids of another size, tuned and timed the same way."""
    from paper_2412_12734_gb300 import scenes
    wl = scenes.workload(args.workload, seed=0, tex_n=tex_n)
    cams = wl["cams"]
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    dev = R.scene_to_device(wl["scenes"][0])
    d = torch.as_tensor(np.concatenate([x.reshape(-1, 3) for x in wl["d_rgb"]]), device="cuda")
    tune = tune_frame(rast, [dev], cams)
    opts = {"tile": tune["tile"], "batch": tune["batch"], "batch_fwd": tune.get("batch_fwd", 0), "ppt": tune["ppt"],
            "bwd_kernel": tune.get("bwd_kernel", 0)}
    run = BatchedStep(rast, torch, R, L, [dev], cams, None, d, opts)
    t = run.time(args, world, lib, sample_clocks=torch.cuda.current_device(), graph=not args.no_graph)
    phases, st = run.phase_times(args)
    dominant = max(phases, key=phases.get)
    return {"value": aggregate(P, t["ms"], world)[1], "unit": "Mpixel/s", "ms_per_step": t["ms"],
            "workload": workload_label(argparse.Namespace(**dict(vars(args), tex_n=tex_n)), wl),
            "options": {k: v for k, v in opts.items()}, "clocks": t["clocks"], "phases_ms": phases,
            "gpu_launches": int(t["launches"]),
            "roofline": roofline_line(dominant, phases, st, t["clocks"], sms=sms)}


def train_step(args, world, rast, torch, R, L, lib):
    """The training-step shape: 3,000,000 splats with BF16 SH (degree 3) and
    8 x 8 BF16 grids, 8 views at 1600 x 1067; a step is the forward, the
    backward and one fused Adam launch over every parameter tensor (FP32
    masters and moments; the kernel writes the BF16 copies the renderer
    reads)."""
    from paper_2412_12734_gb300 import scenes
    wl = scenes.workload("train_3m")
    sc, cams = wl["scenes"][0], wl["cams"]
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    dev = R.scene_to_device(sc)
    names = ("means", "quats", "scales", "opacities", "sh", "textures")
    master = {k: dev[k].float().clone() for k in names}
    # the renderer reads the FP32 masters of the geometry and the BF16 copies of SH and grids
    for k in ("means", "quats", "scales", "opacities"):
        dev[k] = master[k]
    d = torch.as_tensor(np.concatenate([x.reshape(-1, 3) for x in wl["d_rgb"]]), device="cuda") * 1e-3
    tune = tune_frame(rast, [dev], cams)
    opts = {"tile": tune["tile"], "batch": tune["batch"], "batch_fwd": tune.get("batch_fwd", 0), "ppt": tune["ppt"],
            "bwd_kernel": tune.get("bwd_kernel", 0)}
    run = BatchedStep(rast, torch, R, L, [dev], cams, None, d, opts)
    m = {k: torch.zeros_like(master[k]) for k in names}
    v = {k: torch.zeros_like(master[k]) for k in names}
    adam = R.AdamStep(rast, [master[k] for k in names], [run.grads[0][k] for k in names], [m[k] for k in names],
                      [v[k] for k in names], lr=1e-4, betas=(0.9, 0.999), eps=1e-15,
                      shadows=[None, None, None, None, dev["sh"], dev["textures"]])
    run.post = adam
    t = run.time(args, world, lib, graph=not args.no_graph)
    n_params = sum(master[k].numel() for k in names)
    return {"value": aggregate(P, t["ms"], world)[1], "unit": "Mpixel/s", "ms_per_step": t["ms"],
            "params_per_step": int(n_params), "gpu_launches": int(t["launches"]),
            "workload": f"train_3m: 3,000,000 splats, 8 views 1600x1067, 8x8 BF16 grids, SH3 BF16, fused Adam",
            "options": opts,
            "note": "forward + backward from one CUDA graph, then one fused Adam launch (step count advances); "
                    "parameters change every step, so the visible set and instance list are rebuilt each step"}


def multi_scene(args, world, rast, torch, R, L, lib):
    """Twelve scenes (10k-2M splats, 2/4/8 grids, FP16) with 1-4 views each
    rendered forward + backward in one persistent launch sequence per pass,
    against the same scenes one at a time on the plain FP32 path."""
    from paper_2412_12734_gb300 import scenes
    wl = scenes.workload("multi_scene")
    sl, cams, cs = wl["scenes"], wl["cams"], wl["cam_scene"]
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    dev = [R.scene_to_device(s) for s in sl]
    d = torch.as_tensor(np.concatenate([x.reshape(-1, 3) for x in wl["d_rgb"]]), device="cuda")
    tune = tune_frame(rast, dev, cams, cam_scene=cs)
    opts = {"tile": tune["tile"], "batch": tune["batch"], "batch_fwd": tune.get("batch_fwd", 0), "ppt": tune["ppt"],
            "bwd_kernel": tune.get("bwd_kernel", 0)}
    run = BatchedStep(rast, torch, R, L, dev, cams, cs, d, opts, flags=L.GB_FLAG_PERSISTENT)
    t = run.time(args, world, lib, graph=not args.no_graph)
    batched = {"value": aggregate(P, t["ms"], world)[1], "ms_per_step": t["ms"], "options": opts,
               "gpu_launches": int(t["launches"])}
    del run
    # one by one, FP32 storage, each scene's views in one call
    off = np.cumsum([0] + [int(c["width"]) * int(c["height"]) for c in cams])
    runs = []
    for s_i, s in enumerate(sl):
        mine = [i for i in range(len(cams)) if cs[i] == s_i]
        s32 = dict(s, sh_dtype="f32", tex_dtype="f32")
        d32 = R.scene_to_device(s32)
        ds = torch.cat([d[off[i]:off[i + 1]] for i in mine]).contiguous()
        runs.append(BatchedStep(rast, torch, R, L, [d32], [cams[i] for i in mine], None, ds, {"tile": 16}))
    for r in runs:
        for _ in range(args.warmup):
            r.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        for r in runs:
            r.step()
    e1.record()
    torch.cuda.synchronize()
    for r in runs:
        r.saved.check()
    ms1 = e0.elapsed_time(e1) / args.steps
    return {"unit": "Mpixel/s", "pixels_per_step": int(P), "views": len(cams),
            "splats": int(sum(int(s["means"].shape[0]) for s in sl)),
            "batched_persistent": batched,
            "one_by_one_fp32": {"value": aggregate(P, ms1, world)[1], "ms_per_step": ms1,
                                "note": "each scene alone (its views in one call), FP32 storage, tile 16, "
                                        "automatic batch depths, eager launches"}}


def launches_per_step(lib, step):
    import torch
    a = lib.gb_kernel_launches()
    step()
    torch.cuda.synchronize()
    return lib.gb_kernel_launches() - a


# DRAM bytes (read + write) per launch of the render kernels on the full
# 16-view batched_1m workload at 4x4 grids, from ncu captures
# (profiles/render_traffic_batched_1m.md), per launch configuration, with the
# digest of the kernel sources they were taken on.  A kernel whose sources
# differ, or a configuration not captured, reports traffic null.
TRAFFIC = {
    "render_bwd": {"files": ("render_bwd.cuh", "render_common.cuh", "render_bwd.cu", "render_bwd2.cu"),
                   "sha256_16": "fa8633142f80a770", "keys": ("workload", "tex_n", "tile", "batch", "ppt"),
                   "measured": [({"workload": "batched_1m", "tex_n": 4, "tile": 16, "batch": 184, "ppt": 1},
                                 3.5810e9 + 0.9574e9)]},
    "render_fwd": {"files": ("render_fwd.cu", "render_common.cuh"),
                   "sha256_16": "ad0d74dbf8af3db0", "keys": ("workload", "tex_n", "tile", "batch_fwd"),
                   "measured": [({"workload": "batched_1m", "tex_n": 4, "tile": 16, "batch_fwd": 88},
                                 1.8515e9 + 0.4984e9)]},
}


def measured_traffic(kernel, args):
    """Bytes per launch from TRAFFIC when the kernel sources and the launch
    configuration are ones it was measured on, else None."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None or args.views or args.mip or args.tex_sh:
        return None
    h = hashlib.sha256()
    for f in t["files"]:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2412_12734_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != t["sha256_16"]:
        return None
    cfg = {"workload": args.workload, "tex_n": args.tex_n, "tile": args.tile, "batch": args.batch, "ppt": args.ppt,
           "batch_fwd": args.batch_fwd or args.batch}
    cfg = {k: cfg[k] for k in t["keys"]}
    for c, b in t["measured"]:
        if c == cfg:
            return b
    return None


def roofline_line(dominant, phases, st, clocks, traffic=None, sms=152):
    """ALU roofline of the dominant kernel: algorithmic FLOPs per launch over
    its measured launch time, against the nominal FP32 FMA rate of the
    device (its SM count, as queried, x 128 FP32 lanes x 2 FLOP per FMA) at
    the median sampled SM clock.

    FLOPs per (pixel, splat) pair (FMA = 2), counted from the kernels' math:
    forward: 30 per evaluated pair (offset, intersection, rho, Gaussian, alpha
    test) + 61 per blended pair (bilinear 27, cell 16, blend 18); backward:
    30 per evaluated pair + 200 per contributing pair (colour 43, adjoints of
    alpha, Gaussian, intersection and record 130, adj-bilinear weights 27).
    Pair counts come from device counters of the same launches.
    """
    ms = phases[dominant]
    sm = (clocks or {}).get("sm_mhz") or 2070.0
    peak = sms * 128 * 2 * sm * 1e6 / 1e12
    if dominant == "render_bwd":
        flops = 30 * st["pairs_bwd"] + 200 * st["contributing_bwd"]
    elif dominant == "render_fwd":
        flops = 30 * st["pairs_fwd"] + 61 * st["blended_fwd"]
    else:
        flops = None
    achieved = flops / (ms / 1e3) / 1e12 if flops else None
    return {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "peak_source": f"nominal FP32 FMA rate: {sms} SMs (queried) x 128 lanes x 2 FLOP at the median "
                           f"sampled SM clock {sm:.0f} MHz",
            "launch_ms": ms}


def plain_fp32(args, wl, rast, R, L, torch):
    sc = dict(wl["scenes"][0])
    sc["sh_dtype"] = "f32"
    sc["tex_dtype"] = "f32"
    dev = R.scene_to_device(sc)
    cams = wl["cams"]
    d_views, outs, saveds, grads = [], [], [], []
    o = 0
    for c in cams:
        n = int(c["width"]) * int(c["height"])
        d_views.append(torch.as_tensor(wl["d_rgb"][len(d_views)].reshape(-1, 3), device="cuda"))
        outs.append((torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
                     torch.empty(n, device="cuda")))
        s = R.Saved(rast)
        rast.forward([dev], [c], saved=s, out=outs[-1])
        st = s.stats()
        s.reserve(st["records"], int(st["instances"] * 1.1) + 4096, n, st["tiles"])
        saveds.append(s)
        grads.append(rast.backward(s, d_views[-1]))
        o += n

    def step():
        for i, c in enumerate(cams):
            rast.forward([dev], [c], saved=saveds[i], flags=L.GB_FLAG_NO_SYNC, out=outs[i])
            rast.backward(saveds[i], d_views[i], grads=grads[i])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    for s in saveds:
        s.check()
    ms = e0.elapsed_time(e1) / args.steps
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    return {"value": P / (ms / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": ms,
            "note": "same 16 views rendered one by one, FP32 texture/SH storage, eager launches"}


def e2e(args, wl, rast, R, L, torch, cams, P):
    """Same metric through the C ABI with host buffers.  Every step copies the
    scene parameters and dL/drgb from pinned host memory, runs forward +
    backward and reads rgb and every gradient back to pinned host memory.
    As a user would run it: the saved state is reserved once so the forward
    never synchronizes (GB_FLAG_NO_SYNC), and inputs and outputs are double
    buffered so that step k+1's uploads and step k-1's downloads run on a copy
    stream while step k computes.  The timed region spans the first upload to
    the last download."""
    host = R.scene_to_device(wl["scenes"][0], device="cpu")
    keys = ("means", "quats", "scales", "opacities", "sh", "textures")
    meta = {k: host[k] for k in ("sh_degree", "tex_n", "sigma", "mip_level", "tex_sh_degree")}
    h_in = [{k: host[k].pin_memory() for k in keys} for _ in range(2)]
    drgb = torch.as_tensor(np.concatenate([d.reshape(-1, 3) for d in wl["d_rgb"]]))
    h_drgb = [drgb.pin_memory(), drgb.clone().pin_memory()]
    d_in = [{k: torch.empty_like(v, device="cuda") for k, v in h_in[0].items()} for _ in range(2)]
    d_drgb = [torch.empty_like(h_drgb[0], device="cuda") for _ in range(2)]
    comp = torch.cuda.Stream()
    copy = torch.cuda.Stream()
    saved = R.Saved(rast)
    for b in range(2):
        for k in keys:
            d_in[b][k].copy_(h_in[b][k])
        d_drgb[b].copy_(h_drgb[b])
    torch.cuda.synchronize()
    outs, grads = [], []
    for b in range(2):
        o = rast.forward([dict(d_in[b], **meta)], cams, saved=saved, batch=args.batch, batch_fwd=args.batch_fwd,
                         bwd_kernel=args.bwd_kernel,
                         tile=args.tile, ppt=args.ppt)
        outs.append(o[:3])
        grads.append(rast.backward(saved, d_drgb[b]))
    st = saved.stats()
    saved.reserve(st["records"], int(st["instances"] * 1.1) + 4096, P, st["tiles"])
    h_out = [{k: torch.empty_like(v, device="cpu").pin_memory() for k, v in grads[0][0].items()} for _ in range(2)]
    h_rgb = [torch.empty_like(outs[0][0], device="cpu").pin_memory() for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in h_in[0].values()) + h_drgb[0].numel() * 4
    d2h = sum(v.numel() * v.element_size() for v in h_out[0].values()) + h_rgb[0].numel() * 4
    torch.cuda.synchronize()
    done_in = [torch.cuda.Event(), torch.cuda.Event()]     # compute finished reading inputs[b]
    done_out = [torch.cuda.Event(), torch.cuda.Event()]    # downloads of outputs[b] finished
    uploaded = [torch.cuda.Event(), torch.cuda.Event()]
    computed = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(b):
        with torch.cuda.stream(copy):
            copy.wait_event(done_in[b])
            for k in keys:
                d_in[b][k].copy_(h_in[b][k], non_blocking=True)
            d_drgb[b].copy_(h_drgb[b], non_blocking=True)
            uploaded[b].record(copy)

    def compute(b):
        comp.wait_event(uploaded[b])
        comp.wait_event(done_out[b])
        rast.forward([dict(d_in[b], **meta)], cams, saved=saved, out=outs[b], flags=L.GB_FLAG_NO_SYNC,
                     batch=args.batch, batch_fwd=args.batch_fwd, tile=args.tile, ppt=args.ppt, stream=comp,
                     bwd_kernel=args.bwd_kernel)
        rast.backward(saved, d_drgb[b], grads=grads[b], stream=comp)
        done_in[b].record(comp)
        computed[b].record(comp)

    def download(b):
        with torch.cuda.stream(copy):
            copy.wait_event(computed[b])
            for k, v in grads[b][0].items():
                h_out[b][k].copy_(v, non_blocking=True)
            h_rgb[b].copy_(outs[b][0], non_blocking=True)
            done_out[b].record(copy)

    def run(n):
        upload(0)
        for i in range(n):
            b = i & 1
            if i + 1 < n:
                upload(1 - b)
            compute(b)
            download(b)

    for e in done_in + done_out:
        e.record(comp)
    run(args.warmup)
    torch.cuda.synchronize()
    saved.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(copy)
    comp.wait_event(e0)
    run(args.steps)
    e1.record(copy)  # after the last download, which waits for the last compute
    torch.cuda.synchronize()
    saved.check()
    ms = e0.elapsed_time(e1) / args.steps
    return {"value": P / (ms / 1e3) / 1e6, "unit": "Mpixel/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms,
            "note": "no-sync forward on a reserved saved state; uploads and downloads double buffered on a "
                    "copy stream, overlapping the neighbouring steps' compute"}


def grad_ratios(g_gpu, g_ref):
    """Worst |g - g*| / (1e-3 max(|g*|, 1e-3 max|g*|)) per tensor; <= 1 is within tolerance."""
    out = {}
    for k, ref in g_ref.items():
        a = g_gpu[k].detach().double().cpu().numpy().reshape(ref.shape)
        scale = np.abs(ref).max()
        den = 1e-3 * np.maximum(np.abs(ref), 1e-3 * scale) if scale > 0 else 1.0
        out[k] = float((np.abs(a - ref) / den).max())
    return out


def cpu_baseline(args, wl, rgb, alpha, depth, cams, rast, dev_scene):
    import torch

    import oracle
    oracle.build()
    dt, px, ref, win = oracle_sample(wl, args.crop)
    x0, y0, w, h = win
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    img = rgb[:W * H].reshape(H, W, 3)[y0:y0 + h, x0:x0 + w].cpu().numpy().astype(np.float64)
    a = alpha[:W * H].reshape(H, W)[y0:y0 + h, x0:x0 + w].cpu().numpy().astype(np.float64)
    dp = depth[:W * H].reshape(H, W)[y0:y0 + h, x0:x0 + w].cpu().numpy().astype(np.float64)
    mask = ref["margin_fwd"] > 1e-5
    err = np.abs(img - ref["rgb"]).max(axis=2)
    aerr = np.abs(a - ref["alpha"])
    derr = np.abs(dp - ref["depth"]) / np.maximum(1.0, np.abs(ref["depth"]))
    base = {"value": px / dt / 1e6, "unit": "Mpixel/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{w}x{h} crop of camera 0, fwd+bwd, FP64 bbox-prefiltered oracle, {dt:.1f} s"}

    def mx(x, m):
        return float(x[m].max()) if m.any() else 0.0
    errs = {"rgb": mx(err, mask), "alpha": mx(aerr, mask), "depth_rel": mx(derr, mask),
            "rgb_px_over_2e-5": int((mask & (err > 2e-5)).sum()),
            "excluded_px": int((~mask).sum()), "pixels": int(w * h),
            "storage": "errors are against the FP64 oracle on the stored FP16 values; depth relative to "
                       "max(1, |depth|); pixels within 1e-5 (relative) of a forward decision excluded"}
    # gradients of camera 0 alone (same masked upstream gradient) against the oracle's
    d_full = np.zeros((H, W, 3), np.float32)
    d_full[y0:y0 + h, x0:x0 + w] = ref["d_rgb"]
    s0 = rast.forward([dev_scene], cams[:1])[3]
    g = rast.backward(s0, torch.as_tensor(d_full.reshape(-1, 3), device="cuda"))[0]
    errs["grad_worst_ratio"] = grad_ratios(g, ref["grads"])
    errs["grad_tolerance"] = "per element |g-g*| <= 1e-3 max(|g*|, 1e-3 max|g*|); ratio <= 1 passes"
    return base, errs


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
