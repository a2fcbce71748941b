"""2D image fitting (Sec. 4.1) on the GPU library.

One camera looks down +z at an image plane; every splat faces the camera and
may only turn about the view axis.  The trainable parameters are raw: angle
theta, position xy in the splat's plane z (held fixed), log-scales, opacity
logit, the SH term (degree 0) and the colour grid.  One iteration is, all in
the library's kernels:

    gb_fit_params            raw -> activated parameters
    gb_render_forward        image
    gb_mse_loss              MSE against the target and dL/drgb
    gb_render_backward       gradients of the activated parameters, grid, SH
    gb_fit_params_backward   gradients of the raw parameters
    gb_adam_step             Adam (Kingma & Ba) per parameter group

The forward runs in no-sync mode on a saved state sized by one synchronizing
forward, so an iteration never waits for the host.  The steps up to the
raw-parameter gradients are captured once in a CUDA graph and replayed (an
iteration of a small fit is otherwise bound by the host's launch time); the
Adam launches, whose bias corrections change every iteration, follow the
replay with their argument arrays built once.  ``python -m
paper_2412_12734_gb300.fit2d --target wide --splats 1000`` fits a seeded
synthetic target (``scenes.fit_target``; the paper's photographs are not
part of this project).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import time

import numpy as np
import torch

from . import _lib as L
from . import render as R
from . import scenes

# learning rates per parameter group (the renderer's units: the image plane
# spans x in [-1/2, 1/2])
DEFAULT_LR = {"theta": 1e-2, "xy": 2e-4, "log_scales": 5e-3, "logit_opacities": 2e-2, "sh": 2.5e-3,
              "textures": 5e-3}
RAW = ("theta", "xy", "log_scales", "logit_opacities", "sh", "textures")


class ImageFit:
    """Fits K textured splats to a target image [H, W, 3] (float32 in [0, 1])."""

    def __init__(self, target: np.ndarray, K: int, tex_n: int = 4, seed: int = 0, lr: dict | None = None,
                 rasterizer: R.Rasterizer | None = None, device: int = 0, graph: bool = True):
        self.rast = rasterizer or R.Rasterizer(device)
        H, W = target.shape[:2]
        self.cam = scenes.fit_camera(W, H)
        self.P = W * H
        raw = scenes.fit_init(K, W, H, seed=seed, tex_n=tex_n)
        dev = f"cuda:{device}"
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev).contiguous()
        self.K, self.tex_n = K, tex_n
        self.sigma = float(raw["sigma"])
        self.p = {k: t(raw[k]) for k in RAW}
        self.z = t(raw["z"])
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.act = {"quats": torch.empty((K, 4), device=dev), "means": torch.empty((K, 3), device=dev),
                    "scales": torch.empty((K, 2), device=dev), "opacities": torch.empty(K, device=dev)}
        self.gact = {k: torch.empty_like(v) for k, v in self.act.items()}
        self.gact["sh"] = self.g["sh"]
        self.gact["textures"] = self.g["textures"]
        self.target = t(target.reshape(-1, 3))
        self.out = (torch.empty((self.P, 3), device=dev), torch.empty(self.P, device=dev),
                    torch.empty(self.P, device=dev))
        self.d_rgb = torch.empty((self.P, 3), device=dev)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.it = 0
        self.saved = R.Saved(self.rast)
        self.stream = torch.cuda.current_stream(dev)
        self.use_graph = graph
        self._graph = None
        self._adam = [R.AdamStep(self.rast, [self.p[k]], [self.g[k]], [self.m[k]], [self.v[k]], lr=self.lr[k])
                      for k in RAW]
        # one synchronizing forward sizes the saved state; later ones never sync
        self._activate()
        self.rast.forward([self._scene()], [self.cam], saved=self.saved, out=self.out, stream=self.stream)
        st = self.saved.stats()
        self.saved.reserve(st["records"], int(st["instances"] * 2) + 4096, self.P, st["tiles"])

    def _scene(self) -> dict:
        return {"means": self.act["means"], "quats": self.act["quats"], "scales": self.act["scales"],
                "opacities": self.act["opacities"], "sh": self.p["sh"], "textures": self.p["textures"],
                "sh_degree": 0, "tex_n": self.tex_n, "sigma": self.sigma}

    def _activate(self, stream=None):
        a = self.act
        s = stream if stream is not None else self.stream
        L.check(L.load().gb_fit_params(self.rast.ctx, self.K, self.p["theta"].data_ptr(), self.p["xy"].data_ptr(),
                                       self.z.data_ptr(), self.p["log_scales"].data_ptr(),
                                       self.p["logit_opacities"].data_ptr(), a["quats"].data_ptr(),
                                       a["means"].data_ptr(), a["scales"].data_ptr(), a["opacities"].data_ptr(),
                                       C.c_void_p(s.cuda_stream)), self.rast.ctx)

    def forward_loss(self, stream=None):
        """Activation, render and MSE (loss and dL/drgb stay on the device)."""
        st = stream if stream is not None else self.stream
        lib, ctx, s = L.load(), self.rast.ctx, C.c_void_p(st.cuda_stream)
        self._activate(st)
        self.rast.forward([self._scene()], [self.cam], saved=self.saved, out=self.out, stream=st,
                          flags=L.GB_FLAG_NO_SYNC)
        L.check(lib.gb_mse_loss(ctx, self.out[0].data_ptr(), self.target.data_ptr(), self.P * 3,
                                self.d_rgb.data_ptr(), self.loss_dev.data_ptr(), s), ctx)

    def backward(self, stream=None):
        """Gradients of the raw parameters from the current dL/drgb (self.d_rgb)."""
        st = stream if stream is not None else self.stream
        lib, ctx, s = L.load(), self.rast.ctx, C.c_void_p(st.cuda_stream)
        self.rast.backward(self.saved, self.d_rgb, grads=[self.gact], stream=st)
        ga = self.gact
        L.check(lib.gb_fit_params_backward(ctx, self.K, self.p["theta"].data_ptr(), self.p["log_scales"].data_ptr(),
                                           self.p["logit_opacities"].data_ptr(), ga["quats"].data_ptr(),
                                           ga["means"].data_ptr(), ga["scales"].data_ptr(),
                                           ga["opacities"].data_ptr(), self.g["theta"].data_ptr(),
                                           self.g["xy"].data_ptr(), self.g["log_scales"].data_ptr(),
                                           self.g["logit_opacities"].data_ptr(), s), ctx)

    def update(self):
        """Adam step of every parameter group."""
        self.it += 1
        for adam in self._adam:
            adam(self.it, self.stream)

    def _capture(self):
        """Records activation, render, loss, backward and the raw-parameter
        adjoint as one CUDA graph; every buffer they touch is allocated
        already and stays in place, so the graph replays any later iteration."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            s = torch.cuda.current_stream()
            self.forward_loss(s)
            self.backward(s)
        self._graph = g

    def step(self):
        """One iteration; the loss of the image rendered in it stays on the device."""
        if self.use_graph:
            if self._graph is None:
                self._capture()
            with torch.cuda.stream(self.stream):
                self._graph.replay()
        else:
            self.forward_loss()
            self.backward()
        self.update()

    def check(self):
        """Raises if a no-sync forward overflowed its reserved capacity."""
        self.saved.check()

    def ensure_capacity(self, headroom: float = 0.7):
        """Checks the last forward and doubles the instance capacity once it is
        more than ``headroom`` full (splats grow while fitting).  Synchronizes."""
        self.check()
        st = self.saved.stats()
        if st["instances"] > headroom * st["capacity"]:
            self.saved.reserve(st["records"], 2 * st["capacity"], self.P, st["tiles"])
            self._graph = None  # the saved state's buffers moved: capture again

    def loss(self) -> float:
        """MSE of the image rendered in the last step (synchronizes)."""
        self.stream.synchronize()
        return float(self.loss_dev.item())

    def psnr(self) -> float:
        return -10.0 * math.log10(max(self.loss(), 1e-20))

    def image(self) -> np.ndarray:
        self.stream.synchronize()
        return self.out[0].reshape(self.cam["height"], self.cam["width"], 3).cpu().numpy()


def main(argv=None):
    ap = argparse.ArgumentParser(description="Fit textured 2D Gaussian splats to a synthetic image (Sec. 4.1).")
    ap.add_argument("--target", default="wide", help="wide | landscape | portrait, or WxH")
    ap.add_argument("--splats", type=int, default=1000)
    ap.add_argument("--tex-n", type=int, default=4)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-graph", action="store_true", help="launch every step from the host")
    args = ap.parse_args(argv)
    tgt = args.target if args.target in scenes.FIT_TARGETS else tuple(int(x) for x in args.target.split("x"))
    target = scenes.fit_target(tgt, seed=args.seed)
    fit = ImageFit(target, args.splats, tex_n=args.tex_n, seed=args.seed, graph=not args.no_graph)
    t0 = time.perf_counter()
    for i in range(1, args.steps + 1):
        fit.step()
        if i % args.log_every == 0 or i == args.steps:
            fit.ensure_capacity()
            print(json.dumps({"step": i, "loss": fit.loss(), "psnr": fit.psnr(),
                              "s": round(time.perf_counter() - t0, 3)}), flush=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"iterations_per_s": args.steps / dt, "splats": args.splats, "target": list(target.shape)}))


if __name__ == "__main__":
    main()
