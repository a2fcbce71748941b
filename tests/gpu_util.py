"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle

IMG_TOL = 2e-5        # max abs error of rgb and alpha against the FP64 oracle
GRAD_REL = 1e-3       # per-tensor relative gradient tolerance
MARGIN_FWD = 1e-5     # pixels this close (relative) to a forward decision are excluded
MARGIN_GRAD = 1e-4    # pixels this close to any decision get zero upstream gradient


def split_pixels(flat: np.ndarray, cams) -> list:
    out, o = [], 0
    for c in cams:
        n = int(c["width"]) * int(c["height"])
        out.append(flat[o:o + n].reshape(int(c["height"]), int(c["width"]), *flat.shape[1:]))
        o += n
    return out


def gpu_run(scenes_np, cams, cam_scene=None, d_rgb=None, d_depth=None, d_alpha=None, bg=None,
            keys=False, batch=0, rast=None, tile=16, ppt=0, batch_fwd=0, bwd_kernel=0):
    import torch

    from paper_2412_12734_gb300 import render as R
    rast = rast or R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in scenes_np]
    rgb, depth, alpha, saved = rast.forward(dev, cams, cam_scene=cam_scene, background=bg, batch=batch, tile=tile,
                                            ppt=ppt, batch_fwd=batch_fwd, bwd_kernel=bwd_kernel)
    out = {"rgb": split_pixels(rgb.cpu().numpy(), cams),
           "depth": split_pixels(depth.cpu().numpy(), cams),
           "alpha": split_pixels(alpha.cpu().numpy(), cams),
           "stats": saved.stats()}
    if keys:
        out["keys"] = saved.export_keys()
    if d_rgb is not None:
        cat = lambda xs: torch.as_tensor(np.concatenate([x.reshape(-1, *x.shape[2:]) for x in xs]),
                                         dtype=torch.float32, device="cuda").contiguous()
        g = rast.backward(saved, cat(d_rgb), cat(d_depth) if d_depth is not None else None,
                          cat(d_alpha) if d_alpha is not None else None)
        out["grads"] = [{k: v.cpu().numpy() for k, v in gi.items()} for gi in g]
    torch.cuda.synchronize()
    return out


def oracle_run(scene, cam, bg=None, prefilter=False):
    return oracle.render(scene, cam, bg=bg, prefilter=prefilter)


def compare_images(gpu_img, ref, what="rgb", relative_to=None):
    """Max abs error (relative to max(1, |relative_to|) when given) over
    pixels none of whose forward decisions lies within the margin of its
    threshold, and the number of pixels left out."""
    mask = ref["margin_fwd"] > MARGIN_FWD
    a = np.asarray(gpu_img, np.float64)
    b = ref[what]
    err = np.abs(a - b)
    if relative_to is not None:
        err = err / np.maximum(1.0, np.abs(relative_to))
    if err.ndim == 3:
        err = err.max(axis=2)
    excluded = int((~mask).sum())
    return float(err[mask].max()) if mask.any() else 0.0, excluded


GRAD_FLOOR = 1e-3     # elements below this fraction of the tensor's max get an absolute bound


def grad_errors(g_gpu: dict, g_ref: dict) -> dict:
    """Worst ratio |g - g*| / (GRAD_REL * max(|g*|, GRAD_FLOOR max|g*|)) per tensor (<= 1 passes).

    "Within 1e-3 relative" per element, with elements below 1e-3 of the
    tensor's largest entry held to an absolute bound of 1e-6 of that entry
    (their relative error is that of a difference of larger sums)."""
    out = {}
    for k, ref in g_ref.items():
        a = np.asarray(g_gpu[k], np.float64).reshape(ref.shape)
        scale = np.abs(ref).max()
        if scale == 0:
            out[k] = float(np.abs(a).max() > 0)
            continue
        den = GRAD_REL * np.maximum(np.abs(ref), GRAD_FLOOR * scale)
        out[k] = float((np.abs(a - ref) / den).max())
    return out


def masked_upstream(ref, rng, channels=3, scale=1.0):
    mask = ref["margin_grad"] > MARGIN_GRAD
    H, W = mask.shape
    d = rng.standard_normal((H, W, channels)) * scale * mask[..., None]
    return d.astype(np.float32).astype(np.float64)
