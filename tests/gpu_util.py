"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle

IMG_TOL = 2e-5        # max abs error of rgb and alpha against the FP64 oracle
COND_TOL = 32 * 2.0 ** -24  # per unit of the oracle's conditioning: the bar is max(IMG_TOL, COND_TOL*cond)
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
            keys=False, batch=0, rast=None, tile=16, ppt=1, batch_fwd=0):
    import torch

    from paper_2412_12734_gb300 import render as R
    rast = rast or R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in scenes_np]
    rgb, depth, alpha, saved = rast.forward(dev, cams, cam_scene=cam_scene, background=bg, batch=batch, tile=tile,
                                            ppt=ppt, batch_fwd=batch_fwd)
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


def compare_images(gpu_img, ref, what="rgb", tol=IMG_TOL, relative_to=None):
    """Max error, in units of the ``tol`` bar, over pixels whose forward
    decisions are not within the margin.

    The kernels evaluate every pixel/splat pair in FP32 (the design's precision; the paper fixes none), so a
    pixel's error scales with the conditioning of that evaluation: the oracle's
    ``cond`` is the alpha*T-weighted sensitivity of (u, v) to relative rounding
    of the centre-relative terms, about 1 for most pixels and up to a few
    hundred where a sub-pixel-thin splat is seen from far along its long axis.
    A pixel's bar is max(tol, COND_TOL * cond); its error is scaled by
    tol / bar, so the returned value compares directly with ``tol``."""
    mask = ref["margin_fwd"] > MARGIN_FWD
    a = np.asarray(gpu_img, np.float64)
    b = ref[what]
    err = np.abs(a - b)
    if relative_to is not None:
        err = err / np.maximum(1.0, np.abs(relative_to))
    if err.ndim == 3:
        err = err.max(axis=2)
    err = err * (tol / np.maximum(tol, COND_TOL * ref["cond"]))
    excluded = int((~mask).sum())
    return float(err[mask].max()) if mask.any() else 0.0, excluded


GRAD_FLOOR = 1e-2     # elements below this fraction of the tensor's max get an absolute bound


def grad_errors(g_gpu: dict, g_ref: dict) -> dict:
    """Worst ratio |g - g*| / (GRAD_REL * max(|g*|, GRAD_FLOOR max|g*|)) per tensor (<= 1 passes).

    Elements much smaller than the tensor's largest entry are differences of
    larger FP32 sums (u, v carry ~1e-7 relative FP32 error, amplified by
    (N-1)/(2 sigma) in the texel weights), so below 1 % of the maximum the
    bound is absolute: 1e-5 of the maximum."""
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
