"""Finite-difference pins of the oracle's analytic backward (Alg. 1 bwd, Alg. 2).

For tiny scenes (<= 8 splats, <= 24x20 pixels) every parameter of every
splat is perturbed by +-h in FP64 and the central difference of
L = sum(dL/drgb . rgb) + sum(dL/ddepth . depth) + sum(dL/dalpha . alpha)
is compared with the oracle's gradient.  Pixels whose decisions (alpha
threshold, alpha clamp, cutoff, low-pass branch, grid border, grid cell) lie
within 1e-3 relative of a threshold get zero upstream gradient, so no decision
can flip between theta - h and theta + h; the test also checks that the
number of blended splats per pixel is identical at theta +- h.
"""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes

PARAMS = ("means", "quats", "scales", "opacities", "sh", "textures")


def _loss(sc, cam, dC, dD, dA, bg):
    r = oracle.render(sc, cam, bg=bg)
    return (r["rgb"] * dC).sum() + (r["depth"] * dD).sum() + (r["alpha"] * dA).sum(), r


def _check(sc, cam, seed, bg=None, use_depth=True, use_alpha=True, n_sample=None):
    H, W = cam["height"], cam["width"]
    rng = np.random.default_rng(seed)
    base = oracle.render(sc, cam, bg=bg)
    mask = base["margin_grad"] > 1e-3
    dC = rng.standard_normal((H, W, 3)) * mask[..., None]
    dD = rng.standard_normal((H, W)) * mask * (1.0 if use_depth else 0.0)
    dA = rng.standard_normal((H, W)) * mask * (1.0 if use_alpha else 0.0)
    g = oracle.backward(sc, cam, dC, dD, dA, bg=bg)
    # work on an FP64 copy so perturbations are not rounded away
    sc64 = dict(sc)
    for k in PARAMS:
        sc64[k] = np.array(sc[k], dtype=np.float64)
    checked = 0
    for name in PARAMS:
        arr = sc64[name]
        flat_idx = list(np.ndindex(arr.shape))
        if n_sample is not None and len(flat_idx) > n_sample:
            pick = rng.choice(len(flat_idx), n_sample, replace=False)
            flat_idx = [flat_idx[i] for i in pick]
        scale = max(1e-12, float(np.abs(g[name]).max()))
        for idx in flat_idx:
            x0 = arr[idx]
            h = 1e-6 * max(1.0, abs(x0))
            arr[idx] = x0 + h
            lp, rp = _loss(sc64, cam, dC, dD, dA, bg)
            arr[idx] = x0 - h
            lm, rm = _loss(sc64, cam, dC, dD, dA, bg)
            arr[idx] = x0
            assert np.array_equal(rp["n_contrib"], rm["n_contrib"]), (name, idx)
            fd = (lp - lm) / (2 * h)
            an = g[name][idx]
            assert abs(an - fd) <= 1e-5 * abs(fd) + 1e-6 * scale, (name, idx, an, fd)
            checked += 1
    return checked


@pytest.mark.parametrize("N,D", [(1, 0), (2, 3), (4, 3), (8, 1), (16, 0)])
def test_fd_all_gradients(N, D):
    sc = scenes.tiny_scene(20 + N, K=5, tex_n=N, sh_degree=D)
    cam = scenes.tiny_camera(16, 16)
    assert _check(sc, cam, seed=N) > 0


def test_fd_with_background_and_ragged_view():
    sc = scenes.tiny_scene(31, K=6, tex_n=4, sh_degree=2)
    cam = scenes.tiny_camera(24, 20, focal=36.0, eye=(0.7, -0.4, -4.0))
    assert _check(sc, cam, seed=3, bg=np.array([0.3, 0.6, 0.9])) > 0


def test_fd_clamped_opacity_and_lowpass():
    """Opacities close to 1 and a tiny splat drawn by the low-pass branch
    (the near-opaque splats here are not blended clamped at any pixel outside
    the decision margin: test_fd_through_clamped_alpha covers that branch)."""
    sc = scenes.tiny_scene(41, K=4, tex_n=2, sh_degree=0)
    sc["opacities"] = np.array([0.999, 0.9, 0.7, 0.98], np.float32)
    sc["scales"][1] = np.array([0.01, 0.02], np.float32)
    cam = scenes.tiny_camera(16, 16)
    assert _check(sc, cam, seed=4) > 0


def test_fd_through_clamped_alpha():
    """A large, mildly tilted splat with opacity 0.9995 in front of the camera
    is clamped to alpha = 0.99 (Eq. 4) over a patch of pixels: there alpha
    depends on neither the opacity nor the Gaussian, and only the colour and
    depth reach the splat's parameters.  At least four pixels outside the
    decision margin blend it clamped, so the finite differences see the
    clamped branch."""
    import math
    sc = scenes.tiny_scene(43, K=3, tex_n=4, sh_degree=1)
    sc["opacities"] = np.array([0.9995, 0.8, 0.6], np.float32)
    sc["scales"][0] = np.array([1.4, 1.12], np.float32)
    sc["means"][0] = np.array([0.05, -0.03, 0.2], np.float32)
    h = math.radians(10.0)
    sc["quats"][0] = np.array([math.cos(h), 0.8 * math.sin(h), 0.6 * math.sin(h), 0.0], np.float32)
    cam = scenes.tiny_camera(16, 16, focal=45.0)
    margin = oracle.render(sc, cam)["margin_grad"]
    n = 0
    for y in range(16):
        for x in range(16):
            if margin[y, x] > 1e-3:
                tr = oracle.pixel_trace(sc, cam, x, y)
                n += sum(1 for i, a in zip(tr["ids"], tr["alpha"]) if i == 0 and a == 0.99)
    assert n >= 4
    assert _check(sc, cam, seed=6) > 0


def test_fd_texture_only_heavy_grid():
    """Sigma = 2: most pixels inside the grid, so the colour term of the uv
    adjoint (Sec. 3.3, the paper's central backward change) dominates."""
    sc = scenes.tiny_scene(51, K=3, tex_n=4, sh_degree=0, sigma=2.0)
    cam = scenes.tiny_camera(16, 16)
    assert _check(sc, cam, seed=5, use_depth=False, use_alpha=False) > 0
