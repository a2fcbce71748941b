"""Pins of the oracle's mip-level colour grids (Sec. 4.1, Fig. 4 f, g: the
grid box-filtered to 2x2 and to a single colour at render time).

The box filter is checked against explicit loops; rendering is checked
against cases whose answer is fixed without the filter: a constant grid
renders the same at every level, the top level equals the N = 1 scene whose
colour is the grid mean, and the texture gradient at a mip level equals
central differences of the fine texels (the image is linear in them).
"""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes


def test_mip_grid_matches_loops():
    rng = np.random.default_rng(3)
    g = rng.uniform(-1, 1, (3, 8, 8, 3))
    for lvl in range(4):
        f = 1 << lvl
        n = 8 // f
        want = np.zeros((3, n, n, 3))
        for k in range(3):
            for i in range(n):
                for j in range(n):
                    acc = np.zeros(3)
                    for a in range(f):
                        for b in range(f):
                            acc += g[k, f * i + a, f * j + b]
                    want[k, i, j] = acc / (f * f)
        np.testing.assert_allclose(oracle.mip_grid(g, lvl), want, rtol=0, atol=1e-15)


def test_mip_adjoint_is_the_transpose():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 8, 8, 3))
    for lvl in (1, 2, 3):
        y = rng.standard_normal((2, 8 >> lvl, 8 >> lvl, 3))
        lhs = np.sum(oracle.mip_grid(x, lvl) * y)
        rhs = np.sum(x * oracle.mip_grid_adjoint(y, lvl))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_constant_grid_renders_the_same_at_every_level():
    sc = scenes.tiny_scene(11, K=6, tex_n=8, sh_degree=1)
    rng = np.random.default_rng(0)
    colours = rng.uniform(0, 1, (6, 1, 1, 3)).astype(np.float32)
    sc["textures"] = np.ascontiguousarray(np.broadcast_to(colours, (6, 8, 8, 3)))
    cam = scenes.tiny_camera(24, 20)
    base = oracle.render(sc, cam)
    for lvl in (1, 2, 3):
        r = oracle.render(dict(sc, mip_level=lvl), cam)
        np.testing.assert_allclose(r["rgb"], base["rgb"], rtol=0, atol=1e-14)
        np.testing.assert_array_equal(r["alpha"], base["alpha"])


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_top_level_is_the_mean_colour(N):
    sc = scenes.tiny_scene(12, K=5, tex_n=N, sh_degree=2)
    cam = scenes.tiny_camera(20, 18)
    lvl = int(np.log2(N))
    mean = sc["textures"].astype(np.float64).mean(axis=(1, 2), keepdims=True)
    flat = dict(sc, tex_n=1, textures=mean)
    a = oracle.render(dict(sc, mip_level=lvl), cam)
    b = oracle.render(flat, cam)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("lvl", [1, 2])
def test_texture_gradient_at_a_mip_level_by_central_differences(lvl):
    sc = scenes.tiny_scene(13, K=3, tex_n=4, sh_degree=0)
    sc["textures"] = sc["textures"].astype(np.float64)
    sc["mip_level"] = lvl
    cam = scenes.tiny_camera(14, 12)
    rng = np.random.default_rng(1)
    d = rng.standard_normal((12, 14, 3))
    g = oracle.backward(sc, cam, d)["textures"]
    h = 1e-3
    num = np.zeros_like(g)
    for idx in np.ndindex(*g.shape):
        tp = sc["textures"].copy()
        tm = sc["textures"].copy()
        tp[idx] += h
        tm[idx] -= h
        lp = np.sum(d * oracle.render(dict(sc, textures=tp), cam)["rgb"])
        lm = np.sum(d * oracle.render(dict(sc, textures=tm), cam)["rgb"])
        num[idx] = (lp - lm) / (2 * h)
    assert np.abs(g).max() > 1e-3
    np.testing.assert_allclose(g, num, rtol=1e-7, atol=1e-9)
