"""Pins of the oracle with a per-splat grid size (the variable texture
resolution named as future work in Sec. 3.3 and 5): splat k's n_k x n_k grid
sits in rows and columns 0..n_k-1 of its N x N block and Alg. 2 runs with n_k.

- Embedding: grids of size n embedded in larger blocks (the other texels set
  to a value the render must never read) render exactly like the scene with
  tex_n = n, and their gradients land in the embedded texels only.
- Bilinear reproduction: bilinear interpolation reproduces any bilinear
  function exactly, so an n x n grid and its samples on the 16 x 16
  corner-aligned lattice (a lattice that contains the n x n one when n - 1
  divides 15: n = 1, 2, 4) describe the same colour function; a mixed scene
  renders like the upsampled uniform scene, and its texel gradients are the
  upsampling's adjoint applied to the uniform scene's.
- Central differences of every parameter of a mixed tiny scene.
"""
import numpy as np

import oracle
from paper_2412_12734_gb300 import scenes
from tests import test_oracle_fd as fd


def _embed(sc, N):
    n = int(sc["tex_n"])
    K = sc["means"].shape[0]
    tex = np.full((K, N, N, 3), 7.0, np.float32)
    tex[:, :n, :n] = sc["textures"]
    return dict(sc, tex_n=N, textures=tex, splat_tex_n=np.full(K, n, np.int32))


def test_embedded_grids_equal_the_uniform_scene(n=4, N=8):
    sc = scenes.tiny_scene(21, K=7, tex_n=n, sh_degree=2)
    cam = scenes.tiny_camera(36, 28)
    em = _embed(sc, N)
    a, b = oracle.render(sc, cam), oracle.render(em, cam)
    for k in ("rgb", "depth", "alpha"):
        assert np.array_equal(a[k], b[k]), k
    d = np.random.default_rng(0).standard_normal((28, 36, 3))
    ga, gb = oracle.backward(sc, cam, d), oracle.backward(em, cam, d)
    for k in ("means", "quats", "scales", "opacities", "sh"):
        assert np.array_equal(ga[k], gb[k]), k
    assert np.array_equal(gb["textures"][:, :n, :n], ga["textures"])
    assert not np.any(gb["textures"][:, n:, :]) and not np.any(gb["textures"][:, :, n:])


def _upsample_matrix(n, N=16):
    """U [N*N, n*n]: the N x N corner-aligned samples of the bilinear
    interpolant of an n x n grid over the same square (n - 1 divides N - 1)."""
    if n == 1:
        return np.ones((N * N, 1))
    t = np.arange(N) * (n - 1) / (N - 1)  # lattice coordinates in grid units
    i = np.minimum(np.floor(t).astype(int), n - 2)
    f = t - i
    W = np.zeros((N, n))
    W[np.arange(N), i] = 1 - f
    W[np.arange(N), i + 1] += f
    return np.kron(W, W)  # [(a, b), (i, j)] = W[a, i] W[b, j]


def test_mixed_grid_sizes_render_like_their_upsampled_grids():
    N = 16
    base = scenes.tiny_scene(22, K=9, tex_n=N, sh_degree=1)
    mixed = scenes.with_splat_tex_n(base, [1, 2, 4], seed=3)
    up = dict(mixed)
    del up["splat_tex_n"]
    tex = np.zeros_like(mixed["textures"], dtype=np.float64)
    for k, n in enumerate(mixed["splat_tex_n"]):
        g = mixed["textures"][k, :n, :n].astype(np.float64).reshape(n * n, 3)
        tex[k] = (_upsample_matrix(int(n), N) @ g).reshape(N, N, 3)
    up["textures"] = tex
    cam = scenes.tiny_camera(40, 32)
    a, b = oracle.render(mixed, cam), oracle.render(up, cam)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a["depth"], b["depth"], rtol=0, atol=1e-12)
    d = np.random.default_rng(1).standard_normal((32, 40, 3))
    ga, gb = oracle.backward(mixed, cam, d), oracle.backward(up, cam, d)
    for k in ("means", "quats", "scales", "opacities", "sh"):
        np.testing.assert_allclose(ga[k], gb[k], rtol=1e-9, atol=1e-9 * np.abs(gb[k]).max())
    for k, n in enumerate(mixed["splat_tex_n"]):
        expect = (_upsample_matrix(int(n), N).T @ gb["textures"][k].reshape(N * N, 3)).reshape(n, n, 3)
        np.testing.assert_allclose(ga["textures"][k, :n, :n], expect, rtol=1e-9, atol=1e-12)
        assert not np.any(ga["textures"][k][n:, :]) and not np.any(ga["textures"][k][:, n:])


def test_fd_mixed_grid_sizes():
    sc = scenes.with_splat_tex_n(scenes.tiny_scene(23, K=5, tex_n=8, sh_degree=1, scale_range=(0.6, 1.0)),
                                 [1, 2, 3, 5, 8], seed=4)
    cam = scenes.tiny_camera(20, 16, focal=14.0)
    assert fd._check(sc, cam, seed=5, n_sample=40) > 0
