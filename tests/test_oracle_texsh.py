"""Pins of the oracle's per-texel spherical harmonics (Sec. 4.2: M
coefficient triples per texel instead of one RGB colour, evaluated for the
splat's view direction): texels that all hold the same coefficients render
like a one-texel grid whose colour is that SH term, and the coefficient and
centre gradients (the latter through the view direction) match central
differences."""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes


@pytest.mark.parametrize("Dt", [1, 2, 3])
def test_identical_texel_sh_equals_splat_sh(Dt):
    base = scenes.tiny_scene(70 + Dt, K=6, tex_n=4, sh_degree=Dt)
    M = (Dt + 1) ** 2
    rng = np.random.default_rng(Dt)
    c = rng.normal(0, 0.3, (6, 1, 1, M, 3))
    a = dict(base, textures=np.ascontiguousarray(np.broadcast_to(c, (6, 4, 4, M, 3))), tex_sh_degree=Dt,
             sh=np.zeros_like(base["sh"]))
    b = dict(base, tex_n=1, textures=np.zeros((6, 1, 1, 3)), sh=c.reshape(6, M, 3))
    cam = scenes.tiny_camera(24, 20, eye=(0.4, -0.3, -4.0))
    ra, rb = oracle.render(a, cam), oracle.render(b, cam)
    np.testing.assert_allclose(ra["rgb"], rb["rgb"], rtol=0, atol=1e-13)


def test_degree_zero_coefficient_is_the_colour():
    """With only the l = 0 term, a texel shows k00 Y00 (Y00 = 1 / (2 sqrt(pi)))
    from every direction: the plain grid of those colours."""
    sc = scenes.tiny_scene(75, K=5, tex_n=4, sh_degree=1)
    t = scenes.with_texel_sh(sc, 1, seed=1, std=0.0)
    plain = dict(sc, textures=t["textures"][:, :, :, 0, :].astype(np.float64) * (0.5 / np.sqrt(np.pi)))
    cam = scenes.tiny_camera(20, 18)
    np.testing.assert_allclose(oracle.render(t, cam)["rgb"], oracle.render(plain, cam)["rgb"], rtol=0,
                               atol=1e-13)


@pytest.mark.parametrize("name", ["textures", "means"])
def test_texel_sh_gradients_by_central_differences(name):
    sc = scenes.with_texel_sh(scenes.tiny_scene(76, K=3, tex_n=2, sh_degree=1), 2, seed=2, std=0.3)
    for key in ("means", "textures"):
        sc[key] = sc[key].astype(np.float64)
    cam = scenes.tiny_camera(14, 12, eye=(0.5, 0.3, -3.5))
    rng = np.random.default_rng(3)
    d = rng.standard_normal((12, 14, 3))
    g = oracle.backward(sc, cam, d)[name]
    h = 1e-6
    num = np.zeros_like(g)
    for idx in np.ndindex(*g.shape):
        sp, sm = dict(sc), dict(sc)
        sp[name] = sc[name].copy()
        sm[name] = sc[name].copy()
        sp[name][idx] += h
        sm[name][idx] -= h
        rp, rm = oracle.render(sp, cam), oracle.render(sm, cam)
        assert np.array_equal(rp["n_contrib"], rm["n_contrib"])
        num[idx] = (np.sum(d * rp["rgb"]) - np.sum(d * rm["rgb"])) / (2 * h)
    assert np.abs(g).max() > 1e-4
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-7 * np.abs(g).max())
