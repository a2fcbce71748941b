"""Pins of the oracle's image-fitting pieces (Sec. 4.1): the parameter map
(a turn about the view axis, exp scales, sigmoid opacity), the MSE loss and
their composition with the renderer, against closed forms and central
differences of the whole loss."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes


def test_fit_params_closed_forms():
    raw = {"theta": np.array([0.0, math.pi, math.pi / 2]), "xy": np.array([[0.1, -0.2], [0, 0], [1, 2]]),
           "z": np.array([1.0, 2.0, 3.0]), "log_scales": np.log([[0.5, 2.0], [1, 1], [3, 4]]),
           "logit_opacities": np.array([0.0, math.log(3.0), -math.log(3.0)])}
    p = oracle.fit_params(raw)
    np.testing.assert_allclose(p["quats"][0], [1, 0, 0, 0], atol=1e-15)
    np.testing.assert_allclose(p["quats"][1], [0, 0, 0, 1], atol=1e-15)
    # theta = pi/2: the tangent t_u = first column of R(q) is (0, 1, 0)
    w, z = p["quats"][2, 0], p["quats"][2, 3]
    np.testing.assert_allclose([1 - 2 * z * z, 2 * w * z], [0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(p["means"], [[0.1, -0.2, 1], [0, 0, 2], [1, 2, 3]])
    np.testing.assert_allclose(p["scales"], [[0.5, 2.0], [1, 1], [3, 4]])
    np.testing.assert_allclose(p["opacities"], [0.5, 0.75, 0.25])


def test_mse_closed_form_and_gradient():
    rng = np.random.default_rng(0)
    a, b = rng.uniform(0, 1, (5, 4, 3)), rng.uniform(0, 1, (5, 4, 3))
    loss, d = oracle.mse_loss(a, b)
    assert abs(loss - np.sum((a - b) ** 2) / 60) < 1e-15
    h = 1e-6
    for idx in [(0, 0, 0), (4, 3, 2), (2, 1, 1)]:
        ap, am = a.copy(), a.copy()
        ap[idx] += h
        am[idx] -= h
        num = (oracle.mse_loss(ap, b)[0] - oracle.mse_loss(am, b)[0]) / (2 * h)
        assert abs(num - d[idx]) < 1e-9


def _tiny_fit(seed=0, K=5, W=20, H=16):
    raw = scenes.fit_init(K, W, H, seed=seed, tex_n=4)
    rng = np.random.default_rng(seed + 1)
    raw["textures"] = rng.uniform(0, 1, raw["textures"].shape)
    raw["log_scales"] = raw["log_scales"] + 1.0  # larger splats on the tiny image
    for k in ("theta", "xy", "z", "log_scales", "logit_opacities", "sh", "textures"):
        raw[k] = np.asarray(raw[k], np.float64)
    return raw, scenes.fit_camera(W, H), rng.uniform(0, 1, (H, W, 3))


@pytest.mark.parametrize("name", ["theta", "xy", "log_scales", "logit_opacities", "textures"])
def test_fit_gradients_by_central_differences(name):
    raw, cam, target = _tiny_fit()
    out = oracle.fit_step(raw, target, cam)
    g = out[name]
    h = 1e-6
    num = np.zeros_like(g)
    for idx in np.ndindex(*g.shape):
        rp = dict(raw)
        rm = dict(raw)
        rp[name] = raw[name].copy()
        rm[name] = raw[name].copy()
        rp[name][idx] += h
        rm[name][idx] -= h
        lp = oracle.mse_loss(oracle.render(oracle.fit_scene(rp), cam)["rgb"], target)[0]
        lm = oracle.mse_loss(oracle.render(oracle.fit_scene(rm), cam)["rgb"], target)[0]
        num[idx] = (lp - lm) / (2 * h)
    assert np.abs(g).max() > 1e-6
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8 * np.abs(g).max())
