"""Parity of the preprocess step alone: the projected records exported from
the GPU, evaluated in FP64 at sample pixels, against the oracle's ray/splat
intersection (u, v), low-pass branch and alpha (Eq. 3-4, 2DGS intersection).

This isolates the record's precision (double-float centre, FP64 homography
for grazing splats) from the per-pixel FP32 arithmetic of the render.

Bound: each record field is stored in FP32 with an error of a few ulps of its
row's magnitude, so u and v (on the uv branch) carry a relative error of
about 1e-6 times the condition number of zeta_z = m20 dx + m21 dy + m22 at
that pixel, kappa = (|m20 dx| + |m21 dy| + |m22|) / |zeta_z| (large near the
splat plane's vanishing line); kappa is computed from the oracle's FP64
homography.  Alpha must agree within 5e-6 absolute."""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes

pytestmark = pytest.mark.gpu


def _eval_records(rec, xy):
    """u, v, rho and depth of records rec[i] at pixel centres xy[i] (FP64)."""
    r = rec.astype(np.float64)
    dx = (xy[:, 0] - r[:, 8]) - r[:, 10]
    dy = (xy[:, 1] - r[:, 9]) - r[:, 11]
    zx = r[:, 0] * dx + r[:, 1] * dy
    zy = r[:, 2] * dx + r[:, 3] * dy
    zz = r[:, 4] * dx + r[:, 5] * dy + r[:, 6]
    u, v = zx / zz, zy / zz
    ruv = u * u + v * v
    rlp = 2.0 * (dx * dx + dy * dy)
    rho = np.minimum(ruv, rlp)
    alpha = np.minimum(0.99, r[:, 12] * np.exp(-0.5 * rho))
    return u, v, alpha, ruv <= rlp


@pytest.mark.parametrize("case", ["plain_100k", "tiny", "grazing"])
def test_records_match_oracle_intersection(case):
    from paper_2412_12734_gb300 import render as R
    if case == "plain_100k":
        w = scenes.workload("plain_100k")
        sc, cam = w["scenes"][0], w["cams"][0]
    elif case == "tiny":
        sc, cam = scenes.tiny_scene(12, K=40, spread=0.8), scenes.tiny_camera(64, 48)
    else:
        # splats whose normal is nearly perpendicular to the view ray
        sc = scenes.tiny_scene(13, K=40, spread=0.8)
        ang = np.random.default_rng(0).uniform(-0.05, 0.05, 40)
        # rotation about x by 90 deg +- small angle: normal ~ +-y, camera looks along +z
        half = (np.pi / 2 + ang) / 2
        sc["quats"] = np.stack([np.cos(half), np.sin(half), 0 * half, 0 * half], 1).astype(np.float32)
        cam = scenes.tiny_camera(64, 48)
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(sc)
    _, _, _, saved = rast.forward([dev], [cam])
    rec, vis = saved.export_records()
    valid, _, prect = oracle.keys32(sc, cam)
    assert np.array_equal(vis, valid)
    rng = np.random.default_rng(1)
    ks = np.nonzero(valid)[0]
    if len(ks) > 1500:
        ks = rng.choice(ks, 1500, replace=False)
    pr = oracle.project(sc, cam)
    worst_u = worst_a = 0.0
    for k in ks:
        x0, y0, x1, y1 = prect[k]
        xy = np.stack([rng.integers(x0, x1 + 1, 8), rng.integers(y0, y1 + 1, 8)], 1) + 0.5
        ref = oracle.eval_pairs(sc, cam, int(k), xy)
        u, v, a, uvb = _eval_records(np.repeat(rec[k:k + 1], len(xy), 0), xy)
        ok = np.isfinite(ref["u"])
        # condition number of zeta_z from the FP64 homography (centre at the origin)
        T = pr["T"][k]
        z = T[2, 2]
        c = T[:2, 2] / z
        t = T[:2, :2] - np.outer(c, T[2, :2])
        m20 = (t[1, 0] * T[2, 1] - t[1, 1] * T[2, 0]) / z
        m21 = (t[0, 1] * T[2, 0] - t[0, 0] * T[2, 1]) / z
        m22 = (t[0, 0] * t[1, 1] - t[0, 1] * t[1, 0]) / z
        dx, dy = xy[:, 0] - c[0], xy[:, 1] - c[1]
        zz = m20 * dx + m21 * dy + m22
        kappa = (np.abs(m20 * dx) + np.abs(m21 * dy) + np.abs(m22)) / np.abs(zz)
        su = np.abs(u - ref["u"]) / (1.0 + np.abs(ref["u"])) / kappa
        sv = np.abs(v - ref["v"]) / (1.0 + np.abs(ref["v"])) / kappa
        # u, v matter where they set alpha (uv branch) inside the alpha support
        inside = ok & (ref["alpha"] >= 1 / 255) & (ref["uv_branch"] == 1)
        if inside.any():
            worst_u = max(worst_u, float(np.max(np.maximum(su, sv)[inside])))
        worst_a = max(worst_a, float(np.max(np.abs(a - ref["alpha"])[ok])))
    assert worst_u < 1e-5, f"u/v error / (kappa (1+|u|)) = {worst_u:.3e}"
    assert worst_a < 5e-6, f"alpha error {worst_a:.3e}"
