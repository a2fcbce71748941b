"""Parity of the preprocess step alone: the projected records exported from
the GPU, evaluated in FP64 at sample pixels, against the oracle's ray/splat
intersection (u, v), low-pass branch and alpha (Eq. 3-4, 2DGS intersection).

This isolates the record's precision (double-float chain, FP64 homography
for grazing splats) from the per-pixel arithmetic of the render.

Bound: every field is the FP32 rounding of its double-float value.  A record
left unflagged has a conditioning bound of at most 32 (the terms summed into
the plane hit, over its footprint, are at most 32 times the result), so its
FP32 fields give u and v within about 3 x 32 x 2^-24 (1 + |u|) < 1e-5 (1 +
|u|) of the oracle's.  A flagged record (depth stored negated) carries its
low parts, and hi + lo must give u and v within 1e-8 (1 + |u|): any
ill-conditioned record the flag misses, or a wrong low part, fails.  Alpha
must agree within 5e-6 absolute."""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes

pytestmark = pytest.mark.gpu


def _eval_records(rec, lo, xy):
    """u, v, alpha and branch of records rec[i] (low parts lo[i]) at pixel centres xy[i] (FP64)."""
    r = rec.astype(np.float64)
    l = lo.astype(np.float64)
    dx = (xy[:, 0] - r[:, 8]) - r[:, 10]
    dy = (xy[:, 1] - r[:, 9]) - r[:, 11]
    a = r[:, 0:4] + l[:, 0:4]
    m20, m21 = r[:, 4] + l[:, 4], r[:, 5] + l[:, 5]
    # the low part of m22 is folded into the centre term l[:, 10] with -(m20 c_lo.x + m21 c_lo.y)
    m22 = r[:, 6] + np.where(r[:, 7] < 0, l[:, 10] + r[:, 4] * r[:, 10] + r[:, 5] * r[:, 11], 0.0)
    zx = a[:, 0] * dx + a[:, 1] * dy
    zy = a[:, 2] * dx + a[:, 3] * dy
    zz = m20 * dx + m21 * dy + m22
    u, v = zx / zz, zy / zz
    ruv = u * u + v * v
    rlp = 2.0 * (dx * dx + dy * dy)
    rho = np.minimum(ruv, rlp)
    alpha = np.minimum(0.99, r[:, 12] * np.exp(-0.5 * rho))
    return u, v, alpha, ruv <= rlp


@pytest.mark.parametrize("case", ["plain_100k", "tiny", "grazing", "edge_on"])
def test_records_match_oracle_intersection(case):
    from paper_2412_12734_gb300 import render as R
    if case == "plain_100k":
        w = scenes.workload("plain_100k")
        sc, cam = w["scenes"][0], w["cams"][0]
    elif case == "tiny":
        sc, cam = scenes.tiny_scene(12, K=40, spread=0.8), scenes.tiny_camera(64, 48)
    else:
        # splats whose normal is nearly perpendicular to the view ray (within 3
        # degrees; edge_on: within 0.12 degrees, where the homography is
        # redone in FP64 and the screen footprint is a thin line)
        sc = scenes.tiny_scene(13, K=40, spread=0.8)
        cam = scenes.tiny_camera(64, 48)
        rng = np.random.default_rng(0)
        lim = 0.05 if case == "grazing" else 0.002
        ang = rng.uniform(-lim, lim, 40)
        # normal at angle pi/2 - ang to the splat's own view ray
        d = sc["means"].astype(np.float64) - np.array([0.0, 0.0, -4.0])
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        a = np.cross(d, rng.standard_normal((40, 3)))
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        n = a * np.cos(ang)[:, None] + d * np.sin(ang)[:, None]
        sc["quats"] = scenes._normal_aligned_quats(rng, n).astype(np.float32)
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(sc)
    _, _, _, saved = rast.forward([dev], [cam])
    rec, vis, lo = saved.export_records(lo=True)
    valid, _, prect = oracle.keys32(sc, cam)
    assert np.array_equal(vis, valid)
    rng = np.random.default_rng(1)
    ks = np.nonzero(valid)[0]
    flagged = rec[:, 7] < 0
    # every flagged record is in the sample, plus up to 1500 others
    rest = ks[~flagged[ks]]
    if len(rest) > 1500:
        rest = rng.choice(rest, 1500, replace=False)
    ks = np.concatenate([ks[flagged[ks]][:3000], rest])
    worst = {False: 0.0, True: 0.0}
    worst_a = 0.0
    for k in ks:
        x0, y0, x1, y1 = prect[k]
        xy = np.stack([rng.integers(x0, x1 + 1, 8), rng.integers(y0, y1 + 1, 8)], 1) + 0.5
        ref = oracle.eval_pairs(sc, cam, int(k), xy)
        u, v, a, uvb = _eval_records(np.repeat(rec[k:k + 1], len(xy), 0), np.repeat(lo[k:k + 1], len(xy), 0), xy)
        ok = np.isfinite(ref["u"])
        su = np.abs(u - ref["u"]) / (1.0 + np.abs(ref["u"]))
        sv = np.abs(v - ref["v"]) / (1.0 + np.abs(ref["v"]))
        # u, v matter where they set alpha (uv branch) inside the alpha support
        inside = ok & (ref["alpha"] >= 1 / 255) & (ref["uv_branch"] == 1)
        if inside.any():
            f = bool(flagged[k])
            worst[f] = max(worst[f], float(np.max(np.maximum(su, sv)[inside])))
        worst_a = max(worst_a, float(np.max(np.abs(a - ref["alpha"])[ok])))
    assert worst[False] < 1e-5, f"unflagged records: u/v error / (1+|u|) = {worst[False]:.3e}"
    assert worst[True] < 1e-8, f"flagged records (hi + lo): u/v error / (1+|u|) = {worst[True]:.3e}"
    assert worst_a < 5e-6, f"alpha error {worst_a:.3e}"
    if case == "edge_on":
        assert flagged[valid].mean() > 0.5  # edge-on splats take the extended-precision path
