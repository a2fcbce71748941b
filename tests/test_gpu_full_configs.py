"""Parity at the full sizes of the benchmark configurations, on outputs the
FP64 oracle can compute one at a time.

* plain FP32 (100k splats): autograd through ``render`` on the first 64
  splats in a 64 x 64 crop against the oracle's gradients and against FP64
  central differences of the loss along random directions (a gradcheck);
* batched views (1M splats, 16 views, 4x4 and 8x8 FP16 grids) in the launch
  configuration the bench times: camera 0's keys bit for bit, its image, and
  the gradients of a loss on camera 0 only;
* training step (3M splats, BF16 8x8 grids and SH, 8 views of 1600x1067):
  forward, backward and fused Adam over all parameters at full size, the
  error against the oracle on the 20k-splat crop (splats whose centres
  project into a 256 x 256 window of view 0, the first 20k by id) and the
  Adam update on sampled elements;
* uneven multi-scene batch (12 scenes, 10k-2M splats, 2x2/4x4/8x8 FP16
  grids, 1-4 views each) in one persistent launch sequence against the same
  scenes rendered one by one, and the smallest scene's first view against
  the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes
from tests.gpu_util import (IMG_TOL, compare_images, gpu_run, grad_errors, masked_upstream, oracle_run,
                            split_pixels)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _crop_camera(cam, x0, y0, w, h):
    c = dict(cam)
    c["width"], c["height"] = int(w), int(h)
    c["cx"] = np.float32(float(cam["cx"]) - x0)
    c["cy"] = np.float32(float(cam["cy"]) - y0)
    return c


def test_plain_100k_gradcheck_64_splats():
    import torch

    from paper_2412_12734_gb300 import render as R
    w = scenes.workload("plain_100k")
    sc = scenes.subset(w["scenes"][0], np.arange(64))
    cam0 = w["cams"][0]
    # the 64 x 64 window holding the most projected centres of the 64 splats
    c = oracle.project(sc, cam0)["centre"]
    inside = (c[:, 0] > 32) & (c[:, 0] < 1280 - 32) & (c[:, 1] > 32) & (c[:, 1] < 720 - 32)
    counts = [(np.sum((np.abs(c[:, 0] - c[i, 0]) < 32) & (np.abs(c[:, 1] - c[i, 1]) < 32)), i)
              for i in np.nonzero(inside)[0]]
    best = max(counts)[1]
    cam = _crop_camera(cam0, int(c[best, 0]) - 32, int(c[best, 1]) - 32, 64, 64)
    ref = oracle.render(sc, cam)
    rng = np.random.default_rng(8)
    wts = masked_upstream(ref, rng)
    dev = R.scene_to_device(sc)
    names = ("means", "quats", "scales", "opacities", "sh", "textures")
    leaves = [dev[k].clone().requires_grad_(True) for k in names]
    rgb, _, _ = R.render(*leaves, [cam], sh_degree=sc["sh_degree"], tex_n=sc["tex_n"],
                         sigma=sc.get("sigma", 0.5))
    loss = (rgb * torch.as_tensor(wts.reshape(-1, 3), dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    g_gpu = {k: t.grad.double().cpu().numpy() for k, t in zip(names, leaves)}
    og = oracle.backward(sc, cam, wts)
    errs = grad_errors(g_gpu, og)
    assert all(v <= 1.0 for v in errs.values()), errs
    # directional derivatives: <g_autograd, v> against FP64 central differences
    L = lambda s: float(np.sum(wts * oracle.render(s, cam)["rgb"]))
    for k in names:
        v = rng.standard_normal(sc[k].shape)
        h = 1e-7 * max(1.0, float(np.abs(sc[k]).max()))
        sp, sm = dict(sc), dict(sc)
        sp[k] = sc[k].astype(np.float64) + h * v
        sm[k] = sc[k].astype(np.float64) - h * v
        num = (L(sp) - L(sm)) / (2 * h)
        ana = float(np.sum(g_gpu[k] * v))
        scale = float(np.sqrt(np.sum(g_gpu[k] ** 2) * np.sum(v ** 2)))
        assert abs(num - ana) <= 2e-3 * abs(num) + 1e-4 * scale, (k, num, ana)


@pytest.mark.parametrize("tex_n,kernel,batch,batch_fwd", [(4, 1, 184, 88), (8, 1, 64, 48), (4, 2, 176, 88)])
def test_batched_1m_camera0_at_full_size(tex_n, kernel, batch, batch_fwd):
    """Camera 0 of the 16-view workload with all 16 views in the launch, keys
    bit-exact, image and gradients against the oracle, at the tile size and
    batch depths the autotuner picks for the bench on this workload (tile 16;
    backward / forward depth 184 / 88 at N = 4, 64 / 48 at N = 8); kernel 1 / 2:
    the pixel-parallel / splat-parallel backward (the latter at depth 176)."""
    wl = scenes.workload("batched_1m", tex_n=tex_n)
    sc, cams = wl["scenes"][0], wl["cams"]
    ref = oracle_run(sc, cams[0], prefilter=True)
    rng = np.random.default_rng(tex_n)
    d0 = masked_upstream(ref, rng)
    d_rgb = [d0] + [np.zeros((int(c["height"]), int(c["width"]), 3), np.float32) for c in cams[1:]]
    gpu = gpu_run([sc], cams, d_rgb=d_rgb, keys=True, tile=16, batch=batch, batch_fwd=batch_fwd, bwd_kernel=kernel)
    keys, ids, cidx = gpu["keys"]
    k0, i0 = oracle.tile_keys(sc, cams[0], 16, 0)
    assert np.array_equal(keys[cidx == 0], k0)
    assert np.array_equal(ids[cidx == 0], i0)
    e, excl = compare_images(gpu["rgb"][0], ref, "rgb")
    assert excl <= 0.001 * ref["rgb"].shape[0] * ref["rgb"].shape[1], excl
    assert e <= IMG_TOL, e
    og = oracle.backward(sc, cams[0], d0, prefilter=True)
    errs = grad_errors(gpu["grads"][0], og)
    assert all(v <= 1.0 for v in errs.values()), errs


def test_train_3m_step_and_crop():
    import torch

    from paper_2412_12734_gb300 import render as R
    wl = scenes.workload("train_3m")
    sc, cams = wl["scenes"][0], wl["cams"]
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(sc)
    # full-size forward + backward over the 8 views, then fused Adam on every
    # parameter (FP32 masters; BF16 copies of SH and grids written by the kernel)
    rgb, _, _, saved = rast.forward([dev], cams, tile=16)
    d = torch.as_tensor(np.concatenate([x.reshape(-1, 3) for x in wl["d_rgb"]]), device="cuda")
    g = rast.backward(saved, d)[0]
    names = ("means", "quats", "scales", "opacities", "sh", "textures")
    for k in names:
        assert torch.isfinite(g[k]).all(), k
    master = {k: dev[k].float().clone() for k in names}
    m = {k: torch.zeros_like(master[k]) for k in names}
    v = {k: torch.zeros_like(master[k]) for k in names}
    before = {k: master[k].cpu().numpy().astype(np.float64) for k in names}
    shadows = [None, None, None, None, dev["sh"], dev["textures"]]
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-3, 0.9, 0.999, 1e-15))
    R.adam_step(rast, [master[k] for k in names], [g[k] for k in names], [m[k] for k in names],
                [v[k] for k in names], 1, lr=lr, betas=(b1, b2), eps=eps, shadows=shadows)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for k in names:
        flat = master[k].reshape(-1)
        idx = rng.integers(0, flat.numel(), 4096)
        gk = g[k].reshape(-1)[idx].double().cpu().numpy()
        p_ref, _, _ = oracle.adam_step(before[k].reshape(-1)[idx], gk, 0, 0, 1, lr, b1, b2, eps)
        np.testing.assert_allclose(flat[idx].cpu().numpy(), p_ref, rtol=2e-6, atol=2e-6 * lr)
    sh_bf = dev["sh"].reshape(-1)[:4096].float().cpu().numpy()
    np.testing.assert_array_equal(sh_bf, scenes.round_to(master["sh"].reshape(-1)[:4096].cpu().numpy(), "bf16"))
    # the 20k-splat crop of view 0: image and gradients against the oracle
    c = oracle.project(sc, cams[0])["centre"]
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    x0, y0 = W // 2 - 128, H // 2 - 128
    sel = np.nonzero((c[:, 0] >= x0) & (c[:, 0] < x0 + 256) & (c[:, 1] >= y0) & (c[:, 1] < y0 + 256))[0][:20000]
    assert len(sel) >= 5000, len(sel)
    sub = scenes.subset(sc, sel)
    win = (x0, y0, 256, 256)
    ref = oracle.render(sub, cams[0], window=win, prefilter=True)
    d_win = masked_upstream(ref, rng)
    d_full = np.zeros((H, W, 3), np.float32)
    d_full[y0:y0 + 256, x0:x0 + 256] = d_win
    gpu = gpu_run([sub], [cams[0]], d_rgb=[d_full], tile=16)
    e, _ = compare_images(gpu["rgb"][0][y0:y0 + 256, x0:x0 + 256], ref, "rgb")
    assert e <= IMG_TOL, e
    og = oracle.backward(sub, cams[0], d_win, window=win, prefilter=True)
    errs = grad_errors(gpu["grads"][0], og)
    assert all(v <= 1.0 for v in errs.values()), errs


def test_multi_scene_persistent_batch_matches_one_by_one():
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    wl = scenes.workload("multi_scene")
    sl, cams, cs = wl["scenes"], wl["cams"], wl["cam_scene"]
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in sl]
    d = torch.as_tensor(np.concatenate([x.reshape(-1, 3) for x in wl["d_rgb"]]), device="cuda")
    rgb, _, _, saved = rast.forward(dev, cams, cam_scene=cs, tile=16, flags=L.GB_FLAG_PERSISTENT)
    gb = rast.backward(saved, d)
    rgb_b = split_pixels(rgb.cpu().numpy(), cams)
    off = 0
    offs = []
    for c in cams:
        offs.append(off)
        off += int(c["width"]) * int(c["height"])
    for s in range(len(sl)):
        mine = [i for i in range(len(cams)) if cs[i] == s]
        sub_cams = [cams[i] for i in mine]
        d_s = torch.cat([d[offs[i]:offs[i] + int(cams[i]["width"]) * int(cams[i]["height"])] for i in mine])
        r1, _, _, s1 = rast.forward([dev[s]], sub_cams, tile=16)
        g1 = rast.backward(s1, d_s.contiguous())[0]
        r1 = split_pixels(r1.cpu().numpy(), sub_cams)
        for j, i in enumerate(mine):
            assert np.array_equal(rgb_b[i], r1[j]), (s, i)
        for k in g1:
            a, b = gb[s][k], g1[k]
            scale = b.abs().max().item()
            assert (a - b).abs().max().item() <= 1e-5 * max(scale, 1e-12), (s, k)
    # the smallest scene's first view against the oracle
    s = int(np.argmin([x["means"].shape[0] for x in sl]))
    i = cs.index(s)
    ref = oracle_run(sl[s], cams[i], prefilter=True)
    e, _ = compare_images(rgb_b[i], ref, "rgb")
    assert e <= IMG_TOL, e
