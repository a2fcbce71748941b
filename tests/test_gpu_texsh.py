"""Per-texel spherical harmonics on the GPU (Sec. 4.2: M coefficient triples
per texel, evaluated for each splat's view direction): image and every
gradient (coefficients, and the centre through the view direction) against
the FP64 oracle, with several views of a scene (the coefficient gradient sums
over them) and next to a plain scene in the same launch."""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes
from tests.gpu_util import IMG_TOL, compare_images, gpu_run, grad_errors, masked_upstream, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Dt,N,dtype", [(1, 4, "f32"), (3, 4, "f16"), (2, 2, "f32"), (3, 8, "bf16")])
@pytest.mark.parametrize("ppt", [1, 2])
def test_texel_sh_two_views(Dt, N, dtype, ppt):
    base = scenes.tiny_scene(80 + Dt + N, K=8, tex_n=N, sh_degree=1, tex_dtype=dtype)
    sc = scenes.with_texel_sh(base, Dt, seed=Dt, std=0.3)
    cams = [scenes.tiny_camera(40, 32), scenes.tiny_camera(36, 30, eye=(0.8, -0.5, -3.8))]
    refs = [oracle_run(sc, c) for c in cams]
    rng = np.random.default_rng(Dt * 10 + N)
    d = [masked_upstream(r, rng) for r in refs]
    gpu = gpu_run([sc], cams, cam_scene=[0, 0], d_rgb=d, ppt=ppt)
    for i, r in enumerate(refs):
        e, _ = compare_images(gpu["rgb"][i], r, "rgb")
        assert e <= IMG_TOL, (i, e)
    og = None
    for i, c in enumerate(cams):
        og = oracle.backward(sc, c, d[i], grads=og)
    assert gpu["grads"][0]["textures"].shape == og["textures"].shape
    errs = grad_errors(gpu["grads"][0], og)
    assert all(v <= 1.0 for v in errs.values()), errs


def test_texel_sh_next_to_a_plain_scene():
    s0 = scenes.with_texel_sh(scenes.tiny_scene(90, K=6, tex_n=4, sh_degree=2), 2, seed=5, std=0.3)
    s1 = scenes.tiny_scene(91, K=7, tex_n=4, sh_degree=3, tex_dtype="f16")
    cams = [scenes.tiny_camera(30, 26), scenes.tiny_camera(28, 28, eye=(-0.4, 0.2, -4.1)),
            scenes.tiny_camera(33, 21, eye=(0.3, 0.3, -3.9))]
    cs = [0, 1, 0]
    sl = [s0, s1]
    refs = [oracle_run(sl[cs[i]], c) for i, c in enumerate(cams)]
    rng = np.random.default_rng(7)
    d = [masked_upstream(r, rng) for r in refs]
    gpu = gpu_run(sl, cams, cam_scene=cs, d_rgb=d)
    for i, r in enumerate(refs):
        e, _ = compare_images(gpu["rgb"][i], r, "rgb")
        assert e <= IMG_TOL, (i, e)
    for s in range(2):
        og = None
        for i, c in enumerate(cams):
            if cs[i] == s:
                og = oracle.backward(sl[s], c, d[i], grads=og)
        errs = grad_errors(gpu["grads"][s], og)
        assert all(v <= 1.0 for v in errs.values()), (s, errs)


def test_texel_sh_needs_reserved_scratch_in_no_sync_mode():
    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    sc = scenes.with_texel_sh(scenes.tiny_scene(92, K=4, tex_n=4), 1)
    rast = R.Rasterizer(0)
    saved = R.Saved(rast)
    saved.reserve(16, 4096, 4096, 64)
    with pytest.raises(L.GbillError) as ei:
        rast.forward([R.scene_to_device(sc)], [scenes.tiny_camera(16, 16)], saved=saved, flags=L.GB_FLAG_NO_SYNC)
    assert ei.value.status == 4


@pytest.mark.parametrize("Dt,dtype", [(3, "f16"), (1, "f32"), (3, "bf16")])
def test_texel_sh_unaligned_storage_matches_aligned(Dt, dtype):
    """Coefficients and their gradient output that do not start on a 16-byte
    boundary take the passes' scalar-load paths: the same images bit for bit
    and the same gradients up to the order of the render's atomics."""
    import torch

    from paper_2412_12734_gb300 import render as R
    sc = scenes.with_texel_sh(scenes.tiny_scene(95 + Dt, K=9, tex_n=4, sh_degree=1, tex_dtype=dtype), Dt, seed=3,
                              std=0.3)
    cams = [scenes.tiny_camera(36, 28), scenes.tiny_camera(30, 34, eye=(0.6, 0.4, -3.9))]
    rast = R.Rasterizer(0)
    d = torch.as_tensor(np.random.default_rng(4).standard_normal((36 * 28 + 30 * 34, 3)), dtype=torch.float32,
                        device="cuda")

    def run(offset):
        dev = R.scene_to_device(sc)
        tex = dev["textures"]
        if offset:
            # same values one element past a 16-byte boundary
            buf = torch.empty(tex.numel() + 1, dtype=tex.dtype, device="cuda")
            buf[1:] = tex.reshape(-1)
            dev["textures"] = buf[1:].view(tex.shape)
        rgb, _, _, saved = rast.forward([dev], cams, cam_scene=[0, 0])
        K = tex.shape[0]
        gbuf = torch.empty(tex.numel() + offset, device="cuda")
        grads = [{"means": torch.empty((K, 3), device="cuda"), "quats": torch.empty((K, 4), device="cuda"),
                  "scales": torch.empty((K, 2), device="cuda"), "opacities": torch.empty(K, device="cuda"),
                  "sh": torch.empty_like(dev["sh"], dtype=torch.float32),
                  "textures": gbuf[offset:].view(tex.shape)}]
        rast.backward(saved, d, grads=grads)
        torch.cuda.synchronize()
        return rgb.cpu().numpy(), {k: v.cpu().numpy() for k, v in grads[0].items()}

    rgb_a, g_a = run(0)
    rgb_u, g_u = run(1)
    assert np.array_equal(rgb_a, rgb_u)
    for k in ("textures", "means"):
        scale = np.abs(g_a[k]).max()
        assert np.abs(g_a[k] - g_u[k]).max() <= 1e-5 * max(scale, 1e-12), k
