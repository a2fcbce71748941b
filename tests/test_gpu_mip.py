"""Mip-level colour grids on the GPU (Sec. 4.1, Fig. 4 f, g): the grid is
box-filtered to N/2^l at staging and the texture gradient flows back to the
stored N x N texels.  Parity with the FP64 oracle (which filters the grid in
FP64 and renders it), at every level of N = 4 and N = 8, in FP32 and FP16
storage, and with scenes of different levels in one launch.
"""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes
from tests.gpu_util import IMG_TOL, compare_images, gpu_run, grad_errors, masked_upstream, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,lvl,dtype", [(4, 1, "f32"), (4, 2, "f32"), (8, 1, "f16"), (8, 2, "f32"),
                                         (8, 3, "bf16"), (2, 1, "f32"), (16, 1, "f16"), (16, 4, "f32")])
@pytest.mark.parametrize("ppt", [1, 2])
def test_mip_image_and_gradients(N, lvl, dtype, ppt):
    sc = scenes.tiny_scene(40 + N + lvl, K=8, tex_n=N, sh_degree=2, tex_dtype=dtype)
    sc["mip_level"] = lvl
    cam = scenes.tiny_camera(45, 38)
    ref = oracle_run(sc, cam)
    rng = np.random.default_rng(lvl)
    d_rgb = masked_upstream(ref, rng)
    gpu = gpu_run([sc], [cam], d_rgb=[d_rgb], ppt=ppt)
    e, _ = compare_images(gpu["rgb"][0], ref, "rgb")
    assert e <= IMG_TOL, e
    og = oracle.backward(sc, cam, d_rgb)
    errs = grad_errors(gpu["grads"][0], og)
    assert all(v <= 1.0 for v in errs.values()), errs
    assert gpu["grads"][0]["textures"].shape == (8, N, N, 3)


def test_mip_levels_mixed_in_one_launch():
    """Three scenes (N = 8 at levels 0, 1 and 3; the last renders like N = 1)
    in one frame: one render group per rendered grid size."""
    sl = []
    for i, lvl in enumerate((0, 1, 3)):
        s = scenes.tiny_scene(50 + i, K=6, tex_n=8, sh_degree=1)
        s["mip_level"] = lvl
        sl.append(s)
    cams = [scenes.tiny_camera(30, 26), scenes.tiny_camera(33, 21, eye=(0.4, -0.2, -4.0)),
            scenes.tiny_camera(25, 25, eye=(-0.3, 0.3, -4.2))]
    rng = np.random.default_rng(9)
    refs = [oracle_run(sl[i], c) for i, c in enumerate(cams)]
    d_rgb = [masked_upstream(r, rng) for r in refs]
    gpu = gpu_run(sl, cams, cam_scene=[0, 1, 2], d_rgb=d_rgb)
    for i, r in enumerate(refs):
        e, _ = compare_images(gpu["rgb"][i], r, "rgb")
        assert e <= IMG_TOL, (i, e)
        errs = grad_errors(gpu["grads"][i], oracle.backward(sl[i], cams[i], d_rgb[i]))
        assert all(v <= 1.0 for v in errs.values()), (i, errs)


def test_mip_level_out_of_range_is_rejected():
    from paper_2412_12734_gb300 import _lib as L
    sc = scenes.tiny_scene(60, K=4, tex_n=4)
    sc["mip_level"] = 3
    with pytest.raises(L.GbillError) as ei:
        gpu_run([sc], [scenes.tiny_camera(16, 16)])
    assert ei.value.status == 1


def test_autotune_on_mip_and_texel_sh_scenes(tmp_path):
    """The autotuner allocates gradient outputs shaped like the stored grids
    (N x N, and (Dt+1)^2 coefficient triples per texel) and returns a valid
    candidate for frames that render filtered or evaluated grids."""
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    a = scenes.tiny_scene(61, K=12, tex_n=8, sh_degree=1)
    a["mip_level"] = 1
    b = scenes.with_texel_sh(scenes.tiny_scene(62, K=10, tex_n=4, sh_degree=1), 2)
    cams = [scenes.tiny_camera(40, 32), scenes.tiny_camera(36, 36, eye=(0.3, 0.2, -4.0))]
    res = rast.autotune([R.scene_to_device(a), R.scene_to_device(b)], cams, cam_scene=[0, 1], reps=1,
                        cache=str(tmp_path / "tune.json"))
    assert res["tile"] in (8, 16, 32) and res["batch"] in (8, 16, 24, 32, 48, 64, 88, 128)
    assert len(res["candidates"]) > 0
