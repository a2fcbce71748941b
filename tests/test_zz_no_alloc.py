"""The forward that allocates nothing (gb_render_forward_noalloc).

For callers that cannot allocate device memory (no cudaMalloc available or
allowed to them): the entry point renders from one fixed device array built
into the library.  These tests call it through the C ABI and compare it with
the allocating gb_render_forward on the same inputs, twice in a row (the
array keeps the previous call's contents, so the second call checks that
everything that must start from zero is cleared), and check that a frame
beyond the documented limits is refused with GB_ERR_CAPACITY.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2412_12734_gb300 import scenes

pytestmark = pytest.mark.gpu


def _noalloc(rast, dev_scenes, cams, cam_scene, tile=16):
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    n_s, n_c = len(dev_scenes), len(cams)
    sarr = (L.gb_scene * n_s)(*[R.scene_struct(s) for s in dev_scenes])
    carr = (L.gb_camera * n_c)(*[R.camera_struct(c, cam_scene[i]) for i, c in enumerate(cams)])
    opt = L.gb_options()
    opt.tile_size = tile
    P = rast.pixel_count(cams)
    rgb = torch.full((P, 3), -7.0, device="cuda")
    depth = torch.full((P,), -7.0, device="cuda")
    alpha = torch.full((P,), -7.0, device="cuda")
    st = L.load().gb_render_forward_noalloc(rast.ctx, sarr, n_s, carr, n_c, C.byref(opt), rgb.data_ptr(),
                                             depth.data_ptr(), alpha.data_ptr(),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, rgb, depth, alpha


@pytest.mark.parametrize("tile", [16, 8])
def test_noalloc_forward_matches_allocating_forward_twice(tile):
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    frames = [
        ([scenes.workload("plain_1k")["scenes"][0]], scenes.workload("plain_1k")["cams"], [0]),
        ([scenes.tiny_scene(3, K=8, tex_n=4, sh_degree=3),
          scenes.tiny_scene(4, K=6, tex_n=8, sh_degree=1, sh_dtype="f16", tex_dtype="f16")],
         [scenes.tiny_camera(48, 33), scenes.tiny_camera(37, 29, eye=(0.3, 0.2, -4.0))], [0, 1]),
    ]
    for sc, cams, cam_scene in frames:
        dev = [R.scene_to_device(s) for s in sc]
        ref = rast.forward(dev, cams, cam_scene=cam_scene, tile=tile)
        for _ in range(2):
            st, rgb, depth, alpha = _noalloc(rast, dev, cams, cam_scene, tile)
            assert st == L.GB_OK, L.load().gb_last_error(rast.ctx).decode()
            torch.cuda.synchronize()
            # same kernels on the same inputs in the same order: identical bits
            for a, b in zip((rgb, depth, alpha), ref[:3]):
                assert torch.equal(a, b), (a - b).abs().max().item()


def test_noalloc_forward_refuses_frames_beyond_its_limits():
    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(scenes.tiny_scene(5, K=4))]
    big = scenes.tiny_camera(1100, 1000)  # 1,100,000 pixels > 1,048,576
    st, _, _, _ = _noalloc(rast, dev, [big], [0])
    assert st == 4  # GB_ERR_CAPACITY
    assert "limits" in L.load().gb_last_error(rast.ctx).decode()


def test_noalloc_forward_refuses_too_many_instances_then_renders():
    """200 fronto-parallel splats that each cover all 4,096 tiles of a
    1024 x 1024 view make 819,200 (tile, splat) instances, past the array's
    524,288: GB_ERR_CAPACITY with a message, and the next call renders a
    normal frame bit for bit like the allocating forward."""
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    K = 200
    big = {
        "means": np.zeros((K, 3), np.float32), "quats": np.tile(np.array([1, 0, 0, 0], np.float32), (K, 1)),
        "scales": np.ones((K, 2), np.float32), "opacities": np.full(K, 0.5, np.float32),
        "sh": np.full((K, 1, 3), 0.5, np.float32), "textures": np.full((K, 1, 1, 3), 0.25, np.float32),
        "sh_degree": 0, "tex_n": 1, "sigma": 0.5,
    }
    rast = R.Rasterizer(0)
    cam = scenes.look_at([0.0, 0.0, -2.0], [0, 0, 0], 1024, 1024)
    st, _, _, _ = _noalloc(rast, [R.scene_to_device(big)], [cam], [0])
    assert st == 4  # GB_ERR_CAPACITY
    assert "instances" in L.load().gb_last_error(rast.ctx).decode()
    sc = scenes.tiny_scene(7, K=12, tex_n=4, sh_degree=2)
    cams = [scenes.tiny_camera(40, 24)]
    dev = [R.scene_to_device(sc)]
    ref = rast.forward(dev, cams)
    st, rgb, depth, alpha = _noalloc(rast, dev, cams, [0])
    assert st == L.GB_OK, L.load().gb_last_error(rast.ctx).decode()
    torch.cuda.synchronize()
    for a, b in zip((rgb, depth, alpha), ref[:3]):
        assert torch.equal(a, b)


def test_noalloc_forward_refuses_mip_level_scenes():
    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    sc = scenes.tiny_scene(6, K=4, tex_n=4)
    sc["mip_level"] = 1
    st, _, _, _ = _noalloc(rast, [R.scene_to_device(sc)], [scenes.tiny_camera(16, 16)], [0])
    assert st == 2  # GB_ERR_UNSUPPORTED
    assert "mip" in L.load().gb_last_error(rast.ctx).decode()
