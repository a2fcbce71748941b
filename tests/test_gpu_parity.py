"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Keys are compared bit for bit; rgb and alpha within 2e-5 max abs error;
depth within 2e-5 relative to max(1, |depth|); gradients per element within
1e-3 of max(|g*|, 1e-2 max|g*|) (relative above 1 % of the tensor's largest
entry, absolute 1e-5 of it below).  Pixels whose decisions sit within the
oracle's margin of a threshold are excluded from image errors (and counted)
and get zero upstream gradient on both sides.
"""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes
from tests.gpu_util import (GRAD_REL, IMG_TOL, compare_images, gpu_run, grad_errors, masked_upstream,
                            oracle_run)

pytestmark = pytest.mark.gpu


def _tile_offsets(cams, tile=16):
    offs, o = [], 0
    for c in cams:
        offs.append(o)
        o += -(-int(c["width"]) // tile) * -(-int(c["height"]) // tile)
    return offs


def _check_keys(scene_list, cams, cam_scene, gpu, tile=16):
    keys, ids, cidx = gpu["keys"]
    offs = _tile_offsets(cams, tile)
    exp_k, exp_i, exp_c = [], [], []
    for ci, c in enumerate(cams):
        k, i = oracle.tile_keys(scene_list[cam_scene[ci]], c, tile, offs[ci])
        exp_k.append(k)
        exp_i.append(i)
        exp_c.append(np.full(len(k), ci))
    ek, ei = np.concatenate(exp_k), np.concatenate(exp_i)
    assert len(keys) == len(ek), (len(keys), len(ek))
    assert np.array_equal(keys, ek)
    assert np.array_equal(ids, ei)
    assert np.array_equal(cidx, np.concatenate(exp_c))


CASES = {
    "plain_1k": lambda: (scenes.workload("plain_1k")["scenes"], scenes.workload("plain_1k")["cams"]),
    "tiny_n1_d0": lambda: ([scenes.tiny_scene(1, K=6, tex_n=1, sh_degree=0)], [scenes.tiny_camera(40, 24)]),
    "tiny_n2_d3": lambda: ([scenes.tiny_scene(2, K=6, tex_n=2, sh_degree=3)], [scenes.tiny_camera(37, 29)]),
    "tiny_n4_d3": lambda: ([scenes.tiny_scene(3, K=8, tex_n=4, sh_degree=3)], [scenes.tiny_camera(48, 33)]),
    "tiny_n8_d2": lambda: ([scenes.tiny_scene(4, K=8, tex_n=8, sh_degree=2)], [scenes.tiny_camera(50, 50)]),
    "tiny_n16_d1": lambda: ([scenes.tiny_scene(14, K=8, tex_n=16, sh_degree=1, tex_dtype="f16")],
                            [scenes.tiny_camera(56, 44)]),
    "tiny_n4_sigma2": lambda: ([scenes.tiny_scene(5, K=8, tex_n=4, sh_degree=1, sigma=2.0)],
                               [scenes.tiny_camera(33, 47)]),
    "tiny_f16": lambda: ([scenes.tiny_scene(6, K=8, tex_n=4, sh_degree=3, sh_dtype="f16", tex_dtype="f16")],
                         [scenes.tiny_camera(40, 40)]),
    "tiny_bf16": lambda: ([scenes.tiny_scene(7, K=8, tex_n=8, sh_degree=3, sh_dtype="bf16", tex_dtype="bf16")],
                          [scenes.tiny_camera(40, 40)]),
    "planes_2k": lambda: ([scenes.planes_scene(8, K=2000, tex_n=4, log_scale=(-3.0, 0.6))],
                          [scenes.look_at([0.5, 1.0, -8.0], [0, 0, 0], 160, 90)]),
    "dense_many_tiles": lambda: ([scenes.cube_scene(9, K=3000, half=1.0, log_scale=(-2.3, 0.4), sh_degree=3,
                                                    tex_n=4)],
                                [scenes.look_at([0.0, 0.0, -3.5], [0, 0, 0], 200, 136)]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_keys_bit_exact(case):
    sc, cams = CASES[case]()
    gpu = gpu_run(sc, cams, keys=True)
    _check_keys(sc, cams, [0] * len(cams), gpu)


@pytest.mark.parametrize("case", list(CASES))
def test_image_parity(case):
    sc, cams = CASES[case]()
    bg = np.array([0.25, 0.5, 0.75], np.float32) if "tiny" in case else None
    gpu = gpu_run(sc, cams, bg=bg)
    ref = oracle_run(sc[0], cams[0], bg=bg)
    e_rgb, excl = compare_images(gpu["rgb"][0], ref, "rgb")
    e_a, _ = compare_images(gpu["alpha"][0], ref, "alpha")
    e_d, _ = compare_images(gpu["depth"][0], ref, "depth", relative_to=ref["depth"])
    n = ref["rgb"].shape[0] * ref["rgb"].shape[1]
    assert excl <= max(2, 0.01 * n), f"{excl} of {n} pixels near a decision threshold"
    assert e_rgb <= IMG_TOL, f"rgb max err {e_rgb:.3e}"
    assert e_a <= IMG_TOL, f"alpha max err {e_a:.3e}"
    assert e_d <= IMG_TOL, f"depth max rel err {e_d:.3e}"


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kernel", ["pixel", "splat"])
def test_gradient_parity(case, kernel):
    """Both backward loops: pixel-parallel (a lane per pixel, warp reductions
    per splat) and splat-parallel (a lane per splat, prefix scans over the
    splats; grids of N <= 4)."""
    sc, cams = CASES[case]()
    if kernel == "splat" and int(sc[0]["tex_n"]) > 4:
        pytest.skip("the splat-parallel backward takes grids of N <= 4")
    rng = np.random.default_rng(11)
    ref = oracle_run(sc[0], cams[0])
    d_rgb = masked_upstream(ref, rng)
    use_da = case in ("tiny_n4_d3", "tiny_n8_d2", "planes_2k")
    d_dep = masked_upstream(ref, rng, 1, 0.3)[..., 0] if use_da else None
    d_alp = masked_upstream(ref, rng, 1)[..., 0] if use_da else None
    gpu = gpu_run(sc, cams, d_rgb=[d_rgb], d_depth=[d_dep] if use_da else None,
                  d_alpha=[d_alp] if use_da else None, **({"ppt": 1} if kernel == "pixel" else {"bwd_kernel": 2}))
    og = oracle.backward(sc[0], cams[0], d_rgb, d_dep, d_alp)
    errs = grad_errors(gpu["grads"][0], og)
    bad = {k: v for k, v in errs.items() if v > 1.0}
    assert not bad, f"gradient ratios over tolerance {GRAD_REL}: {errs}"


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("tile", [16, 8])
def test_gradient_parity_two_pixels_per_thread(case, tile):
    """Backward with two pixels of a column per thread (packed FP32x2 pipe)."""
    sc, cams = CASES[case]()
    rng = np.random.default_rng(23)
    ref = oracle_run(sc[0], cams[0])
    d_rgb = masked_upstream(ref, rng)
    d_dep = masked_upstream(ref, rng, 1, 0.3)[..., 0]
    d_alp = masked_upstream(ref, rng, 1)[..., 0]
    gpu = gpu_run(sc, cams, d_rgb=[d_rgb], d_depth=[d_dep], d_alpha=[d_alp], tile=tile, ppt=2,
                  bg=np.array([0.2, 0.1, 0.4], np.float32))
    og = oracle.backward(sc[0], cams[0], d_rgb, d_dep, d_alp, bg=np.array([0.2, 0.1, 0.4], np.float32))
    errs = grad_errors(gpu["grads"][0], og)
    assert all(v <= 1.0 for v in errs.values()), errs


@pytest.mark.parametrize("case", ["plain_1k", "tiny_n4_d3", "tiny_bf16", "dense_many_tiles", "tiny_n16_d1"])
@pytest.mark.parametrize("tile", [8, 32])
def test_tile8_tile32_keys_image_gradients(case, tile):
    """8 x 8 and 32 x 32 tiles: the same keys formula with that tile edge, the
    same image and gradients."""
    sc, cams = CASES[case]()
    rng = np.random.default_rng(17)
    ref = oracle_run(sc[0], cams[0])
    d_rgb = masked_upstream(ref, rng)
    gpu = gpu_run(sc, cams, d_rgb=[d_rgb], keys=True, tile=tile)
    _check_keys(sc, cams, [0], gpu, tile=tile)
    e, _ = compare_images(gpu["rgb"][0], ref, "rgb")
    assert e <= IMG_TOL, e
    errs = grad_errors(gpu["grads"][0], oracle.backward(sc[0], cams[0], d_rgb))
    assert all(v <= 1.0 for v in errs.values()), errs


def test_autotune_picks_a_valid_candidate(tmp_path):
    from paper_2412_12734_gb300 import render as R
    sc, cams = CASES["dense_many_tiles"]()
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in sc]
    res = rast.autotune(dev, cams, reps=2, cache=str(tmp_path / "tune.json"))
    # the splat-parallel backward, when it wins, is listed with ppt 3
    sp = res["bwd_kernel"] == 2
    assert res["tile"] in (8, 16, 32) and 8 <= res["batch"] <= 256 and res["batch"] % 8 == 0
    assert len(res["candidates"]) >= 4
    both = [c for c in res["candidates"] if c["ppt"] > 0]
    best = min(both, key=lambda c: c["ms"])
    assert (best["tile"], best["batch"], best["ppt"]) == (res["tile"], res["batch"], 3 if sp else res["ppt"])
    # the second stage times the forward alone at the chosen tile (listed with ppt 0)
    fwd = [c for c in res["candidates"] if c["ppt"] == 0]
    assert fwd and all(c["tile"] == res["tile"] for c in fwd)
    assert min(fwd, key=lambda c: c["ms"])["batch"] == res["batch_fwd"]
    again = rast.autotune(dev, cams, reps=2, cache=str(tmp_path / "tune.json"))
    assert again == res  # served from the cache
    rgb, _, _, _ = rast.forward(dev, cams, tile=res["tile"], batch=res["batch"], batch_fwd=res["batch_fwd"],
                                bwd_kernel=res["bwd_kernel"])
    ref = oracle_run(sc[0], cams[0])
    e, _ = compare_images(rgb.cpu().numpy().reshape(ref["rgb"].shape), ref, "rgb")
    assert e <= IMG_TOL


def test_mixed_texture_sizes_and_storage_in_one_frame():
    """Scenes with different grid sizes and storage types share one forward and
    backward (one render launch per (N, dtype) group over a device tile list)."""
    sl = [scenes.tiny_scene(31, K=6, tex_n=2, sh_degree=1, sh_dtype="f16", tex_dtype="f16"),
          scenes.tiny_scene(32, K=7, tex_n=8, sh_degree=3, sh_dtype="bf16", tex_dtype="bf16"),
          scenes.tiny_scene(33, K=5, tex_n=4, sh_degree=2)]
    cams = [scenes.tiny_camera(40, 24), scenes.tiny_camera(33, 31, eye=(0.4, 0.1, -4.0)),
            scenes.tiny_camera(24, 40, eye=(-0.3, 0.2, -4.2)), scenes.tiny_camera(17, 17)]
    cam_scene = [1, 0, 2, 1]
    rng = np.random.default_rng(8)
    refs = [oracle_run(sl[cam_scene[i]], c) for i, c in enumerate(cams)]
    d_rgb = [masked_upstream(r, rng) for r in refs]
    gpu = gpu_run(sl, cams, cam_scene=cam_scene, d_rgb=d_rgb, keys=True)
    _check_keys(sl, cams, cam_scene, gpu)
    for i, r in enumerate(refs):
        e, _ = compare_images(gpu["rgb"][i], r, "rgb")
        assert e <= IMG_TOL, (i, e)
    for si in range(3):
        og = None
        for i, c in enumerate(cams):
            if cam_scene[i] == si:
                og = oracle.backward(sl[si], c, d_rgb[i], grads=og)
        errs = grad_errors(gpu["grads"][si], og)
        assert all(v <= 1.0 for v in errs.values()), (si, errs)


@pytest.mark.parametrize("tile", [16, 8])
def test_persistent_render_matches_one_block_per_tile(tile):
    """Persistent blocks pulling tiles (largest first) from a device counter
    give the same image bit for bit and the same gradients up to atomic order."""
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    sc, cams = CASES["dense_many_tiles"]()
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in sc]
    d = torch.randn((cams[0]["width"] * cams[0]["height"], 3), device="cuda")
    a = rast.forward(dev, cams, tile=tile)
    ga = rast.backward(a[3], d)[0]
    b = rast.forward(dev, cams, tile=tile, flags=L.GB_FLAG_PERSISTENT)
    gb = rast.backward(b[3], d)[0]
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    for k in ga:
        scale = ga[k].abs().max().item()
        assert (ga[k] - gb[k]).abs().max().item() <= 1e-5 * max(scale, 1e-12), k



@pytest.mark.parametrize("tex_n", [2, 4, 8])
@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
def test_grids_at_an_unaligned_address_render_the_same(tex_n, dtype):
    """Colour grids are staged four texels at a time with 64-bit loads (16-bit
    storage, array 8-byte aligned) or 128-bit loads (FP32, 16-byte aligned),
    texel by texel otherwise: grids stored one element past an aligned
    address give the same image bit for bit and the same gradients up to
    atomic order (the forward at N = 2, 4 converts 16-bit grids to FP32 at
    staging, larger grids stay 16-bit)."""
    import torch

    from paper_2412_12734_gb300 import render as R
    sc = scenes.tiny_scene(31, K=30, tex_n=tex_n, spread=0.8, tex_dtype=dtype)
    cams = [scenes.tiny_camera(72, 56)]
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(sc)
    tex = dev["textures"]
    buf = torch.empty(tex.numel() + 1, dtype=tex.dtype, device="cuda")
    buf[1:] = tex.reshape(-1)
    shifted = dict(dev, textures=buf[1:].view(tex.shape))
    assert shifted["textures"].data_ptr() % 16 == tex.element_size()
    d = torch.randn((72 * 56, 3), device="cuda")
    a = rast.forward([dev], cams)
    ga = rast.backward(a[3], d)[0]
    b = rast.forward([shifted], cams)
    gb = rast.backward(b[3], d)[0]
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    for k in ga:
        scale = ga[k].abs().max().item()
        assert (ga[k] - gb[k]).abs().max().item() <= 1e-5 * max(scale, 1e-12), k


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
def test_sh_at_an_unaligned_address_renders_the_same(dtype):
    """Degree-3 SH coefficients are read 16 bytes at a time when the array is
    16-byte aligned, one value at a time otherwise: coefficients stored one
    element past an aligned address give the same image and gradients up to
    the rounding order of the colour sum and atomic order."""
    import torch

    from paper_2412_12734_gb300 import render as R
    sc = scenes.tiny_scene(34, K=30, tex_n=4, sh_degree=3, spread=0.8, sh_dtype=dtype)
    cams = [scenes.tiny_camera(72, 56)]
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(sc)
    sh = dev["sh"]
    buf = torch.empty(sh.numel() + 1, dtype=sh.dtype, device="cuda")
    buf[1:] = sh.reshape(-1)
    shifted = dict(dev, sh=buf[1:].view(sh.shape))
    assert shifted["sh"].data_ptr() % 16 == sh.element_size()
    d = torch.randn((72 * 56, 3), device="cuda")
    a = rast.forward([dev], cams)
    ga = rast.backward(a[3], d)[0]
    b = rast.forward([shifted], cams)
    gb = rast.backward(b[3], d)[0]
    for x, y in zip(a[:3], b[:3]):
        assert (x - y).abs().max().item() <= 1e-6
    for k in ga:
        scale = ga[k].abs().max().item()
        assert (ga[k] - gb[k]).abs().max().item() <= 1e-5 * max(scale, 1e-12), k


@pytest.mark.parametrize("tex_n", [2, 4, 8, 16])
def test_backward_without_a_texture_gradient_output(tex_n):
    """The texture-gradient output may be left out (null): the backward skips
    every texel atomic and gives the other gradients as with it, up to
    atomic order."""
    import torch

    from paper_2412_12734_gb300 import render as R
    sc = scenes.tiny_scene(33, K=30, tex_n=tex_n, spread=0.8, tex_dtype="f16")
    cams = [scenes.tiny_camera(72, 56)]
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(sc)
    d = torch.randn((72 * 56, 3), device="cuda")
    saved = rast.forward([dev], cams)[3]
    full = rast.backward(saved, d)[0]
    part = {k: torch.empty_like(v) for k, v in full.items() if k != "textures"}
    rast.backward(saved, d, grads=[part])
    for k, v in part.items():
        scale = full[k].abs().max().item()
        assert (v - full[k]).abs().max().item() <= 1e-5 * max(scale, 1e-12), k


@pytest.mark.parametrize("flags", [0, 2])
def test_second_backward_after_one_forward_gives_the_same_gradients(flags):
    """A forward may be followed by several backwards (other upstream
    gradients, or the same again): each starts from zeroed accumulators and,
    with persistent blocks (flag 2), from a fresh tile counter."""
    import torch

    from paper_2412_12734_gb300 import render as R
    sc, cams = CASES["dense_many_tiles"]()
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in sc]
    d = torch.randn((cams[0]["width"] * cams[0]["height"], 3), device="cuda")
    ref = rast.backward(rast.forward(dev, cams)[3], d)[0]
    saved = rast.forward(dev, cams, flags=flags)[3]
    g1 = {k: v.clone() for k, v in rast.backward(saved, d)[0].items()}
    g2 = rast.backward(saved, d)[0]
    for k in ref:
        scale = ref[k].abs().max().item()
        assert (g1[k] - ref[k]).abs().max().item() <= 1e-5 * scale, k
        assert (g2[k] - ref[k]).abs().max().item() <= 1e-5 * scale, k

@pytest.mark.parametrize("flags", [0, 2])
def test_reserve_between_forward_and_backward_keeps_the_forward(flags):
    """A reserve that grows every buffer group (records, instances, pixels,
    tiles) between a synchronizing forward and its backward moves the recorded
    forward with the buffers: the backward equals the same forward's backward
    without the reserve (flag 2: persistent blocks, which also read the tile
    list)."""
    import torch

    from paper_2412_12734_gb300 import render as R
    sc, cams = CASES["dense_many_tiles"]()
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in sc]
    P = rast.pixel_count(cams)
    d = torch.randn((P, 3), device="cuda")
    ref = rast.backward(rast.forward(dev, cams, flags=flags)[3], d)[0]
    saved = rast.forward(dev, cams, flags=flags)[3]
    st = saved.stats()
    saved.reserve(4 * st["records"] + 4096, 4 * st["capacity"], 4 * P, 4 * st["tiles"])
    after = saved.stats()
    assert after["capacity"] > st["capacity"]
    assert after["instances"] == st["instances"]
    g = rast.backward(saved, d)[0]
    torch.cuda.synchronize()
    for k in ref:
        scale = ref[k].abs().max().item()
        assert (g[k] - ref[k]).abs().max().item() <= 1e-5 * max(scale, 1e-12), k


def test_graph_replay_with_new_parameters_matches_eager():
    """A no-sync forward and backward captured in a CUDA graph, replayed after
    the splat parameters were overwritten in place (other centres and sizes:
    another visible set and instance count), equals an eager render of the new
    parameters: images bit for bit, gradients up to the order of atomics."""
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    sc, cams = CASES["dense_many_tiles"]()
    a = sc[0]
    rng = np.random.default_rng(11)
    b = dict(a)
    b["means"] = a["means"] + rng.normal(0.0, 0.15, a["means"].shape)
    b["scales"] = a["scales"] * rng.uniform(0.7, 1.4, a["scales"].shape)
    b["opacities"] = rng.permutation(a["opacities"])
    rast = R.Rasterizer(0)
    da, db = R.scene_to_device(a), R.scene_to_device(b)
    P = rast.pixel_count(cams)
    d = torch.randn((P, 3), device="cuda")
    ref = rast.forward([db], cams)
    gref = rast.backward(ref[3], d)[0]
    sizes = [ref[3].stats(), rast.forward([da], cams)[3].stats()]
    saved = R.Saved(rast)
    saved.reserve(max(s["records"] for s in sizes), 2 * max(s["instances"] for s in sizes) + 1024, P,
                  sizes[0]["tiles"])
    out = (torch.empty((P, 3), device="cuda"), torch.empty(P, device="cuda"), torch.empty(P, device="cuda"))
    rast.forward([da], cams, saved=saved, out=out, flags=L.GB_FLAG_NO_SYNC)
    grads = rast.backward(saved, d)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rast.forward([da], cams, saved=saved, out=out, flags=L.GB_FLAG_NO_SYNC)
        rast.backward(saved, d, grads=grads)
    for k in ("means", "quats", "scales", "opacities", "sh", "textures"):
        da[k].copy_(db[k])
    graph.replay()
    torch.cuda.synchronize()
    saved.check()
    assert saved.stats()["instances"] == sizes[0]["instances"]
    for x, y in zip(out, ref[:3]):
        assert torch.equal(x, y)
    for k, v in gref.items():
        scale = v.abs().max().item()
        assert (grads[0][k] - v).abs().max().item() <= 1e-5 * max(scale, 1e-12), k

@pytest.mark.parametrize("flags", [0, 2])
def test_batched_renderer_replays_match_eager_calls(flags):
    """BatchedRenderer over two scenes of uneven splat counts and three views of
    uneven sizes (flag 2: one persistent launch per pass): graph replays equal
    eager calls, also after the splat parameters changed in place, and a
    repeated backward gives the same gradients."""
    import torch

    from paper_2412_12734_gb300 import render as R
    big = CASES["dense_many_tiles"]()
    a0, a1 = big[0][0], scenes.tiny_scene(22, K=5, tex_n=4, sh_degree=1)
    cams = [big[1][0], scenes.tiny_camera(17, 33, eye=(0.5, 0.2, -4.0)), scenes.tiny_camera(40, 24)]
    cam_scene = [0, 1, 1]
    rng = np.random.default_rng(12)
    b0 = dict(a0)
    b0["means"] = a0["means"] + rng.normal(0.0, 0.15, a0["means"].shape)
    b0["scales"] = a0["scales"] * rng.uniform(0.7, 1.4, a0["scales"].shape)
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(a0), R.scene_to_device(a1)]
    br = R.BatchedRenderer(rast, dev, cams, cam_scene=cam_scene, flags=flags, headroom=3.0)
    d = torch.randn((br.P, 3), device="cuda")

    def eager(scene_list):
        o = rast.forward(scene_list, cams, cam_scene=cam_scene, flags=flags)
        return o[:3], rast.backward(o[3], d)

    def compare(ref):
        out = br.forward()
        grads = br.backward(d)
        torch.cuda.synchronize()
        br.check()
        for x, y in zip(out, ref[0]):
            assert torch.equal(x, y)
        for gs, gr in zip(grads, ref[1]):
            for k, v in gr.items():
                scale = v.abs().max().item()
                assert (gs[k] - v).abs().max().item() <= 1e-5 * max(scale, 1e-12), k

    compare(eager(dev))
    db = R.scene_to_device(b0)
    for k in ("means", "scales"):
        dev[0][k].copy_(db[k])
    ref_b = eager(dev)
    compare(ref_b)
    again = br.backward()
    torch.cuda.synchronize()
    for gs, gr in zip(again, ref_b[1]):
        for k, v in gr.items():
            scale = v.abs().max().item()
            assert (gs[k] - v).abs().max().item() <= 1e-5 * max(scale, 1e-12), k

def test_multi_view_multi_scene():
    """Two scenes, four cameras of different sizes in one launch: per-camera
    keys and images, and gradients summed over each scene's cameras."""
    s0 = scenes.tiny_scene(21, K=7, tex_n=4, sh_degree=3)
    s1 = scenes.tiny_scene(22, K=5, tex_n=4, sh_degree=1)
    cams = [scenes.tiny_camera(40, 24), scenes.tiny_camera(17, 33, eye=(0.5, 0.2, -4.0)),
            scenes.tiny_camera(64, 48, focal=45.0, eye=(-0.7, 0.4, -4.5)), scenes.tiny_camera(16, 16)]
    cam_scene = [0, 1, 0, 1]
    sl = [s0, s1]
    rng = np.random.default_rng(5)
    refs = [oracle_run(sl[cam_scene[i]], c) for i, c in enumerate(cams)]
    d_rgb = [masked_upstream(r, rng) for r in refs]
    gpu = gpu_run(sl, cams, cam_scene=cam_scene, d_rgb=d_rgb, keys=True)
    _check_keys(sl, cams, cam_scene, gpu)
    for i, r in enumerate(refs):
        e, _ = compare_images(gpu["rgb"][i], r, "rgb")
        assert e <= IMG_TOL, (i, e)
    for s in range(2):
        og = None
        for i, c in enumerate(cams):
            if cam_scene[i] == s:
                og = oracle.backward(sl[s], c, d_rgb[i], grads=og)
        errs = grad_errors(gpu["grads"][s], og)
        assert all(v <= 1.0 for v in errs.values()), (s, errs)


def test_plain_100k_full_frame():
    """100,000 planar + clutter splats, SH degree 3, 8x8 FP32 textures, one
    1280x720 camera: full-frame keys, image and gradients against the oracle
    (bbox-prefiltered mode, identical to brute force)."""
    w = scenes.workload("plain_100k")
    sc, cam = w["scenes"][0], w["cams"][0]
    ref = oracle_run(sc, cam, prefilter=True)
    rng = np.random.default_rng(3)
    d_rgb = masked_upstream(ref, rng)
    gpu = gpu_run([sc], [cam], d_rgb=[d_rgb], keys=True)
    _check_keys([sc], [cam], [0], gpu)
    e_rgb, excl = compare_images(gpu["rgb"][0], ref, "rgb")
    assert excl <= 0.001 * 921600, excl
    assert e_rgb <= IMG_TOL, e_rgb
    og = oracle.backward(sc, cam, d_rgb, prefilter=True)
    errs = grad_errors(gpu["grads"][0], og)
    assert all(v <= 1.0 for v in errs.values()), errs


# ------------------------------------------------------------------ edge cases --

def test_empty_and_culled_scenes():
    """K = 0, and every splat behind the camera: images equal the background,
    no instances, zero gradients."""
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    cam = scenes.tiny_camera(20, 12)
    empty = scenes.subset(scenes.tiny_scene(1, K=3), np.arange(0))
    behind = scenes.tiny_scene(2, K=4)
    behind["means"][:, 2] = -6.0  # camera at z = -4 looking at +z
    for sc in (empty, behind):
        d_rgb = np.ones((12, 20, 3))
        gpu = gpu_run([sc], [cam], bg=bg, d_rgb=[d_rgb])
        assert gpu["stats"]["instances"] == 0
        np.testing.assert_array_equal(gpu["rgb"][0], np.broadcast_to(bg, (12, 20, 3)))
        np.testing.assert_array_equal(gpu["alpha"][0], 0.0)
        for v in gpu["grads"][0].values():
            assert np.all(v == 0)


def test_one_pixel_and_degenerate_quaternion():
    sc = scenes.tiny_scene(4, K=5)
    sc["quats"][2] = 0.0  # zero quaternion: culled on both sides
    for cam in (scenes.tiny_camera(1, 1, focal=2.0), scenes.tiny_camera(7, 3)):
        gpu = gpu_run([sc], [cam], keys=True)
        _check_keys([sc], [cam], [0], gpu)
        ref = oracle_run(sc, cam)
        e, _ = compare_images(gpu["rgb"][0], ref, "rgb")
        assert e <= IMG_TOL


@pytest.mark.parametrize("tile,batch,batch_fwd", [(16, 32, 0), (8, 64, 0), (16, 128, 0), (32, 8, 0), (16, 8, 128),
                                                 (16, 88, 16), (8, 16, 64)])
def test_batch_depth_does_not_change_results(tile, batch, batch_fwd):
    """Images are the same bit for bit at any batch depth, including batches
    deeper than the forward block's threads (tile 8: 32 threads, two pixels
    each) that stage two or more splats per thread, and with the forward's
    depth set apart from the backward's; gradients agree up to the order of
    atomics."""
    sc, cams = CASES["dense_many_tiles"]()
    rng = np.random.default_rng(41)
    d_rgb = rng.standard_normal((int(cams[0]["height"]), int(cams[0]["width"]), 3)).astype(np.float32)
    a = gpu_run(sc, cams, d_rgb=[d_rgb], tile=tile, batch=batch, batch_fwd=batch_fwd)
    b = gpu_run(sc, cams, d_rgb=[d_rgb], tile=tile, batch=0)
    np.testing.assert_array_equal(a["rgb"][0], b["rgb"][0])
    np.testing.assert_array_equal(a["depth"][0], b["depth"][0])
    for k in a["grads"][0]:
        x, y = a["grads"][0][k], b["grads"][0][k]
        assert np.abs(x - y).max() <= 2e-5 * max(np.abs(y).max(), 1e-12), k


def test_invalid_arguments_are_rejected():
    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    dev = R.scene_to_device(scenes.tiny_scene(1, K=3, tex_n=4))
    cam = scenes.tiny_camera(8, 8)
    bad = dict(dev)
    bad["tex_n"] = 3
    bad["textures"] = torch.zeros((3, 3, 3, 3), device="cuda")
    with pytest.raises(L.GbillError) as ei:
        rast.forward([bad], [cam])
    assert ei.value.status == 2
    bad_cam = dict(cam)
    bad_cam["width"] = 0
    with pytest.raises(L.GbillError) as ei:
        rast.forward([dev], [bad_cam])
    assert ei.value.status == 1
    nan_cam = dict(cam)
    nan_cam["fx"] = float("nan")
    with pytest.raises(L.GbillError) as ei:
        rast.forward([dev], [nan_cam])
    assert ei.value.status == 6
    with pytest.raises(L.GbillError) as ei:
        rast.forward([dev], [cam], batch=36)  # not a multiple of 8
    assert ei.value.status == 1
    with pytest.raises(L.GbillError) as ei:
        rast.forward([dev], [cam], batch_fwd=36)
    assert ei.value.status == 1
    with pytest.raises(L.GbillError) as ei:
        rast.forward([dev], [cam], tile=8, batch=16, batch_fwd=128)  # deeper than the tile's 64 pixels
    assert ei.value.status == 1


def test_no_sync_capacity_overflow_is_reported():
    """No-sync mode never allocates: too small a reservation is flagged on the
    device and reported by gb_saved_check; a large enough one matches eager."""
    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    sc, cams = CASES["dense_many_tiles"]()
    rast = R.Rasterizer(0)
    dev = [R.scene_to_device(s) for s in sc]
    ref_rgb, _, _, saved0 = rast.forward(dev, cams)
    need = saved0.stats()["instances"]
    P = rast.pixel_count(cams)
    tiles = -(-cams[0]["width"] // 16) * -(-cams[0]["height"] // 16)
    small = R.Saved(rast)
    small.reserve(3000, max(16, need // 4), P, tiles)
    rast.forward(dev, cams, saved=small, flags=L.GB_FLAG_NO_SYNC)
    with pytest.raises(L.GbillError) as ei:
        small.check()
    assert ei.value.status == 4
    big = R.Saved(rast)
    big.reserve(3000, need, P, tiles)
    rgb, _, _, _ = rast.forward(dev, cams, saved=big, flags=L.GB_FLAG_NO_SYNC)
    big.check()
    assert np.array_equal(rgb.cpu().numpy(), ref_rgb.cpu().numpy())


def test_frame_beyond_the_32bit_instance_range_is_refused():
    """600,000 fronto-parallel splats that each cover all 8,160 tiles of a
    1920x1080 view make 4.9e9 (tile, splat) instances, past the 32-bit
    instance index: the synchronizing forward reports GB_ERR_CAPACITY from
    the device count (which must not wrap) before it allocates the list, and
    the context renders the next frame normally."""
    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    K = 600_000
    big = {
        "means": np.zeros((K, 3), np.float32), "quats": np.tile(np.array([1, 0, 0, 0], np.float32), (K, 1)),
        "scales": np.ones((K, 2), np.float32), "opacities": np.full(K, 0.5, np.float32),
        "sh": np.full((K, 1, 3), 0.5, np.float32), "textures": np.full((K, 1, 1, 3), 0.25, np.float32),
        "sh_degree": 0, "tex_n": 1, "sigma": 0.5,
    }
    cam = scenes.look_at([0.0, 0.0, -2.0], [0, 0, 0], 1920, 1080)
    rast = R.Rasterizer(0)
    with pytest.raises(L.GbillError) as ei:
        rast.forward([R.scene_to_device(big)], [cam])
    assert ei.value.status == 4
    sc, cams = CASES["tiny_n4_d3"]()
    rgb = rast.forward([R.scene_to_device(sc[0])], cams)[0]
    e, _ = compare_images(rgb.cpu().numpy().reshape(cams[0]["height"], cams[0]["width"], 3),
                          oracle_run(sc[0], cams[0]), "rgb")
    assert e <= IMG_TOL

def test_non_finite_splats_are_culled_and_reported():
    """A splat with a NaN centre, one with an infinite scale and one with a
    NaN SH coefficient are culled in every camera; the rest of the frame
    equals the oracle's render without them, and gb_saved_check reports
    GB_ERR_NONFINITE."""
    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    sc = scenes.tiny_scene(95, K=9, tex_n=4, sh_degree=2)
    bad = dict(sc)
    bad["means"] = sc["means"].copy()
    bad["scales"] = sc["scales"].copy()
    bad["sh"] = sc["sh"].copy()
    bad["quats"] = sc["quats"].copy()
    bad["means"][2, 1] = np.nan
    bad["scales"][5, 0] = np.inf
    bad["sh"][7, 3, 1] = np.nan
    bad["quats"][8, 0] = np.nan
    keep = np.array([i for i in range(9) if i not in (2, 5, 7, 8)])
    cam = scenes.tiny_camera(40, 32)
    rast = R.Rasterizer(0)
    rgb, _, _, saved = rast.forward([R.scene_to_device(bad)], [cam])
    with pytest.raises(L.GbillError) as ei:
        saved.check()
    assert ei.value.status == 6
    ref = oracle_run(scenes.subset(sc, keep), cam)
    e, _ = compare_images(rgb.cpu().numpy().reshape(32, 40, 3), ref, "rgb")
    assert e <= IMG_TOL, e
    import torch
    g = rast.backward(saved, torch.ones((32 * 40, 3), device="cuda"))[0]
    for k, v in g.items():
        assert torch.isfinite(v).all(), k
        assert (v[[2, 5, 7, 8]] == 0).all(), k
