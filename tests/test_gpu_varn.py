"""Per-splat grid sizes on the GPU (the variable texture resolution of Sec. 3.3
and 5): splat k's n_k x n_k grid in rows and columns 0..n_k-1 of its N x N
block, sampled by Alg. 2 with n_k; the texels outside are set to a value the
kernels must never read.  Images and gradients against the FP64 oracle at the
stated bars, forward bit-identity with the uniform scene when every n_k = N,
a frame mixing a per-splat scene with a uniform one, and the options the path
does not take."""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes
from tests.gpu_util import IMG_TOL, compare_images, gpu_run, grad_errors, masked_upstream, oracle_run

pytestmark = pytest.mark.gpu

CASES = {
    "n4_f32": lambda: (scenes.with_splat_tex_n(scenes.tiny_scene(31, K=10, tex_n=4, sh_degree=2), [1, 2, 3, 4], seed=1),
                       scenes.tiny_camera(48, 36)),
    "n8_f16": lambda: (scenes.with_splat_tex_n(scenes.tiny_scene(32, K=10, tex_n=8, sh_degree=3, sh_dtype="f16",
                                                                 tex_dtype="f16"), [1, 2, 4, 5, 8], seed=2),
                       scenes.tiny_camera(50, 42)),
    "n16_bf16": lambda: (scenes.with_splat_tex_n(scenes.tiny_scene(33, K=8, tex_n=16, sh_degree=1, tex_dtype="bf16"),
                                                 [2, 4, 8, 11, 16], seed=3),
                         scenes.tiny_camera(44, 40)),
    "planes_n8": lambda: (scenes.with_splat_tex_n(scenes.planes_scene(34, K=3000, tex_n=8, log_scale=(-3.0, 0.6)),
                                                  [1, 2, 4, 8], seed=4),
                          scenes.look_at([0.5, 1.0, -8.0], [0, 0, 0], 160, 90)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_per_splat_grid_sizes_match_the_oracle(case):
    sc, cam = CASES[case]()
    ref = oracle_run(sc, cam)
    rng = np.random.default_rng(5)
    d = masked_upstream(ref, rng)
    gpu = gpu_run([sc], [cam], d_rgb=[d])
    e, excl = compare_images(gpu["rgb"][0], ref, "rgb")
    n = ref["rgb"].shape[0] * ref["rgb"].shape[1]
    assert excl <= max(2, 0.01 * n)
    assert e <= IMG_TOL, e
    errs = grad_errors(gpu["grads"][0], oracle.backward(sc, cam, d))
    assert all(v <= 1.0 for v in errs.values()), errs
    # texels outside each splat's grid get no gradient
    gt = gpu["grads"][0]["textures"]
    N = int(sc["tex_n"])
    ii = np.arange(N)
    nk = np.asarray(sc["splat_tex_n"])
    outside = (ii[None, :, None] >= nk[:, None, None]) | (ii[None, None, :] >= nk[:, None, None])
    assert not np.any(gt[outside])


def test_full_size_per_splat_grids_equal_the_uniform_forward():
    """Every n_k = N: the forward is the uniform scene's bit for bit, and the
    gradients agree within the gradient bar."""
    sc = scenes.tiny_scene(35, K=12, tex_n=8, sh_degree=2, tex_dtype="f16")
    var = dict(sc, splat_tex_n=np.full(12, 8, np.int32))
    cam = scenes.tiny_camera(48, 40)
    d = np.random.default_rng(6).standard_normal((40, 48, 3)).astype(np.float32)
    a, b = gpu_run([sc], [cam], d_rgb=[d]), gpu_run([var], [cam], d_rgb=[d])
    for k in ("rgb", "depth", "alpha"):
        assert np.array_equal(a[k][0], b[k][0]), k
    errs = grad_errors(b["grads"][0], {k: v.astype(np.float64) for k, v in a["grads"][0].items()})
    assert all(v <= 1.0 for v in errs.values()), errs


def test_frame_mixing_per_splat_and_uniform_scenes():
    """Two scenes of the same N and storage, one with per-splat sizes (separate
    render groups), in one launch sequence: each camera against the oracle."""
    s_var, cam0 = CASES["n4_f32"]()
    s_uni = scenes.tiny_scene(36, K=9, tex_n=4, sh_degree=2)
    cam1 = scenes.tiny_camera(40, 30, eye=(0.2, -0.1, -4.0))
    rng = np.random.default_rng(7)
    r0, r1 = oracle_run(s_var, cam0), oracle_run(s_uni, cam1)
    d0, d1 = masked_upstream(r0, rng), masked_upstream(r1, rng)
    gpu = gpu_run([s_var, s_uni], [cam0, cam1], cam_scene=[0, 1], d_rgb=[d0, d1])
    for i, (sc, cam, r, d) in enumerate(((s_var, cam0, r0, d0), (s_uni, cam1, r1, d1))):
        e, _ = compare_images(gpu["rgb"][i], r, "rgb")
        assert e <= IMG_TOL, (i, e)
        errs = grad_errors(gpu["grads"][i], oracle.backward(sc, cam, d))
        assert all(v <= 1.0 for v in errs.values()), (i, errs)


@pytest.mark.parametrize("opt", [{"tile": 8}, {"tile": 32}, {"ppt": 2}, {"bwd_kernel": 2}])
def test_options_the_per_splat_path_does_not_take_are_refused(opt):
    from paper_2412_12734_gb300 import _lib as L
    sc, cam = CASES["n4_f32"]()
    with pytest.raises(L.GbillError) as ei:
        gpu_run([sc], [cam], **opt)
    assert ei.value.status == 2  # GB_ERR_UNSUPPORTED


def test_per_splat_sizes_with_a_mip_level_are_refused():
    from paper_2412_12734_gb300 import _lib as L
    sc, cam = CASES["n4_f32"]()
    with pytest.raises(L.GbillError) as ei:
        gpu_run([dict(sc, mip_level=1)], [cam])
    assert ei.value.status == 2
