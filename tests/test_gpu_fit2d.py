"""Image fitting on the GPU (Sec. 4.1): the parameter map, its adjoint and the
MSE loss against the FP64 oracle; the raw-parameter gradients of a whole
fitting iteration (activation, render, loss, backward, adjoint) against the
oracle's; and a short fit that must lower the loss."""
import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes
from tests.gpu_util import grad_errors

pytestmark = pytest.mark.gpu


def _raw_device(raw):
    import torch
    return {k: torch.as_tensor(np.ascontiguousarray(raw[k]), dtype=torch.float32, device="cuda").contiguous()
            for k in ("theta", "xy", "z", "log_scales", "logit_opacities")}


def test_fit_params_and_adjoint_match_oracle():
    import ctypes as C

    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    K = 4099
    raw = scenes.fit_init(K, 640, 480, seed=3)
    raw["theta"] = np.random.default_rng(1).uniform(-7, 7, K).astype(np.float32)
    d = _raw_device(raw)
    out = {"quats": torch.empty((K, 4), device="cuda"), "means": torch.empty((K, 3), device="cuda"),
           "scales": torch.empty((K, 2), device="cuda"), "opacities": torch.empty(K, device="cuda")}
    lib, s = L.load(), C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(lib.gb_fit_params(rast.ctx, K, d["theta"].data_ptr(), d["xy"].data_ptr(), d["z"].data_ptr(),
                              d["log_scales"].data_ptr(), d["logit_opacities"].data_ptr(), out["quats"].data_ptr(),
                              out["means"].data_ptr(), out["scales"].data_ptr(), out["opacities"].data_ptr(), s),
            rast.ctx)
    ref = oracle.fit_params(raw)
    for k in out:
        np.testing.assert_allclose(out[k].cpu().numpy(), ref[k], rtol=2e-6, atol=2e-7)
    rng = np.random.default_rng(2)
    g = {"quats": rng.standard_normal((K, 4)), "means": rng.standard_normal((K, 3)),
         "scales": rng.standard_normal((K, 2)), "opacities": rng.standard_normal(K)}
    gd = {k: torch.as_tensor(v, dtype=torch.float32, device="cuda") for k, v in g.items()}
    res = {"theta": torch.empty(K, device="cuda"), "xy": torch.empty((K, 2), device="cuda"),
           "log_scales": torch.empty((K, 2), device="cuda"), "logit_opacities": torch.empty(K, device="cuda")}
    L.check(lib.gb_fit_params_backward(rast.ctx, K, d["theta"].data_ptr(), d["log_scales"].data_ptr(),
                                       d["logit_opacities"].data_ptr(), gd["quats"].data_ptr(),
                                       gd["means"].data_ptr(), gd["scales"].data_ptr(), gd["opacities"].data_ptr(),
                                       res["theta"].data_ptr(), res["xy"].data_ptr(), res["log_scales"].data_ptr(),
                                       res["logit_opacities"].data_ptr(), s), rast.ctx)
    g32 = {k: v.astype(np.float32).astype(np.float64) for k, v in g.items()}
    ref = oracle.fit_params_backward(raw, g32)
    for k in res:
        np.testing.assert_allclose(res[k].cpu().numpy(), ref[k], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("n", [0, 1, 3 * 1001, 3 * 1920 * 871])
def test_mse_matches_oracle(n):
    import ctypes as C

    import torch

    from paper_2412_12734_gb300 import _lib as L
    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    rng = np.random.default_rng(n)
    a = rng.uniform(0, 1, n).astype(np.float32)
    b = rng.uniform(0, 1, n).astype(np.float32)
    at, bt = torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda")
    d = torch.full((max(n, 1),), 7.0, device="cuda")
    loss = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    L.check(L.load().gb_mse_loss(rast.ctx, at.data_ptr(), bt.data_ptr(), n, d.data_ptr(), loss.data_ptr(),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream)), rast.ctx)
    if n == 0:
        assert loss.item() == 0.0
        return
    ref, dref = oracle.mse_loss(a, b)
    # each difference rgb - target is rounded to FP32 (relative u = 2^-24), so each
    # squared term carries at most 2u relative error; the FP64 sum adds nothing
    assert abs(loss.item() - ref) <= 4 * 2.0 ** -24 * ref
    np.testing.assert_allclose(d.cpu().numpy()[:n], dref, rtol=1e-6, atol=1e-12)


def test_fit_iteration_gradients_match_oracle():
    import torch

    from paper_2412_12734_gb300 import fit2d
    W, H, K = 48, 40, 30
    target = scenes.fit_target((W, H), seed=4)
    fit = fit2d.ImageFit(target, K, tex_n=4, seed=4)
    raw = scenes.fit_init(K, W, H, seed=4, tex_n=4)
    ref = oracle.render(oracle.fit_scene(raw), fit.cam)
    mask = (ref["margin_grad"] > 1e-4).astype(np.float64)
    fit.forward_loss()
    # zero the upstream gradient at pixels within the decision margin (both sides)
    fit.d_rgb.mul_(torch.as_tensor(mask.reshape(-1, 1), dtype=torch.float32, device="cuda"))
    fit.backward()
    torch.cuda.synchronize()
    og = oracle.fit_step(raw, target, fit.cam, mask=mask)
    assert abs(fit.loss() - og["loss"]) <= 1e-5 * og["loss"]
    gpu = {k: fit.g[k].cpu().numpy() for k in fit2d.RAW}
    errs = grad_errors(gpu, {k: og[k] for k in fit2d.RAW})
    assert all(v <= 1.0 for v in errs.values()), errs


def test_fit_lowers_the_loss():
    from paper_2412_12734_gb300 import fit2d
    target = scenes.fit_target((96, 72), seed=5)
    fit = fit2d.ImageFit(target, 200, tex_n=4, seed=5)
    fit.forward_loss()
    l0 = fit.loss()
    for _ in range(150):
        fit.step()
    fit.check()
    l1 = fit.loss()
    assert l1 < 0.5 * l0, (l0, l1)


def _fit_pair(K=200, seed=6, wh=(96, 72)):
    from paper_2412_12734_gb300 import fit2d
    target = scenes.fit_target(wh, seed=seed)
    return (fit2d.ImageFit(target, K, tex_n=4, seed=seed, graph=True),
            fit2d.ImageFit(target, K, tex_n=4, seed=seed, graph=False))


def test_graph_iterations_match_host_launched_iterations():
    """The CUDA-graph iteration replays the same kernels as the host-launched
    one on parameters that Adam moved in place: the first iteration's raw
    gradients agree up to the order of the backward's atomics, and the losses
    of later iterations (other visible sets, other instance counts) stay
    within 1e-3 relative (Adam normalises each step, so rounding noise in a
    near-zero gradient can move a parameter by a whole step)."""
    from paper_2412_12734_gb300 import fit2d
    fg, fe = _fit_pair()
    fg.step()
    fe.step()
    assert abs(fg.loss() - fe.loss()) <= 1e-6 * fe.loss()
    for k in fit2d.RAW:
        a, b = fg.g[k], fe.g[k]
        scale = b.abs().max().item()
        assert (a - b).abs().max().item() <= 1e-4 * max(scale, 1e-12), k
    for i in range(30):
        fg.step()
        fe.step()
        if i % 10 == 9:
            assert abs(fg.loss() - fe.loss()) <= 1e-3 * fe.loss(), (i, fg.loss(), fe.loss())
    fg.check()
    fe.check()


def test_graph_is_captured_again_after_the_saved_state_grows():
    """ensure_capacity doubling the instance capacity moves the saved state's
    buffers; the next graph iteration captures again and keeps fitting."""
    fg, fe = _fit_pair(seed=7)
    for _ in range(5):
        fg.step()
        fe.step()
    cap0 = fg.saved.stats()["capacity"]
    fg.ensure_capacity(headroom=0.0)
    fe.ensure_capacity(headroom=0.0)
    assert fg.saved.stats()["capacity"] >= 2 * cap0
    assert fg._graph is None
    for _ in range(10):
        fg.step()
        fe.step()
    fg.check()
    assert abs(fg.loss() - fe.loss()) <= 1e-3 * fe.loss(), (fg.loss(), fe.loss())
