"""Fused Adam (Sec. 3.3: the paper trains with Adam).

CPU: the oracle's Adam is pinned by closed forms.  GPU: gb_adam_step against
the oracle over several tensors (ragged sizes, unaligned starts, FP16/BF16
shadow copies) for several steps."""
import numpy as np
import pytest

import oracle


def test_oracle_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2, so every step moves the parameter by lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    p, m, v = p0, np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        p, m, v = oracle.adam_step(p, g, m, v, t, lr, b1, b2, eps)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m, (1 - b1 ** 5) * g, rtol=1e-12)
    np.testing.assert_allclose(v, (1 - b2 ** 5) * g * g, rtol=1e-12)


def test_oracle_adam_zero_gradient_keeps_parameters():
    p, m, v = oracle.adam_step(np.ones(4), np.zeros(4), np.zeros(4), np.zeros(4), 1, 0.1, 0.9, 0.999, 1e-8)
    assert np.all(p == 1.0) and np.all(m == 0) and np.all(v == 0)


@pytest.mark.gpu
def test_gpu_adam_matches_oracle():
    import torch

    from paper_2412_12734_gb300 import render as R
    rast = R.Rasterizer(0)
    rng = np.random.default_rng(1)
    sizes = [1, 7, 1000, 4099, 64 * 1024 + 3]
    base = torch.zeros(sum(sizes) + 8, device="cuda")
    params, grads, ms, vs, shadows, host = [], [], [], [], [], []
    off = 1  # unaligned views into one buffer for the first tensors
    for i, n in enumerate(sizes):
        p0 = rng.standard_normal(n).astype(np.float32)
        if i < 2:
            p = base[off:off + n]
            p.copy_(torch.as_tensor(p0))
            off += n
        else:
            p = torch.as_tensor(p0, device="cuda")
        params.append(p)
        ms.append(torch.zeros(n, device="cuda"))
        vs.append(torch.zeros(n, device="cuda"))
        shadows.append(torch.empty(n, device="cuda", dtype=[torch.float16, torch.bfloat16, None, torch.bfloat16,
                                                              torch.float16][i] or torch.float32))
        host.append([p0.astype(np.float64), np.zeros(n), np.zeros(n)])
    # the kernel receives FP32 hyper-parameters; the oracle gets the same values
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-3, 0.9, 0.999, 1e-15))
    for step in range(1, 4):
        gs = [rng.standard_normal(n).astype(np.float32) for n in sizes]
        grads = [torch.as_tensor(g, device="cuda") for g in gs]
        R.adam_step(rast, params, grads, ms, vs, step, lr=lr, betas=(b1, b2), eps=eps, shadows=shadows)
        for i in range(len(sizes)):
            host[i] = list(oracle.adam_step(host[i][0], gs[i], host[i][1], host[i][2], step, lr, b1, b2, eps))
    torch.cuda.synchronize()
    for i in range(len(sizes)):
        p = params[i].cpu().numpy()
        np.testing.assert_allclose(p, host[i][0], rtol=0, atol=2e-6)
        np.testing.assert_allclose(ms[i].cpu().numpy(), host[i][1], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(vs[i].cpu().numpy(), host[i][2], rtol=1e-5, atol=1e-9)
        sh = shadows[i].float().cpu().numpy()
        exp = torch.as_tensor(p).to(shadows[i].dtype).float().numpy()
        np.testing.assert_array_equal(sh, exp)
