"""Host-side checks of the Python binding (no GPU).

The library reads and writes the caller's buffers through plain pointers, so
the binding checks their type and size before a call: the gradient outputs
it allocates itself have exactly the shapes those checks expect (the
gb_grads layout of include/gbill.h), and a buffer of the wrong type, layout,
size or device is refused.
"""
import numpy as np
import pytest
import torch

from paper_2412_12734_gb300 import render as R


@pytest.mark.parametrize("K,D,N,Mt", [(0, 0, 1, 0), (5, 3, 4, 0), (7, 1, 8, 16), (3, 2, 16, 4)])
def test_gradient_shapes_follow_the_abi_layout(K, D, N, Mt):
    shapes = R.grad_shapes(K, D, N, Mt)
    assert tuple(shapes) == R.PARAMS
    n = {k: int(np.prod(v)) for k, v in shapes.items()}
    # means [K,3], quats [K,4], scales [K,2], opacities [K], sh [K,(D+1)^2,3],
    # textures [K,N,N,3] or, with per-texel SH, [K,N,N,(Dt+1)^2,3]
    assert n == {"means": 3 * K, "quats": 4 * K, "scales": 2 * K, "opacities": K, "sh": 3 * K * (D + 1) ** 2,
                 "textures": 3 * K * N * N * max(Mt, 1)}


def test_buffers_of_the_wrong_type_size_or_device_are_refused():
    with pytest.raises(ValueError, match="float32"):
        R._check_buffer(torch.zeros(6, dtype=torch.float64), "d_rgb", 6)
    with pytest.raises(ValueError, match="float32"):
        R._check_buffer(torch.zeros(4, 3).t(), "d_rgb", 12)
    with pytest.raises(ValueError, match="float32"):
        R._check_buffer(np.zeros(6, np.float32), "d_rgb", 6)
    with pytest.raises(ValueError, match="expected 9"):
        R._check_buffer(torch.zeros(6), "d_rgb", 9)
    with pytest.raises(ValueError, match="CUDA"):
        R._check_buffer(torch.zeros(6), "d_rgb", 6)


class _FakeSaved:
    """The binding's record of a forward: 2 scenes, 30 pixels."""
    n_scenes = 2
    shapes = [(5, 3, 4, 0), (7, 1, 8, 4)]  # (K, D, N, Mt): RGB texels; per-texel SH of degree 1
    n_pix = 30
    handle = None


def _backward(**kw):
    # the method up to the library call; only the device check is left to fail on a host without a GPU
    return R.Rasterizer.backward(None, _FakeSaved(), **kw)


def test_backward_checks_reach_the_device_check_for_well_formed_buffers():
    with pytest.raises(ValueError, match="CUDA"):
        _backward(d_rgb=torch.zeros(30, 3))  # gradient outputs allocated by the binding itself
    grads = [{k: torch.zeros(s) for k, s in R.grad_shapes(*sh).items()} for sh in _FakeSaved.shapes]
    with pytest.raises(ValueError, match="CUDA"):
        _backward(d_rgb=torch.zeros(30, 3), grads=grads)


def test_backward_refuses_misfit_buffers():
    grads = [{k: torch.zeros(s) for k, s in R.grad_shapes(*sh).items()} for sh in _FakeSaved.shapes]
    with pytest.raises(ValueError, match="2 scenes"):
        _backward(d_rgb=torch.zeros(30, 3), grads=grads[:1])
    bad = [{}, {"textures": torch.zeros(7, 8, 8, 3)}]  # RGB-sized for a grid of degree-1 SH texels
    with pytest.raises(ValueError, match=r"grads\[1\]\['textures'\]: 1344 elements, expected 5376"):
        _backward(d_rgb=torch.zeros(30, 3), grads=bad)
    with pytest.raises(ValueError, match="d_rgb: 87 elements, expected 90"):
        _backward(d_rgb=torch.zeros(29, 3), grads=[{}, {}])
    with pytest.raises(ValueError, match="d_rgb must be a contiguous float32"):
        _backward(d_rgb=torch.zeros(30, 3, dtype=torch.float64), grads=[{}, {}])
