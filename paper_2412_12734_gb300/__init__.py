"""GB300 (sm_103a) textured 2D-Gaussian-surfel rasterizer ("Gaussian
Billboards", arXiv 2412.12734): forward and backward as hand-written CUDA
behind a C ABI (include/gbill.h), with thin Python bindings.

Modules:
  build    compiles csrc/*.cu into libgbill.so (nvcc, sm_103a)
  _lib     ctypes signatures of the C ABI (argument marshalling only)
  render   Rasterizer (forward, backward, autotune), Saved state, the
           torch.autograd function ``render``, BatchedRenderer (a fixed
           frame's forward and backward replayed from CUDA graphs) and the
           fused Adam (``adam_step``, ``AdamStep``)
  fit2d    the image-fitting loop of Sec. 4.1 on the library's kernels
  scenes   seeded synthetic inputs (no method arithmetic)

There is no CPU fallback: loading the library fails loudly if it has not
been built.
"""
