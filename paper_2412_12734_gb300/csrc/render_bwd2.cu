// Backward per-tile render, two pixels per thread (kernels in render_bwd.cuh;
// a separate translation unit so the two variants compile in parallel).
#include "render_bwd.cuh"

namespace gbill {

template cudaError_t launch_render_bwd_p<2>(const Frame &, const RenderBwdBufs &, int, const uint32_t *,
                                            uint32_t *, bool, cudaStream_t);

}  // namespace gbill
