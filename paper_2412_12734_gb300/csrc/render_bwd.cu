// Backward per-tile render, one pixel per thread (kernels in render_bwd.cuh),
// and the dispatch between the one- and two-pixels-per-thread variants.
#include "render_bwd.cuh"

namespace gbill {

extern template cudaError_t launch_render_bwd_p<2>(const Frame &, const RenderBwdBufs &, int, const uint32_t *,
                                                   uint32_t *, bool, cudaStream_t);
template cudaError_t launch_render_bwd_p<1>(const Frame &, const RenderBwdBufs &, int, const uint32_t *,
                                            uint32_t *, bool, cudaStream_t);

cudaError_t launch_render_bwd(const Frame &f, const RenderBwdBufs &b, int batch, int ppt, const uint32_t *tile_list,
                              uint32_t *work, bool persistent, cudaStream_t s) {
    if (ppt == 2) return launch_render_bwd_p<2>(f, b, batch, tile_list, work, persistent, s);
    if (ppt == 1) return launch_render_bwd_p<1>(f, b, batch, tile_list, work, persistent, s);
    return cudaErrorInvalidValue;
}

}  // namespace gbill
