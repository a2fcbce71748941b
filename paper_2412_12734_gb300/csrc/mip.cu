// Mip-level colour grids (Sec. 4.1, Fig. 4 f, g): the renderer draws every
// grid of a scene box-filtered to (N/2^l) x (N/2^l), each texel the mean of
// its 2^l x 2^l block.  The filter runs once per forward into an FP32 grid
// that the render kernels read like any other; the backward renders the
// gradient of that grid and the adjoint of the filter spreads it over the
// stored texels (1/4^l each).  Both passes are HBM-bound elementwise kernels.
#include <algorithm>

#include "gbill_internal.cuh"

namespace gbill {
namespace {

template <typename TexT>
__global__ void mip_filter_kernel(const TexT *src, int64_t K, int ns, int mip, float *dst) {
    const int n = ns >> mip, fm = 1 << mip;
    const float inv = 1.0f / float(fm * fm);
    const int64_t total = K * n * n * 3;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(e % 3);
        const int64_t t = e / 3;
        const int j = int(t % n);
        const int i = int((t / n) % n);
        const int64_t k = t / (int64_t(n) * n);
        float acc = 0.0f;
        for (int a = 0; a < fm; ++a)
            for (int b = 0; b < fm; ++b)
                acc += load_as_float(src, ((k * ns + fm * i + a) * ns + fm * j + b) * 3 + c);
        dst[e] = acc * inv;
    }
}

__global__ void mip_grad_kernel(const float *gc, int64_t K, int ns, int mip, float *gf) {
    const int n = ns >> mip;
    const float inv = 1.0f / float(1 << (2 * mip));
    const int64_t total = K * ns * ns * 3;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(e % 3);
        const int64_t t = e / 3;
        const int j = int(t % ns) >> mip;
        const int i = int((t / ns) % ns) >> mip;
        const int64_t k = t / (int64_t(ns) * ns);
        gf[e] = gc[((k * n + i) * n + j) * 3 + c] * inv;
    }
}

unsigned grid_for(int64_t n) {
    return unsigned(std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 32));
}

}  // namespace

cudaError_t launch_mip_filter(const void *src, int dtype, int64_t K, int ns, int mip, float *dst, cudaStream_t s) {
    const int64_t n = K * (ns >> mip) * (ns >> mip) * 3;
    if (n == 0) return cudaSuccess;
    switch (dtype) {
        case GB_F16: mip_filter_kernel<<<grid_for(n), 256, 0, s>>>(static_cast<const __half *>(src), K, ns, mip, dst); break;
        case GB_BF16:
            mip_filter_kernel<<<grid_for(n), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(src), K, ns, mip, dst);
            break;
        default: mip_filter_kernel<<<grid_for(n), 256, 0, s>>>(static_cast<const float *>(src), K, ns, mip, dst); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mip_grad(const float *gc, int64_t K, int ns, int mip, float *gf, cudaStream_t s) {
    const int64_t n = K * ns * ns * 3;
    if (n == 0) return cudaSuccess;
    mip_grad_kernel<<<grid_for(n), 256, 0, s>>>(gc, K, ns, mip, gf);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gbill
