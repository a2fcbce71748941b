// Image fitting (Sec. 4.1): splats live in planes facing a camera that looks
// down +z and may only turn about the view axis, so a splat's raw parameters
// are an angle theta, a position (x, y) in its plane z, log-scales and an
// opacity logit.  The map to the renderer's activated parameters and its
// adjoint, and the mean-squared-error loss with its gradient, are elementwise
// HBM-bound kernels; together with the renderer and the fused Adam they make
// one fitting iteration without leaving the library.
#include <algorithm>

#include "gbill_internal.cuh"

namespace gbill {
namespace {

unsigned grid_for(int64_t n) {
    return unsigned(std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 32));
}

// quats = (cos(theta/2), 0, 0, sin(theta/2)), means = (x, y, z),
// scales = exp(log_scales), opacities = 1 / (1 + exp(-logit))
__global__ void fit_params_kernel(const float *theta, const float *xy, const float *z, const float *log_s,
                                  const float *logit, int64_t K, float *quats, float *means, float *scales,
                                  float *opac) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x) {
        float sn, cs;
        sincosf(0.5f * theta[k], &sn, &cs);
        reinterpret_cast<float4 *>(quats)[k] = make_float4(cs, 0.0f, 0.0f, sn);
        means[3 * k + 0] = xy[2 * k + 0];
        means[3 * k + 1] = xy[2 * k + 1];
        means[3 * k + 2] = z[k];
        scales[2 * k + 0] = expf(log_s[2 * k + 0]);
        scales[2 * k + 1] = expf(log_s[2 * k + 1]);
        opac[k] = 1.0f / (1.0f + expf(-logit[k]));
    }
}

// adjoint of fit_params_kernel: d theta = d_q . dq/dtheta, d xy = d_means.xy,
// d log_s = d_scales * scales, d logit = d_opac * o (1 - o)
__global__ void fit_params_bwd_kernel(const float *theta, const float *log_s, const float *logit, int64_t K,
                                      const float *d_quats, const float *d_means, const float *d_scales,
                                      const float *d_opac, float *d_theta, float *d_xy, float *d_log_s,
                                      float *d_logit) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x) {
        float sn, cs;
        sincosf(0.5f * theta[k], &sn, &cs);
        const float4 dq = reinterpret_cast<const float4 *>(d_quats)[k];
        d_theta[k] = 0.5f * (cs * dq.w - sn * dq.x);
        d_xy[2 * k + 0] = d_means[3 * k + 0];
        d_xy[2 * k + 1] = d_means[3 * k + 1];
        d_log_s[2 * k + 0] = d_scales[2 * k + 0] * expf(log_s[2 * k + 0]);
        d_log_s[2 * k + 1] = d_scales[2 * k + 1] * expf(log_s[2 * k + 1]);
        const float o = 1.0f / (1.0f + expf(-logit[k]));
        d_logit[k] = d_opac[k] * o * (1.0f - o);
    }
}

// L = mean over the n values of (rgb - target)^2, dL/drgb = 2 (rgb - target) / n;
// L is summed in FP64 (per-block tree, one FP64 atomic per block)
__global__ void mse_kernel(const float *rgb, const float *target, int64_t n, float *d_rgb, double *loss) {
    __shared__ double s_part[8];
    const float scale = 2.0f / float(n);
    double acc = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const float r = rgb[e] - target[e];
        if (d_rgb) d_rgb[e] = scale * r;
        acc += double(r) * double(r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += s_part[w];
        atomicAdd(loss, t / double(n));
    }
}

}  // namespace

cudaError_t launch_fit_params(const float *theta, const float *xy, const float *z, const float *log_s,
                              const float *logit, int64_t K, float *quats, float *means, float *scales, float *opac,
                              cudaStream_t s) {
    if (K == 0) return cudaSuccess;
    fit_params_kernel<<<grid_for(K), 256, 0, s>>>(theta, xy, z, log_s, logit, K, quats, means, scales, opac);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fit_params_bwd(const float *theta, const float *log_s, const float *logit, int64_t K,
                                  const float *d_quats, const float *d_means, const float *d_scales,
                                  const float *d_opac, float *d_theta, float *d_xy, float *d_log_s, float *d_logit,
                                  cudaStream_t s) {
    if (K == 0) return cudaSuccess;
    fit_params_bwd_kernel<<<grid_for(K), 256, 0, s>>>(theta, log_s, logit, K, d_quats, d_means, d_scales, d_opac,
                                                      d_theta, d_xy, d_log_s, d_logit);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float *rgb, const float *target, int64_t n, float *d_rgb, double *loss, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
    if (e != cudaSuccess || n == 0) return e;
    mse_kernel<<<grid_for(n), 256, 0, s>>>(rgb, target, n, d_rgb, loss);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gbill
