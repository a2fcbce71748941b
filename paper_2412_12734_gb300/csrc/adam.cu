// Fused Adam step over many tensors in one launch (the optimiser the paper
// trains with, Sec. 3.3).  Per element: m = b1 m + (1-b1) g,
// v = b2 v + (1-b2) g^2, p -= lr (m / c1) / (sqrt(v / c2) + eps) with the
// bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t, plus an optional copy of the
// updated value in FP16/BF16 (the storage the renderer reads).  HBM bound:
// 16 bytes read and 12 (+2 or 4) bytes written per element.
#include "gbill_internal.cuh"

namespace gbill {
namespace {

constexpr int kMaxAdamTensors = 16;

struct AdamDesc {
    int n;
    float lr, b1, b2, eps, inv_c1, inv_c2;
    gb_adam_tensor t[kMaxAdamTensors];
};

__device__ __forceinline__ void store_shadow(void *sh, int32_t dt, int64_t i, float x) {
    if (dt == GB_F16) static_cast<__half *>(sh)[i] = __float2half_rn(x);
    else if (dt == GB_BF16) static_cast<__nv_bfloat16 *>(sh)[i] = __float2bfloat16_rn(x);
    else static_cast<float *>(sh)[i] = x;
}

__device__ __forceinline__ float adam_one(float p, float g, float &m, float &v, const AdamDesc &d) {
    m = fmaf(d.b1, m, (1.0f - d.b1) * g);
    v = fmaf(d.b2, v, (1.0f - d.b2) * g * g);
    return p - d.lr * (m * d.inv_c1) / (sqrtf(v * d.inv_c2) + d.eps);
}

__global__ void __launch_bounds__(256) adam_kernel(AdamDesc d) {
    const gb_adam_tensor &t = d.t[blockIdx.y];
    const int64_t n4 = t.n / 4;
    const bool vec = ((reinterpret_cast<uintptr_t>(t.param) | reinterpret_cast<uintptr_t>(t.grad) |
                       reinterpret_cast<uintptr_t>(t.m) | reinterpret_cast<uintptr_t>(t.v)) & 15) == 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t first_scalar = 0;
    if (vec) {
        float4 *p4 = reinterpret_cast<float4 *>(t.param);
        const float4 *g4 = reinterpret_cast<const float4 *>(t.grad);
        float4 *m4 = reinterpret_cast<float4 *>(t.m);
        float4 *v4 = reinterpret_cast<float4 *>(t.v);
        for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 p = p4[i], g = g4[i], m = m4[i], v = v4[i];
            p.x = adam_one(p.x, g.x, m.x, v.x, d);
            p.y = adam_one(p.y, g.y, m.y, v.y, d);
            p.z = adam_one(p.z, g.z, m.z, v.z, d);
            p.w = adam_one(p.w, g.w, m.w, v.w, d);
            p4[i] = p;
            m4[i] = m;
            v4[i] = v;
            if (t.shadow) {
                store_shadow(t.shadow, t.shadow_dtype, 4 * i + 0, p.x);
                store_shadow(t.shadow, t.shadow_dtype, 4 * i + 1, p.y);
                store_shadow(t.shadow, t.shadow_dtype, 4 * i + 2, p.z);
                store_shadow(t.shadow, t.shadow_dtype, 4 * i + 3, p.w);
            }
        }
        first_scalar = 4 * n4;
    }
    for (int64_t i = first_scalar + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < t.n; i += stride) {
        float m = t.m[i], v = t.v[i];
        const float p = adam_one(t.param[i], t.grad[i], m, v, d);
        t.param[i] = p;
        t.m[i] = m;
        t.v[i] = v;
        if (t.shadow) store_shadow(t.shadow, t.shadow_dtype, i, p);
    }
}

}  // namespace

cudaError_t launch_adam(const gb_adam_tensor *ts, int n, const gb_adam_config &c, int grid_x, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n > kMaxAdamTensors) return cudaErrorInvalidValue;
    AdamDesc d;
    d.n = n;
    d.lr = c.lr;
    d.b1 = c.beta1;
    d.b2 = c.beta2;
    d.eps = c.eps;
    d.inv_c1 = float(1.0 / (1.0 - pow(double(c.beta1), double(c.step))));
    d.inv_c2 = float(1.0 / (1.0 - pow(double(c.beta2), double(c.step))));
    for (int i = 0; i < n; ++i) d.t[i] = ts[i];
    adam_kernel<<<dim3(unsigned(grid_x), unsigned(n)), 256, 0, s>>>(d);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gbill
