// Per-texel spherical harmonics (Sec. 4.2: M coefficient triples per texel
// instead of one RGB colour).  A splat's texels are seen along one direction
// per camera, d = (p - camera centre) / |p - camera centre|, so each
// (splat, camera) record gets its own RGB grid, texel colour
// sum_lm k_lm Y_lm(d).  A pre-pass evaluates those grids into FP32 scratch
// indexed by record; the render kernels read them like any other grid.  The
// backward renders the gradient of each record's grid, and a post-pass turns
// it into coefficient gradients (sum over cameras of Y_lm(d) C^) and a centre
// gradient through d (sum of C^ . k dY/dd, projected by (I - d d^T) / |p - c|).
#include <algorithm>

#include "sh.cuh"

namespace gbill {
namespace {

unsigned grid_for(int64_t n) {
    return unsigned(std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 32));
}

__device__ __forceinline__ float load_coef(const void *p, int dtype, int64_t i) {
    switch (dtype) {
        case GB_F16: return load_as_float(static_cast<const __half *>(p), i);
        case GB_BF16: return load_as_float(static_cast<const __nv_bfloat16 *>(p), i);
        default: return load_as_float(static_cast<const float *>(p), i);
    }
}

// unit view direction and distance of splat k seen from camera `cam`
__device__ __forceinline__ void view_dir(const SceneDev &sc, const CamDev &cam, int64_t k, float d[3], float &dist) {
    float v[3];
    for (int i = 0; i < 3; ++i) v[i] = sc.means[3 * k + i] - cam.campos[i];
    dist = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float inv = 1.0f / dist;
    for (int i = 0; i < 3; ++i) d[i] = v[i] * inv;
}

// out[(tex_row + k) * N^2 * 3 + t * 3 + ch] for one camera (blockIdx.y) of scene si
template <int Dt>
__global__ void texsh_eval_kernel(Frame f, int si, const void *coef, int dtype, float *out) {
    constexpr int M = (Dt + 1) * (Dt + 1);
    const CamDev &cam = f.cams[blockIdx.y];
    if (cam.scene != si) return;
    const SceneDev &sc = f.scenes[si];
    const int NN = sc.N * sc.N;
    const int64_t total = sc.K * NN;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = e / NN;
        const int t = int(e - k * NN);
        float d[3], dist;
        view_dir(sc, cam, k, d, dist);
        float Y[16];
        sh_basis(Dt, d[0], d[1], d[2], Y);
        float c[3] = {0.0f, 0.0f, 0.0f};
        const int64_t base = (k * NN + t) * M * 3;
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) c[ch] = fmaf(Y[m], load_coef(coef, dtype, base + m * 3 + ch), c[ch]);
        float *o = out + (cam.tex_row + k) * NN * 3 + t * 3;
        o[0] = c[0];
        o[1] = c[1];
        o[2] = c[2];
    }
}

// one thread per (splat, texel) of scene si: coefficient gradients (written)
// and the centre gradient through the view direction (added to g_means)
template <int Dt>
__global__ void texsh_grad_kernel(Frame f, int si, const void *coef, int dtype, const float *grid_grad,
                                  float *g_coef, float *g_means) {
    constexpr int M = (Dt + 1) * (Dt + 1);
    const SceneDev &sc = f.scenes[si];
    const int NN = sc.N * sc.N;
    const int64_t total = sc.K * NN;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = e / NN;
        const int t = int(e - k * NN);
        const int64_t base = (k * NN + t) * M * 3;
        float kc[M][3], acc[M][3];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                kc[m][ch] = load_coef(coef, dtype, base + m * 3 + ch);
                acc[m][ch] = 0.0f;
            }
        float gp[3] = {0.0f, 0.0f, 0.0f};
        for (int ci = 0; ci < f.n_cams; ++ci) {
            const CamDev &cam = f.cams[ci];
            if (cam.scene != si) continue;
            const float *gg = grid_grad + ((cam.tex_row + k) * NN + t) * 3;
            const float h[3] = {gg[0], gg[1], gg[2]};
            if (h[0] == 0.0f && h[1] == 0.0f && h[2] == 0.0f) continue;
            float d[3], dist;
            view_dir(sc, cam, k, d, dist);
            float Y[16], G[16][3];
            sh_basis(Dt, d[0], d[1], d[2], Y);
            sh_basis_grad(Dt, d[0], d[1], d[2], G);
            float gd[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float s = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    acc[m][ch] = fmaf(Y[m], h[ch], acc[m][ch]);
                    s = fmaf(kc[m][ch], h[ch], s);
                }
                gd[0] = fmaf(s, G[m][0], gd[0]);
                gd[1] = fmaf(s, G[m][1], gd[1]);
                gd[2] = fmaf(s, G[m][2], gd[2]);
            }
            const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
            for (int i = 0; i < 3; ++i) gp[i] += (gd[i] - d[i] * dd) / dist;
        }
        if (g_coef)
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) g_coef[base + m * 3 + ch] = acc[m][ch];
        if (g_means && (gp[0] != 0.0f || gp[1] != 0.0f || gp[2] != 0.0f))
            for (int i = 0; i < 3; ++i) atomicAdd(g_means + 3 * k + i, gp[i]);
    }
}

}  // namespace

cudaError_t launch_texsh_eval(const Frame &f, int si, int Dt, const void *coef, int dtype, float *out,
                              cudaStream_t s) {
    const int64_t n = f.scenes[si].K * f.scenes[si].N * f.scenes[si].N;
    if (n == 0) return cudaSuccess;
    const dim3 grid(grid_for(n), unsigned(f.n_cams));
    switch (Dt) {
        case 1: texsh_eval_kernel<1><<<grid, 256, 0, s>>>(f, si, coef, dtype, out); break;
        case 2: texsh_eval_kernel<2><<<grid, 256, 0, s>>>(f, si, coef, dtype, out); break;
        default: texsh_eval_kernel<3><<<grid, 256, 0, s>>>(f, si, coef, dtype, out); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_texsh_grad(const Frame &f, int si, int Dt, const void *coef, int dtype, const float *grid_grad,
                              float *g_coef, float *g_means, cudaStream_t s) {
    const int64_t n = f.scenes[si].K * f.scenes[si].N * f.scenes[si].N;
    if (n == 0) return cudaSuccess;
    switch (Dt) {
        case 1: texsh_grad_kernel<1><<<grid_for(n), 256, 0, s>>>(f, si, coef, dtype, grid_grad, g_coef, g_means); break;
        case 2: texsh_grad_kernel<2><<<grid_for(n), 256, 0, s>>>(f, si, coef, dtype, grid_grad, g_coef, g_means); break;
        default: texsh_grad_kernel<3><<<grid_for(n), 256, 0, s>>>(f, si, coef, dtype, grid_grad, g_coef, g_means); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gbill
