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
#include <cstdint>
#include <type_traits>

#include "sh.cuh"

namespace gbill {
namespace {

unsigned grid_for(int64_t n) {
    return unsigned(std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 32));
}

// The M coefficient triples of one texel, stored contiguously ([m][ch]).
// VEC: the texel's bytes are read with the widest aligned vector loads (the
// caller checked the base pointer's alignment).
template <int M, typename T, bool VEC>
__device__ __forceinline__ void load_texel(const T *p, float kc[M * 3]) {
    constexpr int B = M * 3 * int(sizeof(T));
    constexpr int W = VEC ? (B % 16 == 0 ? 16 : B % 8 == 0 ? 8 : B % 4 == 0 ? 4 : 0) : 0;
    if constexpr (W == 0 || sizeof(T) == 4 && W == 4) {
#pragma unroll
        for (int i = 0; i < M * 3; ++i) kc[i] = load_as_float(p, i);
    } else {
        constexpr int PER = W / int(sizeof(T));  // values per vector
        using V = typename std::conditional<W == 16, uint4, typename std::conditional<W == 8, uint2, uint32_t>::type>::type;
        const V *vp = reinterpret_cast<const V *>(p);
#pragma unroll
        for (int w = 0; w < M * 3 / PER; ++w) {
            const V v = vp[w];
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int i = 0; i < PER; ++i) kc[w * PER + i] = load_as_float(e, i);
        }
    }
}

// unit view direction and distance from the camera centre to the point p
__device__ __forceinline__ void view_dir(const float p[3], const CamDev &cam, float d[3], float &dist) {
    const float v0 = p[0] - cam.campos[0], v1 = p[1] - cam.campos[1], v2 = p[2] - cam.campos[2];
    dist = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
    const float inv = 1.0f / dist;
    d[0] = v0 * inv;
    d[1] = v1 * inv;
    d[2] = v2 * inv;
}

// One thread per (splat, texel) of scene si: the texel's coefficients are
// read once and its colour written for every camera of the scene,
// out[(tex_row + k) N^2 + t][ch] = sum_m Y_m(d) k_m,ch.
template <int Dt, typename T, bool VEC>
__global__ void __launch_bounds__(256) texsh_eval_kernel(Frame f, int si, const T *coef, float *out) {
    constexpr int M = (Dt + 1) * (Dt + 1);
    const SceneDev &sc = f.scenes[si];
    const int NN = sc.N * sc.N;
    const int64_t total = sc.K * NN;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = e / NN;
        const int t = int(e - k * NN);
        float kc[M * 3];
        load_texel<M, T, VEC>(coef + e * (M * 3), kc);
        const float p[3] = {sc.means[3 * k], sc.means[3 * k + 1], sc.means[3 * k + 2]};
        for (int ci = 0; ci < f.n_cams; ++ci) {
            const CamDev &cam = f.cams[ci];
            if (cam.scene != si) continue;
            float d[3], dist;
            view_dir(p, cam, d, dist);
            float Y[16];
            sh_basis(Dt, d[0], d[1], d[2], Y);
            float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                c0 = fmaf(Y[m], kc[3 * m + 0], c0);
                c1 = fmaf(Y[m], kc[3 * m + 1], c1);
                c2 = fmaf(Y[m], kc[3 * m + 2], c2);
            }
            float *o = out + ((cam.tex_row + k) * NN + t) * 3;
            o[0] = c0;
            o[1] = c1;
            o[2] = c2;
        }
    }
}

// One thread per (splat, texel): coefficient gradients, written,
// g[k][t][m][ch] = sum over the scene's cameras of Y_m(d) C^[ch].  The 256
// texels of a block own one contiguous stretch of the output; VEC: it is
// written through shared memory with coalesced 16-byte stores.
template <int Dt, bool VEC>
__global__ void __launch_bounds__(256) texsh_coef_grad_kernel(Frame f, int si, const float *grid_grad, float *g_coef) {
    constexpr int M = (Dt + 1) * (Dt + 1);
    constexpr int W = M * 3;       // floats per texel
    constexpr int WP = W + 1;      // padded row in shared memory
    extern __shared__ float s_out[];  // [256][WP] (VEC only)
    const SceneDev &sc = f.scenes[si];
    const int NN = sc.N * sc.N;
    const int64_t total = sc.K * NN;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < total; base += stride) {
        const int64_t e = base + threadIdx.x;
        float acc[W];
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] = 0.0f;
        if (e < total) {
            const int64_t k = e / NN;
            const int t = int(e - k * NN);
            const float p[3] = {sc.means[3 * k], sc.means[3 * k + 1], sc.means[3 * k + 2]};
            // cameras in groups of four: the group's grid-gradient loads are
            // issued together (most are zero: the splat is culled in the camera)
            for (int c0 = 0; c0 < f.n_cams; c0 += 4) {
                float h[4][3];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    h[j][0] = h[j][1] = h[j][2] = 0.0f;
                    if (c0 + j < f.n_cams && f.cams[c0 + j].scene == si) {
                        const float *gg = grid_grad + ((f.cams[c0 + j].tex_row + k) * NN + t) * 3;
                        h[j][0] = gg[0];
                        h[j][1] = gg[1];
                        h[j][2] = gg[2];
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (h[j][0] == 0.0f && h[j][1] == 0.0f && h[j][2] == 0.0f) continue;
                    float d[3], dist;
                    view_dir(p, f.cams[c0 + j], d, dist);
                    float Y[16];
                    sh_basis(Dt, d[0], d[1], d[2], Y);
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        acc[3 * m + 0] = fmaf(Y[m], h[j][0], acc[3 * m + 0]);
                        acc[3 * m + 1] = fmaf(Y[m], h[j][1], acc[3 * m + 1]);
                        acc[3 * m + 2] = fmaf(Y[m], h[j][2], acc[3 * m + 2]);
                    }
                }
            }
        }
        if constexpr (VEC) {
            // row threadIdx.x of the block's stretch; then the stretch
            // [base W, (base + n) W) goes out as float4s in address order
#pragma unroll
            for (int i = 0; i < W; ++i) s_out[threadIdx.x * WP + i] = acc[i];
            __syncthreads();
            const int n = total - base < 256 ? int(total - base) : 256;
            float4 *o4 = reinterpret_cast<float4 *>(g_coef + base * W);
            for (int q = threadIdx.x; q < n * W / 4; q += 256) {
                const int f0 = 4 * q, r = f0 / W, c = f0 - r * W;  // W % 4 == 0: a float4 stays in its row
                const float *src = s_out + r * WP + c;
                o4[q] = make_float4(src[0], src[1], src[2], src[3]);
            }
            __syncthreads();
        } else if (e < total) {
            float *o = g_coef + e * W;
#pragma unroll
            for (int i = 0; i < W; ++i) o[i] = acc[i];
        }
    }
}

// The cameras of one scene, in camera order.
struct CamList {
    int32_t n;
    int16_t idx[kMaxCams];
};

// One thread per (splat, camera of scene si): the centre gradient through the
// view direction.  With S_m = sum over texels and channels of k_m C^,
// dL/dd = sum_m S_m grad Y_m(d), and dL/dp = (I - d d^T) dL/dd / |p - c|.
// Threads of a splat are consecutive; their centre gradients are summed over
// the warp (segmented by splat) before one atomic per value.  VEC: the
// coefficients and the record's grid gradient (N^2 a multiple of 4) are read
// with 16-byte loads.
template <int Dt, typename T, bool VEC>
__global__ void __launch_bounds__(256) texsh_centre_grad_kernel(Frame f, int si, CamList cl, const T *coef,
                                                               const float *grid_grad, float *g_means) {
    constexpr int M = (Dt + 1) * (Dt + 1);
    const SceneDev &sc = f.scenes[si];
    const int NN = sc.N * sc.N;
    const int64_t total = sc.K * cl.n;
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    // every lane of a warp runs the same iterations (the warp reduction below)
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < total; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < total;
        const int64_t k = valid ? e / cl.n : -1;
        float gp[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            const CamDev &cam = f.cams[cl.idx[int(e - k * cl.n)]];
            const float *gg = grid_grad + (cam.tex_row + k) * NN * 3;
            float S[M];
#pragma unroll
            for (int m = 0; m < M; ++m) S[m] = 0.0f;
            bool any = false;
            for (int t0 = 0; t0 < NN; t0 += VEC ? 4 : 1) {
                float h[12];
                if constexpr (VEC) {
                    const float4 *g4 = reinterpret_cast<const float4 *>(gg + 3 * t0);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float4 v = g4[i];
                        h[4 * i] = v.x; h[4 * i + 1] = v.y; h[4 * i + 2] = v.z; h[4 * i + 3] = v.w;
                    }
                } else {
                    h[0] = gg[3 * t0]; h[1] = gg[3 * t0 + 1]; h[2] = gg[3 * t0 + 2];
                }
#pragma unroll
                for (int j = 0; j < (VEC ? 4 : 1); ++j) {
                    const float h0 = h[3 * j], h1 = h[3 * j + 1], h2 = h[3 * j + 2];
                    if (h0 == 0.0f && h1 == 0.0f && h2 == 0.0f) continue;
                    any = true;
                    float kc[M * 3];
                    load_texel<M, T, VEC>(coef + (k * NN + t0 + j) * (M * 3), kc);
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        S[m] = fmaf(kc[3 * m], h0, fmaf(kc[3 * m + 1], h1, fmaf(kc[3 * m + 2], h2, S[m])));
                }
            }
            if (any) {
                const float p[3] = {sc.means[3 * k], sc.means[3 * k + 1], sc.means[3 * k + 2]};
                float d[3], dist;
                view_dir(p, cam, d, dist);
                float G[16][3];
                sh_basis_grad(Dt, d[0], d[1], d[2], G);
                float gd[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int m = 1; m < M; ++m) {
                    gd[0] = fmaf(S[m], G[m][0], gd[0]);
                    gd[1] = fmaf(S[m], G[m][1], gd[1]);
                    gd[2] = fmaf(S[m], G[m][2], gd[2]);
                }
                const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
                const float rd = 1.0f / dist;
                for (int i = 0; i < 3; ++i) gp[i] = (gd[i] - d[i] * dd) * rd;
            }
        }
        // segmented sum over lanes of the same splat (contiguous, k non-decreasing
        // with the lane): after the step with offset o, lane l holds the sum over
        // lanes [l, l + 2o) of its segment
        const int kl = int(k);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ko = __shfl_down_sync(0xffffffffu, kl, o);
            const bool same = lane + o < 32 && ko == kl;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float v = __shfl_down_sync(0xffffffffu, gp[i], o);
                if (same) gp[i] += v;
            }
        }
        const int kp = __shfl_up_sync(0xffffffffu, kl, 1);
        if (valid && (lane == 0 || kp != kl))
            for (int i = 0; i < 3; ++i)
                if (gp[i] != 0.0f) atomicAdd(g_means + 3 * k + i, gp[i]);
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int Dt, typename T>
void eval_t(const Frame &f, int si, const void *coef, float *out, unsigned grid, cudaStream_t s) {
    const T *c = static_cast<const T *>(coef);
    if (aligned16(coef)) texsh_eval_kernel<Dt, T, true><<<grid, 256, 0, s>>>(f, si, c, out);
    else texsh_eval_kernel<Dt, T, false><<<grid, 256, 0, s>>>(f, si, c, out);
}

template <int Dt>
void eval_d(const Frame &f, int si, const void *coef, int dtype, float *out, unsigned grid, cudaStream_t s) {
    switch (dtype) {
        case GB_F16: eval_t<Dt, __half>(f, si, coef, out, grid, s); break;
        case GB_BF16: eval_t<Dt, __nv_bfloat16>(f, si, coef, out, grid, s); break;
        default: eval_t<Dt, float>(f, si, coef, out, grid, s); break;
    }
}

template <int Dt, typename T>
void centre_t(const Frame &f, int si, const CamList &cl, const void *coef, const float *gg, float *g_means,
              unsigned grid, cudaStream_t s) {
    const T *c = static_cast<const T *>(coef);
    const int NN = f.scenes[si].N * f.scenes[si].N;
    if (aligned16(coef) && aligned16(gg) && NN % 4 == 0)
        texsh_centre_grad_kernel<Dt, T, true><<<grid, 256, 0, s>>>(f, si, cl, c, gg, g_means);
    else
        texsh_centre_grad_kernel<Dt, T, false><<<grid, 256, 0, s>>>(f, si, cl, c, gg, g_means);
}

template <int Dt>
void coef_grad(const Frame &f, int si, const float *gg, float *g_coef, unsigned grid, cudaStream_t s) {
    constexpr int W = (Dt + 1) * (Dt + 1) * 3;
    if constexpr (W % 4 == 0) {
        if (aligned16(g_coef)) {
            constexpr size_t smem = 256 * (W + 1) * sizeof(float);
            static bool configured = false;
            if (!configured) {
                cudaFuncSetAttribute(texsh_coef_grad_kernel<Dt, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem));
                configured = true;
            }
            texsh_coef_grad_kernel<Dt, true><<<grid, 256, smem, s>>>(f, si, gg, g_coef);
            return;
        }
    }
    texsh_coef_grad_kernel<Dt, false><<<grid, 256, 0, s>>>(f, si, gg, g_coef);
}

template <int Dt>
void grad_d(const Frame &f, int si, const CamList &cl, const void *coef, int dtype, const float *gg, float *g_coef,
            float *g_means, unsigned grid_tex, unsigned grid_cam, cudaStream_t s) {
    if (g_coef) {
        coef_grad<Dt>(f, si, gg, g_coef, grid_tex, s);
        count_launches(1);
    }
    if (g_means && cl.n) {
        switch (dtype) {
            case GB_F16: centre_t<Dt, __half>(f, si, cl, coef, gg, g_means, grid_cam, s); break;
            case GB_BF16: centre_t<Dt, __nv_bfloat16>(f, si, cl, coef, gg, g_means, grid_cam, s); break;
            default: centre_t<Dt, float>(f, si, cl, coef, gg, g_means, grid_cam, s); break;
        }
        count_launches(1);
    }
}

}  // namespace

cudaError_t launch_texsh_eval(const Frame &f, int si, int Dt, const void *coef, int dtype, float *out,
                              cudaStream_t s) {
    const int64_t n = f.scenes[si].K * f.scenes[si].N * f.scenes[si].N;
    if (n == 0) return cudaSuccess;
    const unsigned grid = grid_for(n);
    switch (Dt) {
        case 1: eval_d<1>(f, si, coef, dtype, out, grid, s); break;
        case 2: eval_d<2>(f, si, coef, dtype, out, grid, s); break;
        default: eval_d<3>(f, si, coef, dtype, out, grid, s); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_texsh_grad(const Frame &f, int si, int Dt, const void *coef, int dtype, const float *grid_grad,
                              float *g_coef, float *g_means, cudaStream_t s) {
    const int64_t K = f.scenes[si].K, n = K * f.scenes[si].N * f.scenes[si].N;
    if (n == 0) return cudaSuccess;
    CamList cl;
    cl.n = 0;
    for (int c = 0; c < f.n_cams; ++c)
        if (f.cams[c].scene == si) cl.idx[cl.n++] = int16_t(c);
    const unsigned gt = grid_for(n), gc = grid_for(K * cl.n);
    switch (Dt) {
        case 1: grad_d<1>(f, si, cl, coef, dtype, grid_grad, g_coef, g_means, gt, gc, s); break;
        case 2: grad_d<2>(f, si, cl, coef, dtype, grid_grad, g_coef, g_means, gt, gc, s); break;
        default: grad_d<3>(f, si, cl, coef, dtype, grid_grad, g_coef, g_means, gt, gc, s); break;
    }
    return cudaGetLastError();
}

}  // namespace gbill
