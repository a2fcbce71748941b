// Per-tile render helpers shared by the forward and backward kernels.
#pragma once

#include "gbill_internal.cuh"

namespace gbill {

// Pixel of thread `tid` in a TS x TS tile: each warp covers an 8 x 4 block so
// that its 32 pixels are compact (small splats touch few warps).
template <int TS>
__device__ __forceinline__ void tile_pixel(int tid, int &lx, int &ly) {
    const int lane = tid & 31, warp = tid >> 5;
    lx = (warp % (TS / 8)) * 8 + (lane & 7);
    ly = (warp / (TS / 8)) * 4 + (lane >> 3);
}

// Bytes of dynamic shared memory for one staged batch: records, colour
// grids, splat indices and (backward) record/grid gradient accumulators.
template <int N>
__host__ __device__ inline size_t stage_bytes(int batch, bool bwd) {
    const int texf = N * N * 3;
    size_t b = size_t(batch) * (64 + 4 * texf + 8);
    if (bwd) b += size_t(batch) * (4 * kRecGrad + 4 * texf);
    return b;
}

// Loads the records and colour grids of instances [first, first + nb) of a
// tile range into shared memory.  Caller synchronizes before and after.
template <int N, int NT, typename TexT>
__device__ __forceinline__ void stage_batch(const RenderBufs &b, const CamDev &cam, const SceneDev &sc,
                                            uint32_t first, int nb, float4 *s_rec, float *s_tex,
                                            int32_t *s_k, uint32_t *s_j) {
    constexpr int TEXF = N * N * 3;
    const int t = threadIdx.x;
    if (t < nb) {
        const uint32_t j = b.inst_val[first + t];
        const uint32_t r = b.perm[j];
        const float4 *rp = reinterpret_cast<const float4 *>(b.rec + r);
        s_rec[4 * t + 0] = rp[0];
        s_rec[4 * t + 1] = rp[1];
        s_rec[4 * t + 2] = rp[2];
        s_rec[4 * t + 3] = rp[3];
        s_k[t] = int32_t(int64_t(r) - cam.rec_off);
        s_j[t] = j;
    }
    __syncthreads();
    const TexT *tex = static_cast<const TexT *>(sc.tex);
    for (int e = t; e < nb * TEXF; e += NT) {
        const int s = e / TEXF, o = e - s * TEXF;
        s_tex[e] = load_as_float(tex, int64_t(s_k[s]) * TEXF + o);
    }
}

// Alg. 2 bilinear lookup coordinates: u' = clamp((N-1)(u+sigma)/(2 sigma)),
// cell index min(floor(u'), N-2) and fraction u' - index.
template <int N>
struct Cell {
    int base;    // offset of texel (i_u, i_v) in floats
    float fu, fv;
};

template <int N>
__device__ __forceinline__ Cell<N> grid_cell(float u, float v, float sigma, float kN) {
    Cell<N> c;
    if (N == 1) {
        c.base = 0;
        c.fu = c.fv = 0.0f;
        return c;
    }
    const float up = fminf(fmaxf((u + sigma) * kN, 0.0f), float(N - 1));
    const float vp = fminf(fmaxf((v + sigma) * kN, 0.0f), float(N - 1));
    const int iu = min(int(up), N - 2), iv = min(int(vp), N - 2);
    c.fu = up - float(iu);
    c.fv = vp - float(iv);
    c.base = (iu * N + iv) * 3;
    return c;
}

template <int N>
__device__ __forceinline__ void grid_colour(const float *g, const Cell<N> &c, float col[3]) {
    if (N == 1) {
        col[0] = g[0]; col[1] = g[1]; col[2] = g[2];
        return;
    }
    const float *p00 = g + c.base, *p10 = p00 + 3 * N, *p01 = p00 + 3, *p11 = p10 + 3;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float a = fmaf(c.fu, p10[ch] - p00[ch], p00[ch]);
        const float bb = fmaf(c.fu, p11[ch] - p01[ch], p01[ch]);
        col[ch] = fmaf(c.fv, bb - a, a);
    }
}

// exp(-rho / 2) through the SFU exponential.
__device__ __forceinline__ float gauss(float rho) { return __expf(-0.5f * rho); }

}  // namespace gbill
