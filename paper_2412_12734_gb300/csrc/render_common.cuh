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

// The 8 x 4 pixel block of a warp misses a splat's inclusive pixel rectangle:
// every pixel of the block has alpha < 1/255 for that splat, so the whole
// warp skips it (the same rectangle decides tile membership).
struct WarpBox {
    int x0, y0, x1, y1;
    __device__ __forceinline__ bool misses(uint2 b) const {
        return int(b.x & 0xffffu) > x1 || int(b.y & 0xffffu) < x0 || int(b.x >> 16) > y1 || int(b.y >> 16) < y0;
    }
};

template <int TS>
__device__ __forceinline__ WarpBox warp_box(int tx, int ty, int tid) {
    const int warp = tid >> 5;
    WarpBox w;
    w.x0 = tx * TS + (warp % (TS / 8)) * 8;
    w.y0 = ty * TS + (warp / (TS / 8)) * 4;
    w.x1 = w.x0 + 7;
    w.y1 = w.y0 + 3;
    return w;
}

// Bytes of dynamic shared memory for one staged batch: records, colour
// grids, splat indices and (backward) record/grid gradient accumulators.
// Colour grids are staged as RGBA float4 texels (16 bytes, alpha unused) so a
// texel is one 128-bit shared load.
template <int N>
__host__ __device__ inline size_t stage_bytes(int batch, bool bwd) {
    const int texf = N * N * 3;
    size_t b = size_t(batch) * (64 + 16 * N * N + 16);
    if (bwd) b += size_t(batch) * (4 * kRecGrad + 4 * texf);
    return b;
}

// 1 / x through the SFU (max error 1 ulp; flush-to-zero).
__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Loads the records and colour grids of instances [first, first + nb) of a
// tile range into shared memory.  Caller synchronizes before and after.
template <int N, int NT, typename TexT>
__device__ __forceinline__ void stage_batch(const RenderBufs &b, const CamDev &cam, const SceneDev &sc,
                                            uint32_t first, int nb, float4 *s_rec, float4 *s_tex,
                                            int32_t *s_k, uint32_t *s_j, uint2 *s_box) {
    constexpr int NN = N * N;
    const int t = threadIdx.x;
    if (t < nb) {
        const uint32_t j = b.inst_val[first + t];
        const uint32_t r = b.perm[j];
        s_box[t] = b.pbox[r];
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
    for (int e = t; e < nb * NN; e += NT) {
        const int s = e / NN, o = e - s * NN;
        const int64_t g = (int64_t(s_k[s]) * NN + o) * 3;
        s_tex[e] = make_float4(load_as_float(tex, g), load_as_float(tex, g + 1), load_as_float(tex, g + 2), 0.0f);
    }
}

// Alg. 2 bilinear lookup coordinates: u' = clamp((N-1)(u+sigma)/(2 sigma)),
// cell index min(floor(u'), N-2) and fraction u' - index.
template <int N>
struct Cell {
    int base;    // index of texel (i_u, i_v) in the N x N grid
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
    c.base = iu * N + iv;
    return c;
}

// The four texels of a cell: (i_u, i_v), (i_u+1, i_v), (i_u, i_v+1), (i_u+1, i_v+1).
struct Quad {
    float4 c00, c10, c01, c11;
};

template <int N>
__device__ __forceinline__ Quad grid_quad(const float4 *g, const Cell<N> &c) {
    Quad q;
    q.c00 = g[c.base];
    if (N == 1) {
        q.c10 = q.c01 = q.c11 = q.c00;
    } else {
        q.c10 = g[c.base + N];
        q.c01 = g[c.base + 1];
        q.c11 = g[c.base + N + 1];
    }
    return q;
}

__device__ __forceinline__ float lerp2(float a00, float a10, float a01, float a11, float fu, float fv) {
    const float a = fmaf(fu, a10 - a00, a00);
    const float b = fmaf(fu, a11 - a01, a01);
    return fmaf(fv, b - a, a);
}

template <int N>
__device__ __forceinline__ void grid_colour(const Quad &q, const Cell<N> &c, float col[3]) {
    if (N == 1) {
        col[0] = q.c00.x; col[1] = q.c00.y; col[2] = q.c00.z;
        return;
    }
    col[0] = lerp2(q.c00.x, q.c10.x, q.c01.x, q.c11.x, c.fu, c.fv);
    col[1] = lerp2(q.c00.y, q.c10.y, q.c01.y, q.c11.y, c.fu, c.fv);
    col[2] = lerp2(q.c00.z, q.c10.z, q.c01.z, q.c11.z, c.fu, c.fv);
}

// exp(-rho / 2) through the SFU exponential.
__device__ __forceinline__ float gauss(float rho) { return __expf(-0.5f * rho); }

}  // namespace gbill
