// Forward per-tile render (Alg. 1 fwd with the colour grid of Eq. 5).
//
// One block per TS x TS tile, two pixels per thread (one at N = 16): warp w
// owns an 8 x 8 block of the tile, lane l the pixels (l % 8, l / 8) and
// (l % 8, l / 8 + 4) of it, so a splat's record and warp-block mask bit are
// read once for two pixels (measured on the 1M-splat, 16-view workload:
// 13.1 -> 9.9 ms against one pixel per thread with 8 x 4 warp blocks, although
// the coarser blocks evaluate 19 % more pairs).  The tile's depth-sorted
// splats are staged in batches (record, footprint, warp-block masks, colour
// grid) in shared memory; every pixel walks them front to back:
//   zeta = adj(T') (dx, dy, 1)                (ray/splat intersection)
//   rho  = min(u^2 + v^2, 2 |x - c|^2)        (Eq. 4 plus screen low-pass)
//   alpha = min(0.99, o exp(-rho/2)), skipped below 1/255
//   stop before T (1 - alpha) < 1e-4
//   c = bilinear(C_k, u, v) + SH colour       (Eq. 5, Alg. 2, Sec. 4.2)
//   C += c alpha T, D += z alpha T, T *= 1 - alpha   (Eq. 2)
// Saved for the backward: final T and 1 + index of the last blended splat.
#include <algorithm>

#include "render_common.cuh"

namespace gbill {
namespace {

// Forward state of one pixel.
struct FPix {
    float xf, yf, T, C0, C1, C2, Dp;
    uint32_t last;
    bool inside, done;
};

// One (pixel, splat) pair of the front-to-back walk: evaluated by every lane of
// the warp (a finished pixel's result is dropped), blended only where alpha
// passes the cutoff and the pixel's transmittance stays above the stop bound.
// VAR: the splat's grid is nk x nk (per-splat grid size), kN = (nk - 1) / (2 sigma).
template <int N, typename TexT, bool WIDE, bool VAR>
__device__ __forceinline__ void fwd_pair(FPix &q, const Hit &h, const float4 &q1, const float4 &q3,
                                         const staged_t<TexT, WIDE> *tex, uint32_t idx1, float sigma, float kN,
                                         int nk, uint32_t &npairs, uint32_t &nblend) {
    npairs += q.done ? 0u : 1u;
    const float zz = h.zz;
    const float rz = fast_rcp(zz);
    const float u = h.zx * rz;
    const float v = h.zy * rz;
    const float ruv = fmaf(u, u, v * v);
    const float rlp = kLowPass * fmaf(h.dx, h.dx, h.dy * h.dy);
    const bool uvb = ruv <= rlp;
    const float rho = uvb ? ruv : rlp;
    const float alpha = fminf(kAlphaMax, q3.x * gauss(rho));
    const float tT = q.T * (1.0f - alpha);
    const bool hit = !q.done && zz != 0.0f && alpha >= kAlphaMin;
    q.done = q.done || (hit && tT < kTMin);
    if (hit && !(tT < kTMin)) {
        const Cell<N> cell = VAR ? grid_cell_n<N>(u, v, sigma, kN, nk) : grid_cell<N>(u, v, sigma, kN);
        float col[3];
        grid_colour<N>(grid_quad<N, TexT, WIDE>(tex, cell), cell, col);
        const float w = alpha * q.T;
        q.C0 = fmaf(col[0] + q3.y, w, q.C0);
        q.C1 = fmaf(col[1] + q3.z, w, q.C1);
        q.C2 = fmaf(col[2] + q3.w, w, q.C2);
        const float z = fabsf(q1.w);  // negated on flagged records
        const float zi = uvb ? q1.z * z * rz : z;
        q.Dp = fmaf(zi, w, q.Dp);
        q.T = tT;
        q.last = idx1;
        ++nblend;
    }
}

template <int TS, int N, typename TexT, int P, bool VAR>
__device__ __forceinline__ void fwd_tile(const Frame &f, const RenderBufs &b, int batch, uint32_t tile) {
    constexpr int NT = TS * TS / P;
    constexpr int NN = N * N;
    extern __shared__ float4 smem[];
    float4 *s_rec = smem;
    float4 *s_fp = s_rec + 4 * batch;  // [batch][3] footprints
    constexpr bool WIDE = N <= 4;  // grids staged as FP32 RGBA (room to spare in the forward)
    staged_t<TexT, WIDE> *s_tex = reinterpret_cast<staged_t<TexT, WIDE> *>(s_fp + 3 * batch);
    int32_t *s_k = reinterpret_cast<int32_t *>(s_tex + batch * NN);
    uint32_t *s_j = reinterpret_cast<uint32_t *>(s_k + batch);
    uint2 *s_box = reinterpret_cast<uint2 *>(s_j + batch);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_box + batch);
    int32_t *s_n = reinterpret_cast<int32_t *>(s_mask + batch);  // VAR: per-splat grid size

    const int ci = camera_of_tile(f, tile);
    const CamDev &cam = f.cams[ci];
    const SceneDev &sc = f.scenes[cam.scene];
    const uint32_t lt = tile - cam.tile_off;
    const int tx = int(lt % uint32_t(cam.tiles_x)), ty = int(lt / uint32_t(cam.tiles_x));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbit = 1u << warp;  // this warp's 8 x 4P block in the splat masks
    const int px = tx * TS + (warp % (TS / 8)) * 8 + (lane & 7);
    const int py0 = ty * TS + (warp / (TS / 8)) * (4 * P) + (lane >> 3);
    const uint2 range = b.ranges[tile];
    const int n_inst = int(range.y - range.x);
    const float sigma = sc.sigma;
    const float kN = float(N - 1) / (2.0f * sigma);

    FPix pix[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        FPix &q = pix[p];
        q.inside = px < cam.width && py0 + 4 * p < cam.height;
        q.xf = float(px) + 0.5f;
        q.yf = float(py0 + 4 * p) + 0.5f;
        q.T = 1.0f;
        q.C0 = q.C1 = q.C2 = q.Dp = 0.0f;
        q.last = 0;
        q.done = !q.inside;
    }
    uint32_t npairs = 0, nblend = 0;
    auto all_done = [&]() {
        bool d = true;
#pragma unroll
        for (int p = 0; p < P; ++p) d = d && pix[p].done;
        return d;
    };
    for (int bs = 0; bs < n_inst; bs += batch) {
        if (__syncthreads_count(all_done()) == NT) break;
        const int nb = min(batch, n_inst - bs);
        stage_batch<N, NT, TexT, TS, 4 * P, WIDE, VAR>(b, cam, sc, range.x + bs, nb, tx * TS, ty * TS, s_rec, s_tex,
                                                      s_k, s_j, s_box, s_mask, s_fp, s_n);
        __syncthreads();
        // the staged splats whose footprint may touch this warp's block, front to
        // back, 32 at a time from a ballot of their masks (measured against
        // testing every staged splat: 11.1 -> 9.9 ms at N = 4, 26.0 -> 23.7 ms at
        // N = 16 on the 16-view workload); the warp stops once all its pixels are
        // done, checked every 16 splats it evaluates
        bool stop = false;
        for (int c = 0; c < nb && !stop; c += 32) {
            unsigned wd = __ballot_sync(0xffffffffu, c + lane < nb && (s_mask[c + lane] & wbit));
            for (int ev = 0; wd; ++ev) {
            if ((ev & 15) == 0 && __all_sync(0xffffffffu, all_done())) {
                stop = true;
                break;
            }
            const int i = c + __ffs(wd) - 1;
            wd &= wd - 1u;
            const float4 q0 = s_rec[4 * i + 0], q1 = s_rec[4 * i + 1], q2 = s_rec[4 * i + 2],
                         q3 = s_rec[4 * i + 3];
            const int nk = VAR ? s_n[i] : N;
            const float kNk = VAR ? float(nk - 1) / (2.0f * sigma) : kN;
            if (q1.w < 0.0f) {
                // flagged record (the same for the whole warp): extended-precision plane hit
                const RecordLo L = b.rec_lo[staged_record(cam, s_k[i])];
#pragma unroll
                for (int p = 0; p < P; ++p)
                    fwd_pair<N, TexT, WIDE, VAR>(pix[p], plane_hit_ext(pix[p].xf, pix[p].yf, q0, q1, q2, L), q1, q3,
                                                 s_tex + i * NN, uint32_t(bs + i + 1), sigma, kNk, nk, npairs, nblend);
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    fwd_pair<N, TexT, WIDE, VAR>(pix[p], plane_hit(pix[p].xf, pix[p].yf, q0, q1, q2), q1, q3,
                                                 s_tex + i * NN, uint32_t(bs + i + 1), sigma, kNk, nk, npairs, nblend);
            }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        nblend += __shfl_xor_sync(0xffffffffu, nblend, o);
    }
    if (lane == 0 && npairs) atomicAdd(&b.cnt->pairs_fwd, (unsigned long long)npairs);
    if (lane == 0 && nblend) atomicAdd(&b.cnt->blend_fwd, (unsigned long long)nblend);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const FPix &q = pix[p];
        if (!q.inside) continue;
        const int64_t pi = cam.pix_off + int64_t(py0 + 4 * p) * cam.width + px;
        b.rgb[3 * pi + 0] = q.C0 + q.T * f.bg[0];
        b.rgb[3 * pi + 1] = q.C1 + q.T * f.bg[1];
        b.rgb[3 * pi + 2] = q.C2 + q.T * f.bg[2];
        if (b.depth) b.depth[pi] = q.Dp;
        if (b.alpha) b.alpha[pi] = 1.0f - q.T;
        b.t_final[pi] = q.T;
        b.last[pi] = q.last;
    }
}

// Pixels per thread of the forward: two, but one at N = 16, where the larger
// grid lookups of two pixels per thread cost more than the shared record
// reads save (28.5 against 25.4 ms on the 16-view workload).
template <int N>
__host__ __device__ constexpr int fwd_ppt() {
    return N >= 16 ? 1 : 2;
}

// Resident blocks per SM the register budget is sized for: 1536 threads (six
// blocks of 16 x 16 tiles), but 1280 at N = 16, one pixel per thread, where
// the 40-register cap of 1536 spilled 104 bytes (measured on the 16-view
// workload, images identical: 25.68 ms at six blocks, 24.96 at five with 48
// registers, 25.77 at four with 62).
template <int TS, int N>
__host__ __device__ constexpr int fwd_min_blocks() {
    return (N >= 16 ? 1280 : 1536) / (TS * TS);
}

template <int TS, int N, typename TexT, bool VAR>
__global__ void __launch_bounds__(TS * TS / fwd_ppt<N>(), fwd_min_blocks<TS, N>())
    render_fwd_kernel(Frame f, RenderBufs b, int batch, TileSched ts) {
    __shared__ uint32_t s_next;
    for (int round = 0;; ++round) {
        uint32_t idx;
        if (ts.work) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(ts.work, 1u);
            __syncthreads();
            idx = s_next;
        } else {
            if (round) break;
            idx = blockIdx.x;
        }
        if (idx >= ts.count) break;
        const uint32_t tile = ts.list ? ts.list[ts.off + idx] : ts.off + idx;
        fwd_tile<TS, N, TexT, fwd_ppt<N>(), VAR>(f, b, batch, tile);
    }
}

template <int TS, int N, typename TexT, bool VAR = false>
cudaError_t launch_t(const Frame &f, const RenderBufs &b, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    const size_t smem = stage_bytes<N, TexT, (N <= 4)>(batch, false) + (VAR ? size_t(batch) * 4 : 0);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(render_fwd_kernel<TS, N, TexT, VAR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned grid = ts.count;
    if (persistent) {
        static int per_sm = 0, sms = 0;
        static size_t smem_seen = 0;
        if (!per_sm || smem_seen != smem) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_fwd_kernel<TS, N, TexT, VAR>,
                                                          TS * TS / fwd_ppt<N>(), smem);
            smem_seen = smem;
            if (per_sm < 1) per_sm = 1;
        }
        grid = std::min<unsigned>(grid, unsigned(per_sm * sms));
    } else {
        ts.work = nullptr;
    }
    if (grid == 0) return cudaSuccess;
    render_fwd_kernel<TS, N, TexT, VAR><<<grid, TS * TS / fwd_ppt<N>(), smem, s>>>(f, b, batch, ts);
    count_launches(1);
    return cudaGetLastError();
}

template <int TS, typename TexT>
cudaError_t launch_n(const Frame &f, const RenderBufs &b, int N, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    switch (N) {
        case 1: return launch_t<TS, 1, TexT>(f, b, batch, ts, persistent, s);
        case 2: return launch_t<TS, 2, TexT>(f, b, batch, ts, persistent, s);
        case 4: return launch_t<TS, 4, TexT>(f, b, batch, ts, persistent, s);
        case 8: return launch_t<TS, 8, TexT>(f, b, batch, ts, persistent, s);
        case 16: return launch_t<TS, 16, TexT>(f, b, batch, ts, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

// Per-splat grid sizes (16 x 16 tiles): N is the grid block of the scene.
template <typename TexT>
cudaError_t launch_var(const Frame &f, const RenderBufs &b, int N, int batch, TileSched ts, bool persistent,
                       cudaStream_t s) {
    switch (N) {
        case 2: return launch_t<16, 2, TexT, true>(f, b, batch, ts, persistent, s);
        case 4: return launch_t<16, 4, TexT, true>(f, b, batch, ts, persistent, s);
        case 8: return launch_t<16, 8, TexT, true>(f, b, batch, ts, persistent, s);
        case 16: return launch_t<16, 16, TexT, true>(f, b, batch, ts, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int TS>
cudaError_t launch_d(const Frame &f, const RenderBufs &b, int g, int N, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    if (f.group_var[g]) {
        if (TS != 16) return cudaErrorInvalidValue;
        switch (f.group_dtype[g]) {
            case GB_F16: return launch_var<__half>(f, b, N, batch, ts, persistent, s);
            case GB_BF16: return launch_var<__nv_bfloat16>(f, b, N, batch, ts, persistent, s);
            default: return launch_var<float>(f, b, N, batch, ts, persistent, s);
        }
    }
    switch (f.group_dtype[g]) {
        case GB_F16: return launch_n<TS, __half>(f, b, N, batch, ts, persistent, s);
        case GB_BF16: return launch_n<TS, __nv_bfloat16>(f, b, N, batch, ts, persistent, s);
        default: return launch_n<TS, float>(f, b, N, batch, ts, persistent, s);
    }
}

}  // namespace

cudaError_t launch_render_fwd(const Frame &f, const RenderBufs &b, int batch, const uint32_t *tile_list,
                              uint32_t *work, bool persistent, cudaStream_t s) {
    if (f.n_tiles == 0) return cudaSuccess;
    for (int g = 0; g < f.n_groups; ++g) {
        TileSched ts;
        ts.list = tile_list;
        ts.off = tile_list ? f.group_off[g] : 0;
        ts.count = tile_list ? f.group_count[g] : f.n_tiles;
        ts.work = work ? work + g : nullptr;
        const int N = f.group_N[g];
        cudaError_t e;
        switch (f.tile) {
            case 8: e = launch_d<8>(f, b, g, N, batch, ts, persistent, s); break;
            case 16: e = launch_d<16>(f, b, g, N, batch, ts, persistent, s); break;
            case 32: e = launch_d<32>(f, b, g, N, batch, ts, persistent, s); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbill
