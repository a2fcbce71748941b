// Backward per-tile render with a splat-parallel inner loop (Alg. 1 bwd with
// Alg. 2 adj-bilinear), for grids of N <= 4 on 8 x 8 and 16 x 16 tiles.
//
// Staging and batches are those of the pixel-parallel kernel (render_bwd.cuh):
// one block per tile, the tile's depth-sorted splats staged in shared memory a
// batch at a time, back to front, with the mask of the tile's 8 x 4 warp
// blocks each splat's footprint may touch.  The difference is the warp's
// loop.  Each warp lists the batch's splats that touch its 32 pixels (back to
// front) and takes them 32 at a time, one per lane; for each of its pixels in
// turn every lane evaluates its splat there, and two warp prefix scans over
// the lanes (back to front) give each lane what the sequential walk of Alg. 1
// bwd would: the transmittance in front of its splat, T_j = T_s prod_{k<=j}
// 1 / (1 - alpha_k), and the colour and depth blended behind it, S_j = S_s +
// sum_{k<j} c_k alpha_k T_k, from the pixel's state (T_s, S_s) behind the
// chunk, which then moves in front of it.  A lane adds its splat's record
// gradient (kRecGrad layout) and texel gradients in registers across the
// pixels, so no value is reduced across lanes; per chunk the sums go to the
// batch's shared accumulators once (texel sums also when the splat's grid
// cell changes), and per batch to global memory as in the pixel-parallel
// kernel.
#include <algorithm>

#include "render_common.cuh"

namespace gbill {
namespace bwdsp {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Shared memory of one staged batch: the pixel-parallel layout plus one list
// of batch indices (uint16) per warp.
template <int TS, int N, typename TexT>
__host__ __device__ inline size_t sp_stage_bytes(int batch) {
    constexpr int NW = TS * TS / 32;
    return stage_bytes<N, TexT>(batch, true) + ((size_t(NW) * batch * 2 + 15) & ~size_t(15));
}

// Texel-gradient sums of one grid cell (four texels x RGB) of a lane's splat,
// flushed to the batch's shared accumulator when the cell changes.
template <int N>
struct CellAcc {
    float v[12];
    int base;  // texel index (i_u N + i_v) of the cell's first texel, -1: empty
};

template <int N>
__device__ __forceinline__ void flush_cell(CellAcc<N> &a, float *tg) {
    if (a.base < 0) return;
    // k: 0 -> (iu, iv), 1 -> (iu+1, iv), 2 -> (iu, iv+1), 3 -> (iu+1, iv+1)
#pragma unroll
    for (int k = 0; k < (N == 1 ? 1 : 4); ++k) {
        const int t = a.base + ((k & 1) ? N : 0) + ((k & 2) ? 1 : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = a.v[3 * k + c];
            if (x != 0.0f) atomicAdd(tg + 3 * t + c, x);
            a.v[3 * k + c] = 0.0f;
        }
    }
    a.base = -1;
}

template <int TS, int N, typename TexT>
__device__ __forceinline__ void sp_tile(const Frame &f, const RenderBwdBufs &b, int batch, uint32_t tile) {
    constexpr int NT = TS * TS;
    constexpr int NN = N * N;
    constexpr int TEXF = NN * 3;
    constexpr uint32_t FULL = 0xffffffffu;
    extern __shared__ float4 smem[];
    float4 *s_rec = smem;
    float4 *s_fp = s_rec + 4 * batch;
    staged_t<TexT> *s_tex = reinterpret_cast<staged_t<TexT> *>(s_fp + 3 * batch);
    int32_t *s_k = reinterpret_cast<int32_t *>(s_tex + batch * NN);
    uint32_t *s_j = reinterpret_cast<uint32_t *>(s_k + batch);
    uint2 *s_box = reinterpret_cast<uint2 *>(s_j + batch);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_box + batch);
    float *s_g = reinterpret_cast<float *>(s_mask + batch);  // [batch][kRecGrad]
    float *s_tg = s_g + batch * kRecGrad;                    // [batch][TEXF]
    uint16_t *s_list = reinterpret_cast<uint16_t *>(s_tg + batch * TEXF);
    __shared__ uint32_t s_maxlast;

    const int ci = camera_of_tile(f, tile);
    const CamDev &cam = f.cams[ci];
    const SceneDev &sc = f.scenes[cam.scene];
    const uint32_t lt = tile - cam.tile_off;
    const int tx = int(lt % uint32_t(cam.tiles_x)), ty = int(lt / uint32_t(cam.tiles_x));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbit = 1u << warp;
    const int bx0 = tx * TS + (warp % (TS / 8)) * 8, by0 = ty * TS + (warp / (TS / 8)) * 4;
    const uint2 range = b.fw.ranges[tile];
    const float sigma = sc.sigma;
    const float kN = float(N - 1) / (2.0f * sigma);
    uint16_t *my_list = s_list + warp * batch;

    // this lane's pixel (lane l: (l % 8, l / 8) of the warp's 8 x 4 block) and its reverse-walk state
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < cam.width && py < cam.height;
    float pT = 1.0f, pS0 = 0.0f, pS1 = 0.0f, pS2 = 0.0f, pSD = 0.0f;
    float pdC0 = 0.0f, pdC1 = 0.0f, pdC2 = 0.0f, pdD = 0.0f, pdT = 0.0f;
    uint32_t plast = 0;
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (inside) {
        const int64_t pi = cam.pix_off + int64_t(py) * cam.width + px;
        pT = b.fw.t_final[pi];
        plast = b.fw.last[pi];
        pdC0 = b.d_rgb[3 * pi + 0];
        pdC1 = b.d_rgb[3 * pi + 1];
        pdC2 = b.d_rgb[3 * pi + 2];
        if (b.d_depth) pdD = b.d_depth[pi];
        const float dA = b.d_alpha ? b.d_alpha[pi] : 0.0f;
        pdT = (dA - (pdC0 * f.bg[0] + pdC1 * f.bg[1] + pdC2 * f.bg[2])) * pT;  // times 1/(1-alpha) per splat
    }
    const uint32_t wlast = __reduce_max_sync(FULL, plast);
    if (lane == 0 && wlast) atomicMax(&s_maxlast, wlast);
    __syncthreads();
    const int max_last = int(s_maxlast);
    float *g_tex = sc.g_tex;
    uint32_t npairs = 0;

    for (int be = max_last; be > 0; be -= batch) {
        const int bs = max(0, be - batch), nb = be - bs;
        for (int e = threadIdx.x; e < nb * kRecGrad; e += NT) s_g[e] = 0.0f;
        for (int e = threadIdx.x; e < nb * TEXF; e += NT) s_tg[e] = 0.0f;
        stage_batch<N, NT, TexT, TS, 4>(b.fw, cam, sc, range.x + bs, nb, tx * TS, ty * TS, s_rec, s_tex, s_k, s_j,
                                        s_box, s_mask, s_fp);
        __syncthreads();
        // the warp's list: splats touching its block, in front of its last contributor, back to front
        const int i_hi = min(nb, int(wlast) - bs);
        int n_list = 0;
        for (int base = i_hi - 1; base >= 0; base -= 32) {
            const int i = base - lane;
            const bool t = i >= 0 && (s_mask[i] & wbit);
            const uint32_t bal = __ballot_sync(FULL, t);
            if (t) my_list[n_list + __popc(bal & lanemask_lt())] = uint16_t(i);
            n_list += __popc(bal);
        }
        __syncwarp();
        for (int c0 = 0; c0 < n_list; c0 += 32) {
            // this lane's splat of the chunk (lane 0 the backmost)
            const bool active = c0 + lane < n_list;
            const int slot = active ? int(my_list[c0 + lane]) : 0;
            const float4 q0 = s_rec[4 * slot + 0], q1 = s_rec[4 * slot + 1], q2 = s_rec[4 * slot + 2],
                         q3 = s_rec[4 * slot + 3];
            const bool flagged = q1.w < 0.0f;
            const RecordLo *lo = b.fw.rec_lo + staged_record(cam, s_k[slot]);
            const staged_t<TexT> *tex = s_tex + slot * NN;
            const uint32_t idx = uint32_t(bs + slot);
            const float z = fabsf(q1.w);  // negated on flagged records
            float acc[kRecVals];
#pragma unroll
            for (int q = 0; q < kRecVals; ++q) acc[q] = 0.0f;
            CellAcc<N> ca;
#pragma unroll
            for (int q = 0; q < 12; ++q) ca.v[q] = 0.0f;
            ca.base = -1;
            for (int p = 0; p < 32; ++p) {
                const int qx = bx0 + (p & 7), qy = by0 + (p >> 3);
                if (qx >= cam.width || qy >= cam.height) continue;  // uniform
                const uint32_t last_p = __shfl_sync(FULL, plast, p);
                const float xf = float(qx) + 0.5f, yf = float(qy) + 0.5f;
                const Hit h = flagged ? plane_hit_ext(xf, yf, q0, q1, q2, *lo) : plane_hit(xf, yf, q0, q1, q2);
                const float zz = h.zz;
                const float rz = fast_rcp(zz);
                const float u = h.zx * rz, v = h.zy * rz;
                const float ruv = fmaf(u, u, v * v);
                const float rlp = kLowPass * fmaf(h.dx, h.dx, h.dy * h.dy);
                const bool uvb = ruv <= rlp;
                const float G = gauss(uvb ? ruv : rlp);
                const float ar = q3.x * G;
                const bool clamped = ar > kAlphaMax;
                const float alpha = clamped ? kAlphaMax : ar;
                const bool inrange = active && idx < last_p;
                const bool live = inrange && zz != 0.0f && alpha >= kAlphaMin;
                npairs += inrange ? 1u : 0u;
                if (!__any_sync(FULL, live)) continue;
                // transmittance in front of each lane's splat: prefix product over the lanes behind
                const float iom = live ? fast_rcp(1.0f - alpha) : 1.0f;
                float R = iom;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y = __shfl_up_sync(FULL, R, o);
                    if (lane >= o) R *= y;
                }
                const float Tb = __shfl_sync(FULL, pT, p);
                const float Ti = Tb * R;
                const float w = live ? alpha * Ti : 0.0f;
                // colour and depth of the pair
                float col[3] = {0.0f, 0.0f, 0.0f};
                Cell<N> cell;
                Quad qd;
                cell.base = 0;
                cell.fu = cell.fv = 0.0f;
                if (live) {
                    cell = grid_cell<N>(u, v, sigma, kN);
                    qd = grid_quad<N, TexT>(tex, cell);
                    grid_colour<N>(qd, cell, col);
                    col[0] += q3.y;
                    col[1] += q3.z;
                    col[2] += q3.w;
                }
                const float zi = uvb ? q1.z * z * rz : z;
                // colour and depth blended behind each lane's splat: exclusive prefix sums
                float e0 = col[0] * w, e1 = col[1] * w, e2 = col[2] * w, e3 = zi * w;
                const float o0 = e0, o1 = e1, o2 = e2, o3 = e3;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y0 = __shfl_up_sync(FULL, e0, o), y1 = __shfl_up_sync(FULL, e1, o);
                    const float y2 = __shfl_up_sync(FULL, e2, o), y3 = __shfl_up_sync(FULL, e3, o);
                    if (lane >= o) {
                        e0 += y0;
                        e1 += y1;
                        e2 += y2;
                        e3 += y3;
                    }
                }
                const float S0 = __shfl_sync(FULL, pS0, p) + (e0 - o0);
                const float S1 = __shfl_sync(FULL, pS1, p) + (e1 - o1);
                const float S2 = __shfl_sync(FULL, pS2, p) + (e2 - o2);
                const float SD = __shfl_sync(FULL, pSD, p) + (e3 - o3);
                const float dC0 = __shfl_sync(FULL, pdC0, p), dC1 = __shfl_sync(FULL, pdC1, p);
                const float dC2 = __shfl_sync(FULL, pdC2, p), dD = __shfl_sync(FULL, pdD, p);
                const float dT = __shfl_sync(FULL, pdT, p);
                // the pixel's state moves in front of the chunk (lane 31 holds the totals)
                const float Tn = __shfl_sync(FULL, Ti, 31);
                const float a0 = __shfl_sync(FULL, e0, 31), a1 = __shfl_sync(FULL, e1, 31);
                const float a2 = __shfl_sync(FULL, e2, 31), a3 = __shfl_sync(FULL, e3, 31);
                if (lane == p) {
                    pT = Tn;
                    pS0 += a0;
                    pS1 += a1;
                    pS2 += a2;
                    pSD += a3;
                }
                if (!live) continue;
                // adjoints of the pair (as in the pixel-parallel kernel)
                const float ch0 = w * dC0, ch1 = w * dC1, ch2 = w * dC2;
                acc[kGRgb + 0] += ch0;
                acc[kGRgb + 1] += ch1;
                acc[kGRgb + 2] += ch2;
                float uh = 0.0f, vh = 0.0f;
                if (N == 1) {
                    ca.base = 0;
                    ca.v[0] += ch0;
                    ca.v[1] += ch1;
                    ca.v[2] += ch2;
                } else {
                    const float fu = cell.fu, fv = cell.fv;
                    const float w00 = (1.0f - fu) * (1.0f - fv), w10 = fu * (1.0f - fv);
                    const float w01 = (1.0f - fu) * fv, w11 = fu * fv;
                    const float fuh = ch0 * ((qd.c10.x - qd.c00.x) * (1.0f - fv) + (qd.c11.x - qd.c01.x) * fv) +
                                      ch1 * ((qd.c10.y - qd.c00.y) * (1.0f - fv) + (qd.c11.y - qd.c01.y) * fv) +
                                      ch2 * ((qd.c10.z - qd.c00.z) * (1.0f - fv) + (qd.c11.z - qd.c01.z) * fv);
                    const float fvh = ch0 * ((qd.c01.x - qd.c00.x) * (1.0f - fu) + (qd.c11.x - qd.c10.x) * fu) +
                                      ch1 * ((qd.c01.y - qd.c00.y) * (1.0f - fu) + (qd.c11.y - qd.c10.y) * fu) +
                                      ch2 * ((qd.c01.z - qd.c00.z) * (1.0f - fu) + (qd.c11.z - qd.c10.z) * fu);
                    if (cell.base != ca.base) flush_cell<N>(ca, s_tg + slot * TEXF);
                    ca.base = cell.base;
                    ca.v[0] = fmaf(w00, ch0, ca.v[0]); ca.v[1] = fmaf(w00, ch1, ca.v[1]); ca.v[2] = fmaf(w00, ch2, ca.v[2]);
                    ca.v[3] = fmaf(w10, ch0, ca.v[3]); ca.v[4] = fmaf(w10, ch1, ca.v[4]); ca.v[5] = fmaf(w10, ch2, ca.v[5]);
                    ca.v[6] = fmaf(w01, ch0, ca.v[6]); ca.v[7] = fmaf(w01, ch1, ca.v[7]); ca.v[8] = fmaf(w01, ch2, ca.v[8]);
                    ca.v[9] = fmaf(w11, ch0, ca.v[9]); ca.v[10] = fmaf(w11, ch1, ca.v[10]); ca.v[11] = fmaf(w11, ch2, ca.v[11]);
                    if (u > -sigma && u < sigma) uh = kN * fuh;
                    if (v > -sigma && v < sigma) vh = kN * fvh;
                }
                float ah = dC0 * (col[0] * Ti - S0 * iom) + dC1 * (col[1] * Ti - S1 * iom) +
                           dC2 * (col[2] * Ti - S2 * iom);
                ah += dD * (zi * Ti - SD * iom) + dT * iom;
                const float zih = dD * w;
                float rhoh = 0.0f;
                if (!clamped) {
                    acc[kGOpacity] += ah * G;
                    rhoh = -0.5f * alpha * ah;
                }
                float W;
                if (uvb) {
                    uh = fmaf(2.0f * u, rhoh, uh);
                    vh = fmaf(2.0f * v, rhoh, vh);
                    W = -zih * zi;
                } else {
                    const float cl = -2.0f * kLowPass * rhoh;
                    acc[kGCentreLP + 0] += cl * h.dx;
                    acc[kGCentreLP + 1] += cl * h.dy;
                    acc[kGDepthLP] += zih;
                    W = 0.0f;
                }
                W = W - fmaf(uh, u, vh * v);
                acc[kGH + 0] = fmaf(uh, u, acc[kGH + 0]);
                acc[kGH + 1] = fmaf(uh, v, acc[kGH + 1]);
                acc[kGH + 2] += uh;
                acc[kGH + 3] = fmaf(vh, u, acc[kGH + 3]);
                acc[kGH + 4] = fmaf(vh, v, acc[kGH + 4]);
                acc[kGH + 5] += vh;
                acc[kGH + 6] = fmaf(W, u, acc[kGH + 6]);
                acc[kGH + 7] = fmaf(W, v, acc[kGH + 7]);
                acc[kGH + 8] += W;
            }
            // the chunk's sums of this lane's splat to the batch's shared accumulators
            if (active) {
                float *sg = s_g + slot * kRecGrad;
#pragma unroll
                for (int q = 0; q < kRecVals; ++q)
                    if (acc[q] != 0.0f) atomicAdd(sg + q, acc[q]);
                flush_cell<N>(ca, s_tg + slot * TEXF);
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nb * kRecGrad; e += NT) {
            const float v = s_g[e];
            if (v != 0.0f) {
                const int s = e / kRecGrad, q = e - s * kRecGrad;
                atomicAdd(b.rec_grad + int64_t(s_j[s]) * kRecGrad + q, v);
            }
        }
        if (g_tex)
            for (int e = threadIdx.x; e < nb * TEXF; e += NT) {
                const float v = s_tg[e];
                if (v != 0.0f) {
                    const int s = e / TEXF, o = e - s * TEXF;
                    atomicAdd(g_tex + int64_t(s_k[s]) * TEXF + o, v);
                }
            }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        npairs += __shfl_xor_sync(FULL, npairs, o);
    }
    if (lane == 0 && npairs) atomicAdd(&b.fw.cnt->pairs_bwd, (unsigned long long)npairs);
}

// Registers: two resident blocks of 256 threads per SM (up to 128 a thread).
template <int TS>
constexpr int sp_min_blocks() {
    return 512 / (TS * TS);
}

template <int TS, int N, typename TexT>
__global__ void __launch_bounds__(TS * TS, sp_min_blocks<TS>())
    render_bwd_sp_kernel(Frame f, RenderBwdBufs b, int batch, TileSched ts) {
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
        sp_tile<TS, N, TexT>(f, b, batch, tile);
    }
}

template <int TS, int N, typename TexT>
cudaError_t launch_t(const Frame &f, const RenderBwdBufs &b, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    constexpr int NT = TS * TS;
    const size_t smem = sp_stage_bytes<TS, N, TexT>(batch);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(render_bwd_sp_kernel<TS, N, TexT>,
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
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_bwd_sp_kernel<TS, N, TexT>, NT, smem);
            smem_seen = smem;
            if (per_sm < 1) per_sm = 1;
        }
        grid = std::min<unsigned>(grid, unsigned(per_sm * sms));
    } else {
        ts.work = nullptr;
    }
    if (grid == 0) return cudaSuccess;
    render_bwd_sp_kernel<TS, N, TexT><<<grid, NT, smem, s>>>(f, b, batch, ts);
    count_launches(1);
    return cudaGetLastError();
}

template <int TS, typename TexT>
cudaError_t launch_n(const Frame &f, const RenderBwdBufs &b, int N, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    switch (N) {
        case 1: return launch_t<TS, 1, TexT>(f, b, batch, ts, persistent, s);
        case 2: return launch_t<TS, 2, TexT>(f, b, batch, ts, persistent, s);
        case 4: return launch_t<TS, 4, TexT>(f, b, batch, ts, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int TS>
cudaError_t launch_d(const Frame &f, const RenderBwdBufs &b, int g, int N, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    switch (f.group_dtype[g]) {
        case GB_F16: return launch_n<TS, __half>(f, b, N, batch, ts, persistent, s);
        case GB_BF16: return launch_n<TS, __nv_bfloat16>(f, b, N, batch, ts, persistent, s);
        default: return launch_n<TS, float>(f, b, N, batch, ts, persistent, s);
    }
}

}  // namespace bwdsp

bool render_bwd_sp_supported(int tile, int N) { return (tile == 8 || tile == 16) && N <= 4; }

size_t render_bwd_sp_smem(int tile, int N, int dtype, int batch) {
    auto pick = [&](auto texT) -> size_t {
        using T = decltype(texT);
        switch (N) {
            case 1: return tile == 8 ? bwdsp::sp_stage_bytes<8, 1, T>(batch) : bwdsp::sp_stage_bytes<16, 1, T>(batch);
            case 2: return tile == 8 ? bwdsp::sp_stage_bytes<8, 2, T>(batch) : bwdsp::sp_stage_bytes<16, 2, T>(batch);
            default: return tile == 8 ? bwdsp::sp_stage_bytes<8, 4, T>(batch) : bwdsp::sp_stage_bytes<16, 4, T>(batch);
        }
    };
    if (dtype == GB_F16) return pick(__half());
    if (dtype == GB_BF16) return pick(__nv_bfloat16());
    return pick(float());
}

// Launches the splat-parallel backward render of every render group (each
// group must satisfy render_bwd_sp_supported).
cudaError_t launch_render_bwd_sp(const Frame &f, const RenderBwdBufs &b, int batch, const uint32_t *tile_list,
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
            case 8: e = bwdsp::launch_d<8>(f, b, g, N, batch, ts, persistent, s); break;
            case 16: e = bwdsp::launch_d<16>(f, b, g, N, batch, ts, persistent, s); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbill
