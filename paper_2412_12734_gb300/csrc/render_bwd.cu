// Backward per-tile render (Alg. 1 bwd with Alg. 2 adj-bilinear).
//
// One block per tile, one thread per pixel, batches walked back to front
// from the last blended splat of the tile.  Each pixel recomputes alpha and
// the colour of every splat it blended and its transmittance
// T_i = T_{i+1} / (1 - alpha_i) from the saved final T, then forms:
//   colour adjoint  c^ = alpha T dL/dC                       (-> SH colour, grid)
//   (C^, u^, v^)    = adj-bilinear(u, v, C_k, c^)            (Alg. 2)
//   alpha^          = dL/dC . (c T - S / (1 - alpha)) + depth and alpha terms
//   Gaussian:  rho^ -> (u^, v^) on the uv branch, -> centre on the low-pass one
//   intersection:   (u^, v^) -> zeta^ -> record (adj(T'), centre) gradients
// Record gradients (14 floats) are reduced over the warp, summed per batch in
// shared memory and added to global memory with one atomic per value per tile;
// colour-grid gradients are summed per batch in shared memory and added to the
// global texel gradient with one atomic per non-zero texel channel per tile.
#include <algorithm>

#include "render_common.cuh"

namespace gbill {
namespace {

// Reduce-scatter of 16 values over the warp (16 shuffles): lane l ends with the
// warp total of value index 8 b4 + 4 b3 + 2 b2 + b1 (b_i = bit i of l); lanes
// l and l^1 hold the same total.
__device__ __forceinline__ float warp_reduce_scatter16(float v[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 8], keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 4], keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 2], keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const bool up = lane & 2;
    const float send = up ? v[0] : v[1], keep = up ? v[1] : v[0];
    const float t = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

// Reduce-scatter of 32 values over the warp (31 shuffles): lane l ends with
// the warp total of value index l (bits of l select the kept half at each
// exchange step, most significant first).
__device__ __forceinline__ float warp_reduce_scatter32(float v[32], int lane) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 16], keep = up ? v[i + 16] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 8], keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 4], keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 2;
        const float send = up ? v[i] : v[i + 2], keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    const bool up = lane & 1;
    const float send = up ? v[0] : v[1], keep = up ? v[1] : v[0];
    return keep + __shfl_xor_sync(0xffffffffu, send, 1);
}

// Warp-reduced values: 0..13 record gradients, 14..25 the RGB gradient of the
// grid's four corner texels (0,0), (0,N-1), (N-1,0), (N-1,N-1).
constexpr int kCornerSlot = 14;
// For N = 8, above this many distinct edge/interior cells in a (warp, splat)
// pair the lanes add their texel weights to shared memory directly instead of
// one reduce-scatter per cell (measured: faster at N = 8, slower at N <= 4).
constexpr int kGroupCells8 = 4;

template <int TS, int N, typename TexT>
__device__ __forceinline__ void bwd_tile(const Frame &f, const RenderBwdBufs &b, int batch, uint32_t tile) {
    constexpr int NT = TS * TS;
    constexpr int NN = N * N;
    constexpr int TEXF = NN * 3;
    extern __shared__ float4 smem[];
    float4 *s_rec = smem;
    float4 *s_tex = s_rec + 4 * batch;
    int32_t *s_k = reinterpret_cast<int32_t *>(s_tex + batch * NN);
    uint32_t *s_j = reinterpret_cast<uint32_t *>(s_k + batch);
    uint2 *s_box = reinterpret_cast<uint2 *>(s_j + batch);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_box + batch);
    float *s_g = reinterpret_cast<float *>(s_mask + batch);  // [batch][16]
    float *s_tg = s_g + batch * kRecGrad;                  // [batch][TEXF]
    __shared__ uint32_t s_maxlast;

    const int ci = camera_of_tile(f, tile);
    const CamDev &cam = f.cams[ci];
    const SceneDev &sc = f.scenes[cam.scene];
    const uint32_t lt = tile - cam.tile_off;
    const int tx = int(lt % uint32_t(cam.tiles_x)), ty = int(lt / uint32_t(cam.tiles_x));
    int lx, ly;
    tile_pixel<TS>(threadIdx.x, lx, ly);
    const int lane = threadIdx.x & 31;
    const int px = tx * TS + lx, py = ty * TS + ly;
    const bool inside = px < cam.width && py < cam.height;
    const float xf = float(px) + 0.5f, yf = float(py) + 0.5f;
    const uint2 range = b.fw.ranges[tile];
    const float sigma = sc.sigma;
    const float kN = float(N - 1) / (2.0f * sigma);
    const uint32_t wbit = 1u << (threadIdx.x >> 5);  // this warp's 8 x 4 block in the splat masks

    float T = 1.0f, T_final = 1.0f, dC0 = 0, dC1 = 0, dC2 = 0, dD = 0, dA = 0;
    uint32_t last = 0, npairs = 0, ncontrib = 0;
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (inside) {
        const int64_t pix = cam.pix_off + int64_t(py) * cam.width + px;
        T = T_final = b.fw.t_final[pix];
        last = b.fw.last[pix];
        dC0 = b.d_rgb[3 * pix + 0];
        dC1 = b.d_rgb[3 * pix + 1];
        dC2 = b.d_rgb[3 * pix + 2];
        if (b.d_depth) dD = b.d_depth[pix];
        if (b.d_alpha) dA = b.d_alpha[pix];
    }
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0 && wlast) atomicMax(&s_maxlast, wlast);
    const float bgdot = dC0 * f.bg[0] + dC1 * f.bg[1] + dC2 * f.bg[2];
    const float dTfin = (dA - bgdot) * T_final;  // times 1/(1-alpha) per splat
    float S0 = 0, S1 = 0, S2 = 0, SD = 0;
    __syncthreads();
    const int max_last = int(s_maxlast);
    float *g_tex = sc.g_tex;
    const int my_q16 = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    // flat index (i_u N + i_v) of the corner texel this lane's reduced value feeds
    const int my_corner = lane >= kCornerSlot && lane < kCornerSlot + 12 ? (lane - kCornerSlot) / 3 : -1;
    const int my_corner_off = my_corner < 0 ? 0
                              : 3 * ((my_corner & 2 ? (N - 1) * N : 0) + (my_corner & 1 ? N - 1 : 0)) +
                                    (lane - kCornerSlot) % 3;

    for (int be = max_last; be > 0; be -= batch) {
        const int bs = max(0, be - batch), nb = be - bs;
        for (int e = threadIdx.x; e < nb * kRecGrad; e += NT) s_g[e] = 0.0f;
        for (int e = threadIdx.x; e < nb * TEXF; e += NT) s_tg[e] = 0.0f;
        stage_batch<N, NT, TexT, TS, 4>(b.fw, cam, sc, range.x + bs, nb, tx * TS, ty * TS, s_rec, s_tex, s_k, s_j,
                                        s_box, s_mask);
        __syncthreads();
        // splats at or beyond the warp's last contributor are skipped warp-wide
        const int i_hi = min(nb, int(wlast) - bs);
        for (int i = i_hi - 1; i >= 0; --i) {
            if (!(s_mask[i] & wbit)) continue;
            float g[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) g[q] = 0.0f;
            bool act = inside && uint32_t(bs + i) < last;
            npairs += act ? 1u : 0u;
            // texel weights not reduced through the corner slots, and their cell
            float rw00 = 0.0f, rw10 = 0.0f, rw01 = 0.0f, rw11 = 0.0f, rch0 = 0.0f, rch1 = 0.0f, rch2 = 0.0f;
            int rbase = 0;
            if (act) {
                const float4 q0 = s_rec[4 * i + 0], q1 = s_rec[4 * i + 1], q2 = s_rec[4 * i + 2],
                             q3 = s_rec[4 * i + 3];
                const float dx = (xf - q2.x) - q2.z, dy = (yf - q2.y) - q2.w;
                const float zz = fmaf(q1.x, dx, fmaf(q1.y, dy, q1.z));
                act = zz != 0.0f;
                if (act) {
                    const float rz = fast_rcp(zz);
                    const float u = fmaf(q0.x, dx, q0.y * dy) * rz;
                    const float v = fmaf(q0.z, dx, q0.w * dy) * rz;
                    const float ruv = fmaf(u, u, v * v);
                    const float rlp = kLowPass * fmaf(dx, dx, dy * dy);
                    const bool uvb = ruv <= rlp;
                    const float rho = uvb ? ruv : rlp;
                    const float G = gauss(rho);
                    const float ar = q3.x * G;
                    const bool clamped = ar > kAlphaMax;
                    const float alpha = clamped ? kAlphaMax : ar;
                    act = alpha >= kAlphaMin;
                    if (act) {
                        ++ncontrib;
                        const float iom = fast_rcp(1.0f - alpha);
                        const float Ti = T * iom;
                        const Cell<N> cell = grid_cell<N>(u, v, sigma, kN);
                        const Quad qd = grid_quad<N>(s_tex + i * NN, cell);
                        float col[3];
                        grid_colour<N>(qd, cell, col);
                        col[0] += q3.y;
                        col[1] += q3.z;
                        col[2] += q3.w;
                        const float w = alpha * Ti;
                        const float ch0 = w * dC0, ch1 = w * dC1, ch2 = w * dC2;
                        g[11] = ch0; g[12] = ch1; g[13] = ch2;
                        // adj-bilinear: grid adjoint and uv adjoint
                        float uh = 0.0f, vh = 0.0f;
                        if (N == 1) {
                            // the single texel is corner 0: reduced over the warp
                            g[kCornerSlot + 0] = ch0;
                            g[kCornerSlot + 1] = ch1;
                            g[kCornerSlot + 2] = ch2;
                        } else {
                            const float fu = cell.fu, fv = cell.fv;
                            const float w00 = (1.0f - fu) * (1.0f - fv), w10 = fu * (1.0f - fv);
                            const float w01 = (1.0f - fu) * fv, w11 = fu * fv;
                            // d colour / d f_u and d f_v, dotted with the colour adjoint
                            const float fuh = ch0 * ((qd.c10.x - qd.c00.x) * (1.0f - fv) + (qd.c11.x - qd.c01.x) * fv) +
                                              ch1 * ((qd.c10.y - qd.c00.y) * (1.0f - fv) + (qd.c11.y - qd.c01.y) * fv) +
                                              ch2 * ((qd.c10.z - qd.c00.z) * (1.0f - fv) + (qd.c11.z - qd.c01.z) * fv);
                            const float fvh = ch0 * ((qd.c01.x - qd.c00.x) * (1.0f - fu) + (qd.c11.x - qd.c10.x) * fu) +
                                              ch1 * ((qd.c01.y - qd.c00.y) * (1.0f - fu) + (qd.c11.y - qd.c10.y) * fu) +
                                              ch2 * ((qd.c01.z - qd.c00.z) * (1.0f - fu) + (qd.c11.z - qd.c10.z) * fu);
                            // weights landing on a grid-corner texel go to the warp-reduced corner
                            // slots; the rest (edge and interior texels) to the cell-group pass below
                            const int iu = cell.base / N, iv = cell.base - iu * N;
                            const float wc0 = (iu == 0 && iv == 0) ? w00 : 0.0f;
                            const float wc1 = (iu == 0 && iv == N - 2) ? w01 : 0.0f;
                            const float wc2 = (iu == N - 2 && iv == 0) ? w10 : 0.0f;
                            const float wc3 = (iu == N - 2 && iv == N - 2) ? w11 : 0.0f;
                            g[kCornerSlot + 0] = wc0 * ch0; g[kCornerSlot + 1] = wc0 * ch1; g[kCornerSlot + 2] = wc0 * ch2;
                            g[kCornerSlot + 3] = wc1 * ch0; g[kCornerSlot + 4] = wc1 * ch1; g[kCornerSlot + 5] = wc1 * ch2;
                            g[kCornerSlot + 6] = wc2 * ch0; g[kCornerSlot + 7] = wc2 * ch1; g[kCornerSlot + 8] = wc2 * ch2;
                            g[kCornerSlot + 9] = wc3 * ch0; g[kCornerSlot + 10] = wc3 * ch1; g[kCornerSlot + 11] = wc3 * ch2;
                            rw00 = w00 - wc0;
                            rw10 = w10 - wc2;
                            rw01 = w01 - wc1;
                            rw11 = w11 - wc3;
                            rbase = cell.base;
                            rch0 = ch0; rch1 = ch1; rch2 = ch2;
                            if (u > -sigma && u < sigma) uh = kN * fuh;
                            if (v > -sigma && v < sigma) vh = kN * fvh;
                        }
                        // alpha adjoint
                        const float zi = uvb ? q1.z * q1.w * rz : q1.w;
                        float ah = dC0 * (col[0] * Ti - S0 * iom) + dC1 * (col[1] * Ti - S1 * iom) +
                                   dC2 * (col[2] * Ti - S2 * iom);
                        ah += dD * (zi * Ti - SD * iom) + dTfin * iom;
                        S0 = fmaf(col[0], w, S0);
                        S1 = fmaf(col[1], w, S1);
                        S2 = fmaf(col[2], w, S2);
                        SD = fmaf(zi, w, SD);
                        T = Ti;
                        const float zih = dD * w;
                        float rhoh = 0.0f;
                        if (!clamped) {
                            g[10] = ah * G;
                            rhoh = -0.5f * alpha * ah;
                        }
                        float zzh = 0.0f, dxh = 0.0f, dyh = 0.0f;
                        if (uvb) {
                            uh = fmaf(2.0f * u, rhoh, uh);
                            vh = fmaf(2.0f * v, rhoh, vh);
                            // zi = m22 z / zeta_z
                            g[6] += zih * q1.w * rz;
                            g[7] += zih * q1.z * rz;
                            zzh = -zih * zi * rz;
                        } else {
                            dxh = 2.0f * kLowPass * dx * rhoh;
                            dyh = 2.0f * kLowPass * dy * rhoh;
                            g[7] += zih;
                        }
                        const float zxh = uh * rz, zyh = vh * rz;
                        zzh -= (uh * u + vh * v) * rz;
                        g[0] = zxh * dx;
                        g[1] = zxh * dy;
                        g[2] = zyh * dx;
                        g[3] = zyh * dy;
                        g[4] = zzh * dx;
                        g[5] = zzh * dy;
                        g[6] += zzh;
                        dxh += zxh * q0.x + zyh * q0.z + zzh * q1.x;
                        dyh += zxh * q0.y + zyh * q0.w + zzh * q1.y;
                        g[8] = -dxh;
                        g[9] = -dyh;
                    }
                }
            }
            if (__any_sync(0xffffffffu, act)) {
                const float tot = warp_reduce_scatter32(g, lane);
                if (tot != 0.0f) {
                    if (lane < kCornerSlot) atomicAdd(s_g + i * kRecGrad + lane, tot);
                    else if (my_corner >= 0) atomicAdd(s_tg + i * TEXF + my_corner_off, tot);
                }
                // edge / interior texels: lanes sharing a cell are reduced together
                // (one reduce-scatter and one conflict-free atomic per cell); at
                // N = 8, when many distinct cells are hit, each lane adds its
                // weights to shared memory directly instead.
                if (N > 2) {
                    const bool has_rem = (rw00 != 0.0f) | (rw10 != 0.0f) | (rw01 != 0.0f) | (rw11 != 0.0f);
                    unsigned pending = __ballot_sync(0xffffffffu, has_rem);
                    int cells = 0;
                    if (N >= 8 && pending) {
                        const unsigned same = __match_any_sync(0xffffffffu, has_rem ? rbase : -1);
                        cells = __popc(__ballot_sync(0xffffffffu, has_rem && (__ffs(same) - 1) == lane));
                    }
                    if (cells > kGroupCells8) {
                        if (has_rem) {
                            float *t = s_tg + i * TEXF + 3 * rbase;
                            if (rw00 != 0.0f) {
                                atomicAdd(t + 0, rw00 * rch0); atomicAdd(t + 1, rw00 * rch1); atomicAdd(t + 2, rw00 * rch2);
                            }
                            if (rw10 != 0.0f) {
                                atomicAdd(t + 3 * N + 0, rw10 * rch0); atomicAdd(t + 3 * N + 1, rw10 * rch1);
                                atomicAdd(t + 3 * N + 2, rw10 * rch2);
                            }
                            if (rw01 != 0.0f) {
                                atomicAdd(t + 3, rw01 * rch0); atomicAdd(t + 4, rw01 * rch1); atomicAdd(t + 5, rw01 * rch2);
                            }
                            if (rw11 != 0.0f) {
                                atomicAdd(t + 3 * N + 3, rw11 * rch0); atomicAdd(t + 3 * N + 4, rw11 * rch1);
                                atomicAdd(t + 3 * N + 5, rw11 * rch2);
                            }
                        }
                        pending = 0u;
                    }
                    while (pending) {
                        const int leader = __ffs(pending) - 1;
                        const int key = __shfl_sync(0xffffffffu, rbase, leader);
                        const bool mine = ((pending >> lane) & 1u) && rbase == key;
                        pending &= ~__ballot_sync(0xffffffffu, mine);
                        float h[16];
                        h[0] = mine ? rw00 * rch0 : 0.0f; h[1] = mine ? rw00 * rch1 : 0.0f; h[2] = mine ? rw00 * rch2 : 0.0f;
                        h[3] = mine ? rw10 * rch0 : 0.0f; h[4] = mine ? rw10 * rch1 : 0.0f; h[5] = mine ? rw10 * rch2 : 0.0f;
                        h[6] = mine ? rw01 * rch0 : 0.0f; h[7] = mine ? rw01 * rch1 : 0.0f; h[8] = mine ? rw01 * rch2 : 0.0f;
                        h[9] = mine ? rw11 * rch0 : 0.0f; h[10] = mine ? rw11 * rch1 : 0.0f; h[11] = mine ? rw11 * rch2 : 0.0f;
                        h[12] = h[13] = h[14] = h[15] = 0.0f;
                        const float t = warp_reduce_scatter16(h, lane);
                        if (!(lane & 1) && my_q16 < 12 && t != 0.0f) {
                            const int k = my_q16 / 3, c = my_q16 - 3 * k;
                            // k: 0 -> (iu, iv), 1 -> (iu+1, iv), 2 -> (iu, iv+1), 3 -> (iu+1, iv+1)
                            const int off = 3 * (key + ((k & 1) ? N : 0) + ((k & 2) ? 1 : 0)) + c;
                            atomicAdd(s_tg + i * TEXF + off, t);
                        }
                    }
                }
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
        npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        ncontrib += __shfl_xor_sync(0xffffffffu, ncontrib, o);
    }
    if (lane == 0 && npairs) atomicAdd(&b.fw.cnt->pairs_bwd, (unsigned long long)npairs);
    if (lane == 0 && ncontrib) atomicAdd(&b.fw.cnt->contrib_bwd, (unsigned long long)ncontrib);
}

template <int TS, int N, typename TexT>
__global__ void __launch_bounds__(TS * TS, 1024 / (TS * TS)) render_bwd_kernel(Frame f, RenderBwdBufs b, int batch, TileSched ts) {
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
        bwd_tile<TS, N, TexT>(f, b, batch, tile);
    }
}

template <int TS, int N, typename TexT>
cudaError_t launch_t(const Frame &f, const RenderBwdBufs &b, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    const size_t smem = stage_bytes<N>(batch, true);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(render_bwd_kernel<TS, N, TexT>,
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
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_bwd_kernel<TS, N, TexT>, TS * TS, smem);
            smem_seen = smem;
            if (per_sm < 1) per_sm = 1;
        }
        grid = std::min<unsigned>(grid, unsigned(per_sm * sms));
    } else {
        ts.work = nullptr;
    }
    if (grid == 0) return cudaSuccess;
    render_bwd_kernel<TS, N, TexT><<<grid, TS * TS, smem, s>>>(f, b, batch, ts);
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
        case 8: return launch_t<TS, 8, TexT>(f, b, batch, ts, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_render_bwd(const Frame &f, const RenderBwdBufs &b, int batch, const uint32_t *tile_list,
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
        if (f.tile == 8) {
            switch (f.group_dtype[g]) {
                case GB_F16: e = launch_n<8, __half>(f, b, N, batch, ts, persistent, s); break;
                case GB_BF16: e = launch_n<8, __nv_bfloat16>(f, b, N, batch, ts, persistent, s); break;
                default: e = launch_n<8, float>(f, b, N, batch, ts, persistent, s); break;
            }
        } else if (f.tile == 16) {
            switch (f.group_dtype[g]) {
                case GB_F16: e = launch_n<16, __half>(f, b, N, batch, ts, persistent, s); break;
                case GB_BF16: e = launch_n<16, __nv_bfloat16>(f, b, N, batch, ts, persistent, s); break;
                default: e = launch_n<16, float>(f, b, N, batch, ts, persistent, s); break;
            }
        } else {
            return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbill
