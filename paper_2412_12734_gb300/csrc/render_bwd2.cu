// Backward per-tile render, two pixels per thread (Alg. 1 bwd with Alg. 2
// adj-bilinear; same mathematics as render_bwd.cu).
//
// A warp covers an 8 x 8 pixel block: lane l owns pixels (x, y) and (x, y + 4)
// of the same column, so the horizontal offset to a splat's centre is shared
// and the per-pixel arithmetic runs on Blackwell's packed FP32x2 pipe
// (__ffma2_rn / __fmul2_rn / __fadd2_rn).  Record loads, the warp
// reduce-scatter of the 14 record gradients and the loop overhead are paid
// once per 64 pixels; a 16 x 16 tile is 4 warps, so fewer warps wait at each
// batch barrier.  Every per-pixel quantity of an inactive pixel is forced to
// zero before it can reach a gradient.
#include <algorithm>

#include "render_common.cuh"

namespace gbill {
namespace {

__device__ __forceinline__ float2 bc(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sel2(bool a, bool b, float2 x, float2 y) {
    return make_float2(a ? x.x : y.x, b ? x.y : y.y);
}

__device__ __forceinline__ float warp_reduce_scatter16b(float v[16], int lane) {
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
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1], keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Grid colour, texel-gradient atomics and the colour part of the uv adjoint
// of one pixel (Alg. 2 bilinear / adj-bilinear).
template <int N>
__device__ __forceinline__ void pixel_grid(const float4 *tex, float *tgo, float u, float v, float sigma, float kN,
                                           bool act, float ch0, float ch1, float ch2, float col[3], float &uh,
                                           float &vh) {
    const Cell<N> cell = grid_cell<N>(u, v, sigma, kN);
    uh = vh = 0.0f;
    if (!act) {
        col[0] = col[1] = col[2] = 0.0f;
        return;
    }
    const Quad qd = grid_quad<N>(tex, cell);
    grid_colour<N>(qd, cell, col);
    if (N == 1) {
        atomicAdd(tgo + 0, ch0);
        atomicAdd(tgo + 1, ch1);
        atomicAdd(tgo + 2, ch2);
        return;
    }
    const float fu = cell.fu, fv = cell.fv;
    const float w00 = (1.0f - fu) * (1.0f - fv), w10 = fu * (1.0f - fv);
    const float w01 = (1.0f - fu) * fv, w11 = fu * fv;
    const int o00 = 3 * cell.base, o10 = o00 + 3 * N, o01 = o00 + 3, o11 = o10 + 3;
    if (w00 != 0.0f) {
        atomicAdd(tgo + o00 + 0, ch0 * w00);
        atomicAdd(tgo + o00 + 1, ch1 * w00);
        atomicAdd(tgo + o00 + 2, ch2 * w00);
    }
    if (w10 != 0.0f) {
        atomicAdd(tgo + o10 + 0, ch0 * w10);
        atomicAdd(tgo + o10 + 1, ch1 * w10);
        atomicAdd(tgo + o10 + 2, ch2 * w10);
    }
    if (w01 != 0.0f) {
        atomicAdd(tgo + o01 + 0, ch0 * w01);
        atomicAdd(tgo + o01 + 1, ch1 * w01);
        atomicAdd(tgo + o01 + 2, ch2 * w01);
    }
    if (w11 != 0.0f) {
        atomicAdd(tgo + o11 + 0, ch0 * w11);
        atomicAdd(tgo + o11 + 1, ch1 * w11);
        atomicAdd(tgo + o11 + 2, ch2 * w11);
    }
    if (u > -sigma && u < sigma)
        uh = kN * (ch0 * ((qd.c10.x - qd.c00.x) * (1.0f - fv) + (qd.c11.x - qd.c01.x) * fv) +
                   ch1 * ((qd.c10.y - qd.c00.y) * (1.0f - fv) + (qd.c11.y - qd.c01.y) * fv) +
                   ch2 * ((qd.c10.z - qd.c00.z) * (1.0f - fv) + (qd.c11.z - qd.c01.z) * fv));
    if (v > -sigma && v < sigma)
        vh = kN * (ch0 * ((qd.c01.x - qd.c00.x) * (1.0f - fu) + (qd.c11.x - qd.c10.x) * fu) +
                   ch1 * ((qd.c01.y - qd.c00.y) * (1.0f - fu) + (qd.c11.y - qd.c10.y) * fu) +
                   ch2 * ((qd.c01.z - qd.c00.z) * (1.0f - fu) + (qd.c11.z - qd.c10.z) * fu));
}

template <int TS, int N, typename TexT>
__device__ __forceinline__ void bwd2_tile(const Frame &f, const RenderBwdBufs &b, int batch, uint32_t tile) {
    constexpr int NT = TS * TS / 2;
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
    float *s_tg = s_g + batch * kRecGrad;                    // [batch][TEXF]
    __shared__ uint32_t s_maxlast;

    const int ci = camera_of_tile(f, tile);
    const CamDev &cam = f.cams[ci];
    const SceneDev &sc = f.scenes[cam.scene];
    const uint32_t lt = tile - cam.tile_off;
    const int tx = int(lt % uint32_t(cam.tiles_x)), ty = int(lt / uint32_t(cam.tiles_x));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = (warp % (TS / 8)) * 8, by = (warp / (TS / 8)) * 8;
    const int px = tx * TS + bx + (lane & 7);
    const int py0 = ty * TS + by + (lane >> 3), py1 = py0 + 4;
    const bool in0 = px < cam.width && py0 < cam.height, in1 = px < cam.width && py1 < cam.height;
    const float xf = float(px) + 0.5f;
    const float2 yf = make_float2(float(py0) + 0.5f, float(py1) + 0.5f);
    const uint2 range = b.fw.ranges[tile];
    const float sigma = sc.sigma;
    const float kN = float(N - 1) / (2.0f * sigma);
    const uint32_t wbit = 1u << warp;  // this warp's 8 x 8 block in the splat masks

    float2 T = bc(1.0f), Tfin = bc(1.0f), dR = bc(0.0f), dG = bc(0.0f), dB = bc(0.0f), dDp = bc(0.0f), dA = bc(0.0f);
    uint32_t last0 = 0, last1 = 0, npairs = 0;
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    const int64_t pix0 = cam.pix_off + int64_t(py0) * cam.width + px;
    const int64_t pix1 = cam.pix_off + int64_t(py1) * cam.width + px;
    if (in0) {
        T.x = Tfin.x = b.fw.t_final[pix0];
        last0 = b.fw.last[pix0];
        dR.x = b.d_rgb[3 * pix0 + 0];
        dG.x = b.d_rgb[3 * pix0 + 1];
        dB.x = b.d_rgb[3 * pix0 + 2];
        if (b.d_depth) dDp.x = b.d_depth[pix0];
        if (b.d_alpha) dA.x = b.d_alpha[pix0];
    }
    if (in1) {
        T.y = Tfin.y = b.fw.t_final[pix1];
        last1 = b.fw.last[pix1];
        dR.y = b.d_rgb[3 * pix1 + 0];
        dG.y = b.d_rgb[3 * pix1 + 1];
        dB.y = b.d_rgb[3 * pix1 + 2];
        if (b.d_depth) dDp.y = b.d_depth[pix1];
        if (b.d_alpha) dA.y = b.d_alpha[pix1];
    }
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, max(last0, last1));
    if (lane == 0 && wlast) atomicMax(&s_maxlast, wlast);
    // (dL/dalpha - dL/drgb . bg) T_final, divided by (1 - alpha) per splat
    const float2 bgdot = fma2(dR, bc(f.bg[0]), fma2(dG, bc(f.bg[1]), mul2(dB, bc(f.bg[2]))));
    const float2 dTfin = mul2(sub2(dA, bgdot), Tfin);
    float2 SR = bc(0.0f), SG = bc(0.0f), SB = bc(0.0f), SD = bc(0.0f);
    __syncthreads();
    const int max_last = int(s_maxlast);
    float *g_tex = sc.g_tex;
    const int my_q = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);

    for (int be = max_last; be > 0; be -= batch) {
        const int bs = max(0, be - batch), nb = be - bs;
        for (int e = threadIdx.x; e < nb * kRecGrad; e += NT) s_g[e] = 0.0f;
        for (int e = threadIdx.x; e < nb * TEXF; e += NT) s_tg[e] = 0.0f;
        stage_batch<N, NT, TexT, TS, 8>(b.fw, cam, sc, range.x + bs, nb, tx * TS, ty * TS, s_rec, s_tex, s_k, s_j,
                                        s_box, s_mask);
        __syncthreads();
        const int i_hi = min(nb, int(wlast) - bs);
        for (int i = i_hi - 1; i >= 0; --i) {
            if (!(s_mask[i] & wbit)) continue;
            const uint32_t idx = uint32_t(bs + i);
            bool a0 = in0 && idx < last0, a1 = in1 && idx < last1;
            if (!__any_sync(0xffffffffu, a0 || a1)) continue;
            const float4 q0 = s_rec[4 * i + 0], q1 = s_rec[4 * i + 1], q2 = s_rec[4 * i + 2], q3 = s_rec[4 * i + 3];
            const float dx = (xf - q2.x) - q2.z;
            const float2 dy = sub2(sub2(yf, bc(q2.y)), bc(q2.w));
            const float2 zz = fma2(bc(q1.y), dy, bc(fmaf(q1.x, dx, q1.z)));
            a0 = a0 && zz.x != 0.0f;
            a1 = a1 && zz.y != 0.0f;
            float2 rz = make_float2(fast_rcp(zz.x), fast_rcp(zz.y));
            float2 u = mul2(fma2(bc(q0.y), dy, bc(q0.x * dx)), rz);
            float2 v = mul2(fma2(bc(q0.w), dy, bc(q0.z * dx)), rz);
            const float2 ruv = fma2(u, u, mul2(v, v));
            const float2 rlp = mul2(bc(kLowPass), fma2(dy, dy, bc(dx * dx)));
            const bool uvb0 = ruv.x <= rlp.x, uvb1 = ruv.y <= rlp.y;
            const float2 rho = sel2(uvb0, uvb1, ruv, rlp);
            const float2 G = make_float2(gauss(rho.x), gauss(rho.y));
            const float2 ar = mul2(bc(q3.x), G);
            const bool cl0 = ar.x > kAlphaMax, cl1 = ar.y > kAlphaMax;
            const float2 alpha = make_float2(fminf(ar.x, kAlphaMax), fminf(ar.y, kAlphaMax));
            a0 = a0 && alpha.x >= kAlphaMin;
            a1 = a1 && alpha.y >= kAlphaMin;
            if (!__any_sync(0xffffffffu, a0 || a1)) continue;
            npairs += uint32_t(a0) + uint32_t(a1);
            // from here on every quantity of an inactive pixel is zero
            rz = sel2(a0, a1, rz, bc(0.0f));
            u = sel2(a0, a1, u, bc(0.0f));
            v = sel2(a0, a1, v, bc(0.0f));
            const float2 iom = make_float2(fast_rcp(1.0f - alpha.x), fast_rcp(1.0f - alpha.y));
            const float2 Ti = mul2(T, iom);
            const float2 w = sel2(a0, a1, mul2(alpha, Ti), bc(0.0f));
            const float2 chR = mul2(w, dR), chG = mul2(w, dG), chB = mul2(w, dB);
            float col0[3], col1[3], uhc0, vhc0, uhc1, vhc1;
            float *tgo = s_tg + i * TEXF;
            pixel_grid<N>(s_tex + i * NN, tgo, u.x, v.x, sigma, kN, a0, chR.x, chG.x, chB.x, col0, uhc0, vhc0);
            pixel_grid<N>(s_tex + i * NN, tgo, u.y, v.y, sigma, kN, a1, chR.y, chG.y, chB.y, col1, uhc1, vhc1);
            const float2 cR = add2(make_float2(col0[0], col1[0]), bc(q3.y));
            const float2 cG = add2(make_float2(col0[1], col1[1]), bc(q3.z));
            const float2 cB = add2(make_float2(col0[2], col1[2]), bc(q3.w));
            // alpha adjoint (zero for inactive pixels)
            const float2 zi = sel2(uvb0, uvb1, mul2(bc(q1.z * q1.w), rz), bc(q1.w));
            float2 ah = mul2(dR, sub2(mul2(cR, Ti), mul2(SR, iom)));
            ah = fma2(dG, sub2(mul2(cG, Ti), mul2(SG, iom)), ah);
            ah = fma2(dB, sub2(mul2(cB, Ti), mul2(SB, iom)), ah);
            ah = fma2(dDp, sub2(mul2(zi, Ti), mul2(SD, iom)), ah);
            ah = sel2(a0, a1, fma2(dTfin, iom, ah), bc(0.0f));
            SR = fma2(cR, w, SR);
            SG = fma2(cG, w, SG);
            SB = fma2(cB, w, SB);
            SD = fma2(zi, w, SD);
            T = sel2(a0, a1, Ti, T);
            const float2 zih = mul2(dDp, w);
            const float2 rhoh = sel2(cl0, cl1, bc(0.0f), mul2(bc(-0.5f), mul2(alpha, ah)));
            const float2 oh = sel2(cl0, cl1, bc(0.0f), mul2(ah, G));
            // Gaussian adjoint: uv branch -> (u, v); low-pass branch -> centre
            const float2 two_rhoh = mul2(bc(2.0f), rhoh);
            float2 uh = add2(make_float2(uhc0, uhc1), sel2(uvb0, uvb1, mul2(two_rhoh, u), bc(0.0f)));
            float2 vh = add2(make_float2(vhc0, vhc1), sel2(uvb0, uvb1, mul2(two_rhoh, v), bc(0.0f)));
            const float2 lp = sel2(uvb0, uvb1, bc(0.0f), mul2(bc(2.0f * kLowPass), rhoh));
            // depth: uv branch zi = m22 z / zeta_z, low-pass branch zi = z
            const float2 zuv = sel2(uvb0, uvb1, zih, bc(0.0f));
            const float2 zlp = sub2(zih, zuv);
            const float2 zxh = mul2(uh, rz), zyh = mul2(vh, rz);
            const float2 zzh = mul2(bc(-1.0f), mul2(fma2(uh, u, fma2(vh, v, mul2(zuv, zi))), rz));
            float g[16];
            const float szxh = zxh.x + zxh.y, szyh = zyh.x + zyh.y, szzh = zzh.x + zzh.y;
            g[0] = szxh * dx;
            g[1] = zxh.x * dy.x + zxh.y * dy.y;
            g[2] = szyh * dx;
            g[3] = zyh.x * dy.x + zyh.y * dy.y;
            g[4] = szzh * dx;
            g[5] = zzh.x * dy.x + zzh.y * dy.y;
            const float2 zr = mul2(zuv, rz);
            g[6] = szzh + q1.w * (zr.x + zr.y);
            g[7] = q1.z * (zr.x + zr.y) + zlp.x + zlp.y;
            // d/dc = -(d/d(dx), d/d(dy))
            const float dxh = szxh * q0.x + szyh * q0.z + szzh * q1.x + dx * (lp.x + lp.y);
            const float2 dyh2 = fma2(lp, dy, fma2(zxh, bc(q0.y), fma2(zyh, bc(q0.w), mul2(zzh, bc(q1.y)))));
            g[8] = -dxh;
            g[9] = -(dyh2.x + dyh2.y);
            g[10] = oh.x + oh.y;
            g[11] = chR.x + chR.y;
            g[12] = chG.x + chG.y;
            g[13] = chB.x + chB.y;
            g[14] = g[15] = 0.0f;
            const float tot = warp_reduce_scatter16b(g, lane);
            if (!(lane & 1) && my_q < 14 && tot != 0.0f) atomicAdd(s_g + i * kRecGrad + my_q, tot);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nb * kRecGrad; e += NT) {
            const float val = s_g[e];
            if (val != 0.0f) {
                const int s = e / kRecGrad, q = e - s * kRecGrad;
                atomicAdd(b.rec_grad + int64_t(s_j[s]) * kRecGrad + q, val);
            }
        }
        if (g_tex)
            for (int e = threadIdx.x; e < nb * TEXF; e += NT) {
                const float val = s_tg[e];
                if (val != 0.0f) {
                    const int s = e / TEXF, o = e - s * TEXF;
                    atomicAdd(g_tex + int64_t(s_k[s]) * TEXF + o, val);
                }
            }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if (lane == 0 && npairs) atomicAdd(&b.fw.cnt->contrib_bwd, (unsigned long long)npairs);
}

template <int TS, int N, typename TexT>
__global__ void __launch_bounds__(TS * TS / 2, 1280 / (TS * TS)) render_bwd2_kernel(Frame f, RenderBwdBufs b,
                                                                                  int batch, TileSched ts) {
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
        bwd2_tile<TS, N, TexT>(f, b, batch, tile);
    }
}

template <int TS, int N, typename TexT>
cudaError_t launch_t(const Frame &f, const RenderBwdBufs &b, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    const size_t smem = stage_bytes<N>(batch, true);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(render_bwd2_kernel<TS, N, TexT>,
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
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_bwd2_kernel<TS, N, TexT>, TS * TS / 2, smem);
            smem_seen = smem;
            if (per_sm < 1) per_sm = 1;
        }
        grid = std::min<unsigned>(grid, unsigned(per_sm * sms));
    } else {
        ts.work = nullptr;
    }
    if (grid == 0) return cudaSuccess;
    render_bwd2_kernel<TS, N, TexT><<<grid, TS * TS / 2, smem, s>>>(f, b, batch, ts);
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

cudaError_t launch_render_bwd2(const Frame &f, const RenderBwdBufs &b, int batch, const uint32_t *tile_list,
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
