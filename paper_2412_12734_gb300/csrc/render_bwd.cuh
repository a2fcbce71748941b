// Backward per-tile render (Alg. 1 bwd with Alg. 2 adj-bilinear), shared by
// the one- and two-pixels-per-thread instantiations (render_bwd.cu,
// render_bwd2.cu).
//
// One block per tile; thread t owns P pixels of its warp's 8 x 4P block
// (P = 1: rows y; P = 2: rows y and y + 4 of the same column).  Batches of
// the tile's splats are walked back to front from the last blended splat of
// the warp.  Each pixel recomputes alpha and the colour of every splat it
// blended and its transmittance T_i = T_{i+1} / (1 - alpha_i) from the saved
// final T, then forms:
//   colour adjoint  c^ = alpha T dL/dC                       (-> SH colour, grid)
//   (C^, u^, v^)    = adj-bilinear(u, v, C_k, c^)            (Alg. 2)
//   alpha^          = dL/dC . (c T - S / (1 - alpha)) + depth and alpha terms
//   Gaussian:  rho^ -> (u^, v^) on the uv branch, -> centre on the low-pass one
//   intersection:   (u^, v^) -> zeta^ -> record (adj(T'), centre) gradients
// Scatter: a thread first sums its P pixels' values; the 16 record gradients
// and 12 texel values go through one 32-value warp reduce-scatter: at N = 2 the
// four texels; at N = 4 the four grid corners or one grid border line when
// every texel the warp's pixels weight lies there (where the weight of a
// clamped u or v lands); at N >= 8 the four grid corners.  The other texel
// weights are added to global memory by each lane (N = 4 pairs that fit no
// window; pairs of larger grids that weight more than one cell) or reduced for
// the one grid cell they weight (a 16-value reduce-scatter); at N = 4 a pair
// with few contributing lanes skips the reduce-scatter altogether
// (kFewLanes4).  Every reduced value goes to global memory with one atomic per
// (warp, splat) pair: nothing accumulates in shared memory, which holds only
// the staged batch.  Measured on the 1M-splat, 16-view workload against
// per-batch shared accumulators flushed once per tile: 40.5 -> 37.8 ms at
// N = 4 (batch 88 -> 184 in the same 48 KB), 54.0 -> 41.0 ms at N = 8 (32 ->
// 64), 76.4 -> 54.1 ms at N = 16 (8 -> 16).
#pragma once

#include <algorithm>

#include "render_common.cuh"

namespace gbill {
namespace bwd {

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

// Warp-reduced values: 0..15 record gradients (kRecGrad layout), 16..27 the
// RGB gradient of the grid's four corner texels (0,0), (0,N-1), (N-1,0),
// (N-1,N-1).
constexpr int kCornerSlot = kRecVals;
static_assert(kCornerSlot + 12 <= 32, "record and corner-texel values share one 32-value reduce-scatter");
// For N >= 8 (and per-splat grid sizes), above this many distinct edge or
// interior cells in a (warp, splat) pair the lanes add their texel weights to
// global memory themselves instead of one 16-value reduce-scatter per cell;
// N = 4 pairs that fit no corner or line window always do.  Measured on the
// 16-view workload: N = 8 / 16 backward 36.0 / 44.2 ms at 0, 34.5 / 43.5 at
// 1, 35.6 / 44.3 at 2, 37.3 / 45.6 at 3; at N = 4 adding directly the lanes
// of the pairs without a window took 33.5 ms against 37.0 with the border
// line holding most of their pixels reduced through the window and a per-cell
// pass for the rest, and adding every texel weight directly (no window at all)
// 48.6 ms: the lanes of a window pair mostly weight the same few texels, whose
// atomics serialize.
constexpr int kDirectCells = 1;

// At N = 4 a (warp, splat) pair with at most this many contributing lanes
// skips the window and the reduce-scatter: each of those lanes adds its own
// record values (four 128-bit reductions) and texel weights (a 64-bit and a
// 32-bit reduction per texel) to global memory.  Measured on the 16-view
// workload (render_bwd at N = 4): 29.55 ms without; with scalar reductions
// 29.03 / 28.53 / 28.82 / 31.19 ms at 4 / 8 / 12 / 16 lanes; with the record
// values as 128-bit reductions 26.50 ms at 8, 25.42 / 25.49 / 26.14 / 67.3 ms
// at 16 / 20 / 24 / 32 lanes (every pair direct: the lanes' reductions to the
// same texels serialize), and 25.06 ms at 16 with the texels' 64-bit pairs.
// At N = 8 every threshold from 1 to 4 was slower (35.6-35.8 against 34.4 ms
// with scalar reductions).
constexpr int kFewLanes4 = 16;

// Adds w (c0, c1, c2) to the RGB texel at t: one 64-bit and one 32-bit
// reduction (t is 4-byte aligned; the pair goes where it is 8-byte aligned).
// Used where few lanes add texels (at N >= 8, in the direct texel pass of many
// lanes, three 32-bit reductions measured faster: 34.4 against 34.9 ms).
__device__ __forceinline__ void add_texel(float *t, float w, float c0, float c1, float c2) {
    if ((reinterpret_cast<uintptr_t>(t) & 7u) == 0) {
        atomicAdd(reinterpret_cast<float2 *>(t), make_float2(w * c0, w * c1));
        atomicAdd(t + 2, w * c2);
    } else {
        atomicAdd(t, w * c0);
        atomicAdd(reinterpret_cast<float2 *>(t + 1), make_float2(w * c1, w * c2));
    }
}

// State of one pixel in the reverse walk.
struct Pix {
    float xf, yf;                // pixel centre
    float T;                     // transmittance in front of the current splat's successor
    float dC0, dC1, dC2, dD;     // dL/drgb, dL/ddepth
    float dTfin;                 // (dL/dalpha - dL/drgb . bg) T_final
    float S0, S1, S2, SD;        // colour and depth blended behind the current splat
    uint32_t last;               // 1 + index of the last blended splat (0: none)
    bool inside;
};

// Texel weights of one pixel that the corner slots do not take (N = 4: the
// four of its cell, routed through a corner or border-line window of the
// reduce-scatter or added directly; N >= 8: those off the grid corners), with
// the colour adjoint they multiply and the cell they belong to.
struct Rem {
    float w00, w10, w01, w11, c0, c1, c2;
    int base;
    __device__ __forceinline__ bool any() const {
        return (w00 != 0.0f) | (w10 != 0.0f) | (w01 != 0.0f) | (w11 != 0.0f);
    }
};

// Adjoints of one (pixel, splat) pair: adds the record gradients and the
// corner-texel gradients to g[], sets the remaining texel weights and steps
// the pixel's reverse state.  Returns whether the pixel blended the splat.
template <bool ACC>
__device__ __forceinline__ void put(float &slot, float v) {
    if (ACC) slot += v; else slot = v;
}

// ACC: add to g[] (second and later pixels of a thread); otherwise the slots
// this pair owns are assigned (g[] holds zeros on entry).
// lo: the splat's RecordLo when its record is flagged for the extended-
// precision plane hit (the same splat for the whole warp), else null.
// VAR: the splat's grid is nk x nk (per-splat grid size; kN = (nk - 1) / (2
// sigma)) and every texel weight goes to the cell or direct texel pass.
template <int N, typename TexT, bool ACC, bool VAR = false>
__device__ __forceinline__ bool pair_adjoint(Pix &px, uint32_t idx, const float4 *rec, const RecordLo *lo,
                                             const staged_t<TexT> *tex, float sigma, float kN, int nk, float g[32],
                                             Rem &rem) {
    rem.w00 = rem.w10 = rem.w01 = rem.w11 = 0.0f;
    rem.c0 = rem.c1 = rem.c2 = 0.0f;
    rem.base = 0;
    // every lane evaluates (lanes past their last splat too, result dropped) so
    // that the only divergent region is the adjoint of the contributing lanes
    const bool live = px.inside && idx < px.last;
    const float4 q0 = rec[0], q1 = rec[1], q2 = rec[2], q3 = rec[3];
    const Hit h = lo ? plane_hit_ext(px.xf, px.yf, q0, q1, q2, *lo) : plane_hit(px.xf, px.yf, q0, q1, q2);
    const float dx = h.dx, dy = h.dy, zz = h.zz;
    const float rz = fast_rcp(zz);
    const float u = h.zx * rz;
    const float v = h.zy * rz;
    const float ruv = fmaf(u, u, v * v);
    const float rlp = kLowPass * fmaf(dx, dx, dy * dy);
    const bool uvb = ruv <= rlp;
    const float rho = uvb ? ruv : rlp;
    const float G = gauss(rho);
    const float ar = q3.x * G;
    const bool clamped = ar > kAlphaMax;
    const float alpha = clamped ? kAlphaMax : ar;
    if (!(live && zz != 0.0f && alpha >= kAlphaMin)) return false;
    const float iom = fast_rcp(1.0f - alpha);
    const float Ti = px.T * iom;
    const Cell<N> cell = VAR ? grid_cell_n<N>(u, v, sigma, kN, nk) : grid_cell<N>(u, v, sigma, kN);
    const Quad qd = grid_quad<N, TexT>(tex, cell);
    // bilinear colour (the forward's lerp order) and its derivatives in f_u
    // and f_v from the same differences: d col / d f_v = b - a, d col / d f_u
    // = d10 + f_v (d11 - d10)
    float col[3], dcu[3], dcv[3];
    if (N == 1) {
        grid_colour<N>(qd, cell, col);
    } else {
        const float c00[3] = {qd.c00.x, qd.c00.y, qd.c00.z}, c10[3] = {qd.c10.x, qd.c10.y, qd.c10.z};
        const float c01[3] = {qd.c01.x, qd.c01.y, qd.c01.z}, c11[3] = {qd.c11.x, qd.c11.y, qd.c11.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float d10 = c10[k] - c00[k], d11 = c11[k] - c01[k];
            const float a = fmaf(cell.fu, d10, c00[k]), bb = fmaf(cell.fu, d11, c01[k]);
            dcv[k] = bb - a;
            col[k] = fmaf(cell.fv, dcv[k], a);
            dcu[k] = fmaf(cell.fv, d11 - d10, d10);
        }
    }
    col[0] += q3.y;
    col[1] += q3.z;
    col[2] += q3.w;
    const float w = alpha * Ti;
    const float ch0 = w * px.dC0, ch1 = w * px.dC1, ch2 = w * px.dC2;
    put<ACC>(g[kGRgb + 0], ch0);
    put<ACC>(g[kGRgb + 1], ch1);
    put<ACC>(g[kGRgb + 2], ch2);
    // adj-bilinear: grid adjoint and uv adjoint
    float uh = 0.0f, vh = 0.0f;
    if (N == 1) {
        // the single texel is corner 0
        put<ACC>(g[kCornerSlot + 0], ch0);
        put<ACC>(g[kCornerSlot + 1], ch1);
        put<ACC>(g[kCornerSlot + 2], ch2);
    } else {
        const float fu = cell.fu, fv = cell.fv;
        const float w00 = (1.0f - fu) * (1.0f - fv), w10 = fu * (1.0f - fv);
        const float w01 = (1.0f - fu) * fv, w11 = fu * fv;
        // d colour / d f_u and d f_v, dotted with the colour adjoint
        const float fuh = fmaf(ch0, dcu[0], fmaf(ch1, dcu[1], ch2 * dcu[2]));
        const float fvh = fmaf(ch0, dcv[0], fmaf(ch1, dcv[1], ch2 * dcv[2]));
        if (VAR) {
            // the grid's size is the splat's own: every weight to the texel pass
            rem.w00 = w00;
            rem.w10 = w10;
            rem.w01 = w01;
            rem.w11 = w11;
        } else if (N == 2) {
            // every texel of a 2 x 2 grid is a corner: all four weights go to the
            // warp-reduced corner slots
            put<ACC>(g[kCornerSlot + 0], w00 * ch0); put<ACC>(g[kCornerSlot + 1], w00 * ch1); put<ACC>(g[kCornerSlot + 2], w00 * ch2);
            put<ACC>(g[kCornerSlot + 3], w01 * ch0); put<ACC>(g[kCornerSlot + 4], w01 * ch1); put<ACC>(g[kCornerSlot + 5], w01 * ch2);
            put<ACC>(g[kCornerSlot + 6], w10 * ch0); put<ACC>(g[kCornerSlot + 7], w10 * ch1); put<ACC>(g[kCornerSlot + 8], w10 * ch2);
            put<ACC>(g[kCornerSlot + 9], w11 * ch0); put<ACC>(g[kCornerSlot + 10], w11 * ch1); put<ACC>(g[kCornerSlot + 11], w11 * ch2);
        } else if (N == 4) {
            // the warp routes these through a corner or border-line window of
            // the reduce-scatter, or the full-grid layout (grid4_window)
            rem.w00 = w00;
            rem.w10 = w10;
            rem.w01 = w01;
            rem.w11 = w11;
        } else {
            // weights landing on a grid-corner texel go to the warp-reduced
            // corner slots; the rest (edge and interior texels) to the texel pass
            const int iu = cell.base / N, iv = cell.base - iu * N;
            const float wc0 = (iu == 0 && iv == 0) ? w00 : 0.0f;
            const float wc1 = (iu == 0 && iv == N - 2) ? w01 : 0.0f;
            const float wc2 = (iu == N - 2 && iv == 0) ? w10 : 0.0f;
            const float wc3 = (iu == N - 2 && iv == N - 2) ? w11 : 0.0f;
            put<ACC>(g[kCornerSlot + 0], wc0 * ch0); put<ACC>(g[kCornerSlot + 1], wc0 * ch1); put<ACC>(g[kCornerSlot + 2], wc0 * ch2);
            put<ACC>(g[kCornerSlot + 3], wc1 * ch0); put<ACC>(g[kCornerSlot + 4], wc1 * ch1); put<ACC>(g[kCornerSlot + 5], wc1 * ch2);
            put<ACC>(g[kCornerSlot + 6], wc2 * ch0); put<ACC>(g[kCornerSlot + 7], wc2 * ch1); put<ACC>(g[kCornerSlot + 8], wc2 * ch2);
            put<ACC>(g[kCornerSlot + 9], wc3 * ch0); put<ACC>(g[kCornerSlot + 10], wc3 * ch1); put<ACC>(g[kCornerSlot + 11], wc3 * ch2);
            rem.w00 = w00 - wc0;
            rem.w10 = w10 - wc2;
            rem.w01 = w01 - wc1;
            rem.w11 = w11 - wc3;
        }
        rem.base = cell.base;
        rem.c0 = ch0;
        rem.c1 = ch1;
        rem.c2 = ch2;
        if (u > -sigma && u < sigma) uh = kN * fuh;
        if (v > -sigma && v < sigma) vh = kN * fvh;
    }
    // alpha adjoint
    const float z = fabsf(q1.w);  // negated on flagged records
    const float zi = uvb ? q1.z * z * rz : z;
    float ah = px.dC0 * (col[0] * Ti - px.S0 * iom) + px.dC1 * (col[1] * Ti - px.S1 * iom) +
               px.dC2 * (col[2] * Ti - px.S2 * iom);
    ah += px.dD * (zi * Ti - px.SD * iom) + px.dTfin * iom;
    px.S0 = fmaf(col[0], w, px.S0);
    px.S1 = fmaf(col[1], w, px.S1);
    px.S2 = fmaf(col[2], w, px.S2);
    px.SD = fmaf(zi, w, px.SD);
    px.T = Ti;
    const float zih = px.dD * w;
    float rhoh = 0.0f;
    if (!clamped) {
        put<ACC>(g[kGOpacity], ah * G);
        rhoh = -0.5f * alpha * ah;
    }
    // W = zeta_z zeta_z^: the depth's and (u, v)'s dependence on zeta_z
    float W;
    if (uvb) {
        uh = fmaf(2.0f * u, rhoh, uh);
        vh = fmaf(2.0f * v, rhoh, vh);
        // the hit depth zi moves with the plane coordinates: its adjoint enters W
        W = -zih * zi;
    } else {
        const float c = -2.0f * kLowPass * rhoh;
        g[kGCentreLP + 0] += c * dx;
        g[kGCentreLP + 1] += c * dy;
        g[kGDepthLP] += zih;
        W = 0.0f;
    }
    W = W - fmaf(uh, u, vh * v);
    put<ACC>(g[kGH + 0], uh * u);
    put<ACC>(g[kGH + 1], uh * v);
    put<ACC>(g[kGH + 2], uh);
    put<ACC>(g[kGH + 3], vh * u);
    put<ACC>(g[kGH + 4], vh * v);
    put<ACC>(g[kGH + 5], vh);
    put<ACC>(g[kGH + 6], W * u);
    put<ACC>(g[kGH + 7], W * v);
    put<ACC>(g[kGH + 8], W);
    return true;
}

// Grids of N = 4 (16 texels, index 4 i_u + i_v).  The warp ORs the masks of
// the texels its lanes weight (nonzero bilinear weight).  When they all lie
// among the four grid corners (a pixel whose u and v are both clamped to the
// grid's border weights one corner) or on one border line (first or last
// column i_u = 0, 3, or row i_v = 0, 3: a pixel with one clamped coordinate
// weights two neighbours along it), the weights move to slots kCornerSlot ..
// kCornerSlot + 11 of the 32-value reduce-scatter (window position q, channel
// c: slot kCornerSlot + 3q + c) and the window kind is returned: 0..3 the
// lines (texel grid4_texel(kind, q)), 4 the corners.  Otherwise 5: the lanes
// add their texel weights to global memory themselves.  Measured on a sample
// of camera 0 of the 1M-splat workload, 77 % of the (warp, splat) pairs fit a
// corner or line window.
constexpr unsigned kGrid4Corners = 0x9009u;                          // texels 0, 3, 12, 15
// border lines i_u = 0, i_u = 3, i_v = 0, i_v = 3
constexpr unsigned kGrid4Line0 = 0x000fu, kGrid4Line1 = 0xf000u, kGrid4Line2 = 0x1111u, kGrid4Line3 = 0x8888u;

__device__ __forceinline__ int grid4_texel(int kind, int q) {
    return kind == 0 ? q : kind == 1 ? 12 + q : kind == 2 ? 4 * q : kind == 3 ? 4 * q + 3
                                                                           : (q & 2 ? 12 : 0) + (q & 1 ? 3 : 0);
}

template <int P>
__device__ __forceinline__ int grid4_window(const Rem rem[P], float g[32]) {
    unsigned m = 0u;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const Rem &r = rem[p];
        m |= (r.w00 != 0.0f ? 1u << r.base : 0u) | (r.w01 != 0.0f ? 2u << r.base : 0u) |
             (r.w10 != 0.0f ? 16u << r.base : 0u) | (r.w11 != 0.0f ? 32u << r.base : 0u);
    }
    const unsigned tm = __reduce_or_sync(0xffffffffu, m);
    int kind;
    if ((tm & ~kGrid4Corners) == 0u) kind = 4;
    else if ((tm & ~kGrid4Line0) == 0u) kind = 0;
    else if ((tm & ~kGrid4Line1) == 0u) kind = 1;
    else if ((tm & ~kGrid4Line2) == 0u) kind = 2;
    else if ((tm & ~kGrid4Line3) == 0u) kind = 3;
    else return 5;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const Rem &r = rem[p];
        float w0, w1, w2, w3;
        if (kind == 4) {
            // a lane weights at most one corner: (0,0) by w00 from cell (0,0),
            // (0,3) by w01 from (0,2), (3,0) by w10 from (2,0), (3,3) by w11 from (2,2)
            w0 = r.base == 0 ? r.w00 : 0.0f;
            w1 = r.base == 2 ? r.w01 : 0.0f;
            w2 = r.base == 8 ? r.w10 : 0.0f;
            w3 = r.base == 10 ? r.w11 : 0.0f;
        } else {
            // the lane's weights lie on the line: wa at position pos, wb at pos + 1
            const int pos = kind < 2 ? (r.base & 3) : (r.base >> 2);
            const float wa = kind == 0 ? r.w00 : kind == 1 ? r.w10 : kind == 2 ? r.w00 : r.w01;
            const float wb = kind == 0 ? r.w01 : kind == 1 ? r.w11 : kind == 2 ? r.w10 : r.w11;
            w0 = pos == 0 ? wa : 0.0f;
            w1 = pos == 0 ? wb : (pos == 1 ? wa : 0.0f);
            w2 = pos == 1 ? wb : (pos == 2 ? wa : 0.0f);
            w3 = pos == 2 ? wb : 0.0f;
        }
        g[kCornerSlot + 0] = fmaf(w0, r.c0, g[kCornerSlot + 0]);
        g[kCornerSlot + 1] = fmaf(w0, r.c1, g[kCornerSlot + 1]);
        g[kCornerSlot + 2] = fmaf(w0, r.c2, g[kCornerSlot + 2]);
        g[kCornerSlot + 3] = fmaf(w1, r.c0, g[kCornerSlot + 3]);
        g[kCornerSlot + 4] = fmaf(w1, r.c1, g[kCornerSlot + 4]);
        g[kCornerSlot + 5] = fmaf(w1, r.c2, g[kCornerSlot + 5]);
        g[kCornerSlot + 6] = fmaf(w2, r.c0, g[kCornerSlot + 6]);
        g[kCornerSlot + 7] = fmaf(w2, r.c1, g[kCornerSlot + 7]);
        g[kCornerSlot + 8] = fmaf(w2, r.c2, g[kCornerSlot + 8]);
        g[kCornerSlot + 9] = fmaf(w3, r.c0, g[kCornerSlot + 9]);
        g[kCornerSlot + 10] = fmaf(w3, r.c1, g[kCornerSlot + 10]);
        g[kCornerSlot + 11] = fmaf(w3, r.c2, g[kCornerSlot + 11]);
    }
    return kind;
}

template <int TS, int N, typename TexT, int P, bool VAR>
__device__ __forceinline__ void bwd_tile(const Frame &f, const RenderBwdBufs &b, int batch, uint32_t tile) {
    constexpr int NT = TS * TS / P;
    constexpr int NN = N * N;
    constexpr int TEXF = NN * 3;
    extern __shared__ float4 smem[];
    float4 *s_rec = smem;
    float4 *s_fp = s_rec + 4 * batch;  // [batch][3] footprints
    staged_t<TexT> *s_tex = reinterpret_cast<staged_t<TexT> *>(s_fp + 3 * batch);
    int32_t *s_k = reinterpret_cast<int32_t *>(s_tex + batch * NN);
    uint32_t *s_j = reinterpret_cast<uint32_t *>(s_k + batch);
    uint2 *s_box = reinterpret_cast<uint2 *>(s_j + batch);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_box + batch);
    int32_t *s_n = reinterpret_cast<int32_t *>(s_mask + batch);  // VAR: per-splat grid size
    __shared__ uint32_t s_maxlast;

    const int ci = camera_of_tile(f, tile);
    const CamDev &cam = f.cams[ci];
    const SceneDev &sc = f.scenes[cam.scene];
    const uint32_t lt = tile - cam.tile_off;
    const int tx = int(lt % uint32_t(cam.tiles_x)), ty = int(lt / uint32_t(cam.tiles_x));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbit = 1u << warp;  // this warp's 8 x 4P block in the splat masks
    const int px0 = tx * TS + (warp % (TS / 8)) * 8 + (lane & 7);
    const int py0 = ty * TS + (warp / (TS / 8)) * (4 * P) + (lane >> 3);
    const uint2 range = b.fw.ranges[tile];
    const float sigma = sc.sigma;
    const float kN = float(N - 1) / (2.0f * sigma);

    Pix pix[P];
    uint32_t mylast = 0;
    // evaluated (live) pairs of this warp, counted once per batch into shared
    // memory: per-pair counters held registers through the event loop
    // (measured: 1.1 ms of 32.3 on the 16-view workload at N = 4, through the
    // register cap; a ballot per pair instead cost 0.5 ms more)
    __shared__ uint32_t s_np[NT / 32];
    if (lane == 0) s_np[warp] = 0;
    // per warp and batch, the bits of the staged splats whose footprint may
    // touch its block (32 splats a word; a batch holds at most NT splats): the
    // walk visits only those (measured against testing every staged splat's
    // mask: 31.2 -> 30.1 ms at N = 4, 38.6 -> 35.5 ms at N = 8)
    __shared__ uint32_t s_wm[NT / 32][NT / 32];
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p) {
        Pix &q = pix[p];
        const int py = py0 + 4 * p;
        q.inside = px0 < cam.width && py < cam.height;
        q.xf = float(px0) + 0.5f;
        q.yf = float(py) + 0.5f;
        q.T = 1.0f;
        q.dC0 = q.dC1 = q.dC2 = q.dD = 0.0f;
        q.S0 = q.S1 = q.S2 = q.SD = 0.0f;
        q.last = 0;
        float dA = 0.0f, T_final = 1.0f;
        if (q.inside) {
            const int64_t pi = cam.pix_off + int64_t(py) * cam.width + px0;
            q.T = T_final = b.fw.t_final[pi];
            q.last = b.fw.last[pi];
            q.dC0 = b.d_rgb[3 * pi + 0];
            q.dC1 = b.d_rgb[3 * pi + 1];
            q.dC2 = b.d_rgb[3 * pi + 2];
            if (b.d_depth) q.dD = b.d_depth[pi];
            if (b.d_alpha) dA = b.d_alpha[pi];
        }
        const float bgdot = q.dC0 * f.bg[0] + q.dC1 * f.bg[1] + q.dC2 * f.bg[2];
        q.dTfin = (dA - bgdot) * T_final;  // times 1/(1-alpha) per splat
        mylast = max(mylast, q.last);
    }
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, mylast);
    if (lane == 0 && wlast) atomicMax(&s_maxlast, wlast);
    __syncthreads();
    const int max_last = int(s_maxlast);
    float *g_tex = sc.g_tex;
    const int my_q16 = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    // flat index (i_u N + i_v) of the corner texel this lane's reduced value feeds
    const int my_corner = lane >= kCornerSlot && lane < kCornerSlot + 12 ? (lane - kCornerSlot) / 3 : -1;
    const int my_corner_off = my_corner < 0 ? 0
                              : 3 * ((my_corner & 2 ? (N - 1) * N : 0) + (my_corner & 1 ? N - 1 : 0)) +
                                    (lane - kCornerSlot) % 3;
    // N = 4: window position and channel of this lane's reduced slot
    const int my_q = (lane - kCornerSlot) / 3, my_c = (lane - kCornerSlot) - 3 * ((lane - kCornerSlot) / 3);
    constexpr bool kGrid4 = N == 4 && !VAR;

    for (int be = max_last; be > 0; be -= batch) {
        const int bs = max(0, be - batch), nb = be - bs;
        stage_batch<N, NT, TexT, TS, 4 * P, false, VAR>(b.fw, cam, sc, range.x + bs, nb, tx * TS, ty * TS, s_rec,
                                                        s_tex, s_k, s_j, s_box, s_mask, s_fp, s_n);
        __syncthreads();
        // splats at or beyond the warp's last contributor are skipped warp-wide;
        // below it at least one lane of the warp is active
        const int i_hi = min(nb, int(wlast) - bs);
        {
            // per pixel, the splats of its warp block below its last contributor
            uint32_t cnt = 0;
            for (int c = 0; c < i_hi; c += 32) {
                const unsigned word = __ballot_sync(0xffffffffu, c + lane < i_hi && (s_mask[c + lane] & wbit));
                if (lane == 0) s_wm[warp][c >> 5] = word;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const int k = pix[p].inside ? min(int(pix[p].last) - bs, i_hi) - c : 0;
                    cnt += __popc(k >= 32 ? word : (k <= 0 ? 0u : word & ((1u << k) - 1u)));
                }
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0) s_np[warp] += cnt;
        }
        __syncwarp();
        // back to front over the set bits
        for (int c = (i_hi - 1) >> 5; c >= 0; --c)
            for (unsigned wd = s_wm[warp][c]; wd;) {
            const int i = 32 * c + 31 - __clz(wd);
            wd &= ~(1u << (i & 31));
            float g[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) g[q] = 0.0f;
            Rem rem[P];
            const RecordLo *lo = s_rec[4 * i + 1].w < 0.0f ? b.fw.rec_lo + staged_record(cam, s_k[i]) : nullptr;
            const int nk = VAR ? s_n[i] : N;
            const float kNk = VAR ? float(nk - 1) / (2.0f * sigma) : kN;
            bool act = pair_adjoint<N, TexT, false, VAR>(pix[0], uint32_t(bs + i), s_rec + 4 * i, lo, s_tex + i * NN,
                                                         sigma, kNk, nk, g, rem[0]);
#pragma unroll
            for (int p = 1; p < P; ++p)
                act |= pair_adjoint<N, TexT, true, VAR>(pix[p], uint32_t(bs + i), s_rec + 4 * i, lo, s_tex + i * NN,
                                                        sigma, kNk, nk, g, rem[p]);
            if (!__any_sync(0xffffffffu, act)) continue;
            if (kGrid4 && P == 1 && __popc(__ballot_sync(0xffffffffu, act)) <= kFewLanes4) {
                // few contributing lanes: each adds its own values
                if (act) {
                    // the record's 16 slots are 64-byte aligned (rows of the gradient array)
                    float4 *rg = reinterpret_cast<float4 *>(b.rec_grad + int64_t(s_j[i]) * kRecGrad);
#pragma unroll
                    for (int q = 0; q < kRecVals / 4; ++q)
                        atomicAdd(rg + q, make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]));
                    if (g_tex) {
                        const Rem &r = rem[0];
                        float *t = g_tex + int64_t(s_k[i]) * TEXF + 3 * r.base;
                        if (r.w00 != 0.0f) add_texel(t, r.w00, r.c0, r.c1, r.c2);
                        if (r.w10 != 0.0f) add_texel(t + 3 * N, r.w10, r.c0, r.c1, r.c2);
                        if (r.w01 != 0.0f) add_texel(t + 3, r.w01, r.c0, r.c1, r.c2);
                        if (r.w11 != 0.0f) add_texel(t + 3 * N + 3, r.w11, r.c0, r.c1, r.c2);
                    }
                }
                continue;
            }
            const int kind = kGrid4 ? grid4_window<P>(rem, g) : 0;
            const float tot = warp_reduce_scatter32(g, lane);
            // this splat's texel gradients, formed where used (fewer live registers)
            const bool want_tex = g_tex != nullptr;
            auto gt = [&]() -> float * { return g_tex + int64_t(s_k[i]) * TEXF; };
            if (tot != 0.0f) {
                if (lane < kCornerSlot) {
                    atomicAdd(b.rec_grad + (s_j[i] * uint32_t(kRecGrad) + uint32_t(lane)), tot);
                } else if (want_tex) {
                    if (kGrid4) {
                        if (lane < kCornerSlot + 12) atomicAdd(gt() + 3 * grid4_texel(kind, my_q) + my_c, tot);
                    } else if (my_corner >= 0) {
                        atomicAdd(gt() + my_corner_off, tot);
                    }
                }
            }
            if (N > 4 || VAR || (kGrid4 && kind == 5)) {
                // edge / interior texels: added by each lane, or, when the lanes
                // share one cell (the same four texels), one reduce-scatter and
                // one atomic per value (a lane's P pixels join the same group when
                // they share its cell)
                bool has[P];
                unsigned pend[P];
                unsigned any_pend = 0u;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    has[p] = rem[p].any();
                    pend[p] = __ballot_sync(0xffffffffu, has[p]);
                    any_pend |= pend[p];
                }
                if (!want_tex) any_pend = 0u;
                int cells = 0;
                if (any_pend && !kGrid4) {
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const unsigned same = __match_any_sync(0xffffffffu, has[p] ? rem[p].base : -1);
                        cells += __popc(__ballot_sync(0xffffffffu, has[p] && (__ffs(same) - 1) == lane));
                    }
                }
                if (any_pend && (kGrid4 || cells > kDirectCells)) {
                    float *st = gt();
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (!has[p]) continue;
                        const Rem &r = rem[p];
                        float *t = st + 3 * r.base;
                        if (r.w00 != 0.0f) {
                            atomicAdd(t + 0, r.w00 * r.c0); atomicAdd(t + 1, r.w00 * r.c1); atomicAdd(t + 2, r.w00 * r.c2);
                        }
                        if (r.w10 != 0.0f) {
                            atomicAdd(t + 3 * N + 0, r.w10 * r.c0); atomicAdd(t + 3 * N + 1, r.w10 * r.c1);
                            atomicAdd(t + 3 * N + 2, r.w10 * r.c2);
                        }
                        if (r.w01 != 0.0f) {
                            atomicAdd(t + 3, r.w01 * r.c0); atomicAdd(t + 4, r.w01 * r.c1); atomicAdd(t + 5, r.w01 * r.c2);
                        }
                        if (r.w11 != 0.0f) {
                            atomicAdd(t + 3 * N + 3, r.w11 * r.c0); atomicAdd(t + 3 * N + 4, r.w11 * r.c1);
                            atomicAdd(t + 3 * N + 5, r.w11 * r.c2);
                        }
                    }
                    any_pend = 0u;
                }
                while (any_pend) {
                    // the first pending entry (pixel slot p0, lowest lane) names the cell
                    int p0 = 0;
#pragma unroll
                    for (int p = P - 1; p >= 0; --p)
                        if (pend[p]) p0 = p;
                    int kb = rem[0].base;
#pragma unroll
                    for (int p = 1; p < P; ++p)
                        if (p0 == p) kb = rem[p].base;
                    unsigned lead_mask = pend[0];
#pragma unroll
                    for (int p = 1; p < P; ++p)
                        if (p0 == p) lead_mask = pend[p];
                    const int key = __shfl_sync(0xffffffffu, kb, __ffs(lead_mask) - 1);
                    float h[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) h[q] = 0.0f;
                    any_pend = 0u;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const Rem &r = rem[p];
                        const bool mine = ((pend[p] >> lane) & 1u) && r.base == key;
                        pend[p] &= ~__ballot_sync(0xffffffffu, mine);
                        any_pend |= pend[p];
                        if (mine) {
                            h[0] += r.w00 * r.c0; h[1] += r.w00 * r.c1; h[2] += r.w00 * r.c2;
                            h[3] += r.w10 * r.c0; h[4] += r.w10 * r.c1; h[5] += r.w10 * r.c2;
                            h[6] += r.w01 * r.c0; h[7] += r.w01 * r.c1; h[8] += r.w01 * r.c2;
                            h[9] += r.w11 * r.c0; h[10] += r.w11 * r.c1; h[11] += r.w11 * r.c2;
                        }
                    }
                    const float t = warp_reduce_scatter16(h, lane);
                    if (!(lane & 1) && my_q16 < 12 && t != 0.0f) {
                        const int k = my_q16 / 3, c = my_q16 - 3 * k;
                        // k: 0 -> (iu, iv), 1 -> (iu+1, iv), 2 -> (iu, iv+1), 3 -> (iu+1, iv+1)
                        const int off = 3 * (key + ((k & 1) ? N : 0) + ((k & 2) ? 1 : 0)) + c;
                        atomicAdd(gt() + off, t);
                    }
                }
            }
        }
        __syncthreads();  // the next batch's staging overwrites this one
    }
    if (lane == 0 && s_np[warp]) atomicAdd(&b.fw.cnt->pairs_bwd, (unsigned long long)s_np[warp]);
}

// Resident blocks per SM the register budget is set for: one pixel per thread
// fits 64 registers at 1024 threads per SM; two pixels per thread get ~100.
template <int TS, int P>
constexpr int min_blocks() {
    return P == 1 ? 1024 / (TS * TS) : 1280 / (TS * TS);
}

template <int TS, int N, typename TexT, int P, bool VAR>
__global__ void __launch_bounds__(TS * TS / P, min_blocks<TS, P>())
    render_bwd_kernel(Frame f, RenderBwdBufs b, int batch, TileSched ts) {
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
        bwd_tile<TS, N, TexT, P, VAR>(f, b, batch, tile);
    }
}

template <int TS, int N, typename TexT, int P, bool VAR = false>
cudaError_t launch_t(const Frame &f, const RenderBwdBufs &b, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    constexpr int NT = TS * TS / P;
    const size_t smem = bwd_stage_bytes<N, TexT>(batch) + (VAR ? size_t(batch) * 4 : 0);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(render_bwd_kernel<TS, N, TexT, P, VAR>,
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
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_bwd_kernel<TS, N, TexT, P, VAR>, NT, smem);
            smem_seen = smem;
            if (per_sm < 1) per_sm = 1;
        }
        grid = std::min<unsigned>(grid, unsigned(per_sm * sms));
    } else {
        ts.work = nullptr;
    }
    if (grid == 0) return cudaSuccess;
    render_bwd_kernel<TS, N, TexT, P, VAR><<<grid, NT, smem, s>>>(f, b, batch, ts);
    count_launches(1);
    return cudaGetLastError();
}

template <int TS, typename TexT, int P>
cudaError_t launch_n(const Frame &f, const RenderBwdBufs &b, int N, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    switch (N) {
        case 1: return launch_t<TS, 1, TexT, P>(f, b, batch, ts, persistent, s);
        case 2: return launch_t<TS, 2, TexT, P>(f, b, batch, ts, persistent, s);
        case 4: return launch_t<TS, 4, TexT, P>(f, b, batch, ts, persistent, s);
        case 8: return launch_t<TS, 8, TexT, P>(f, b, batch, ts, persistent, s);
        case 16: return launch_t<TS, 16, TexT, P>(f, b, batch, ts, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

// Per-splat grid sizes: 16 x 16 tiles, one pixel per thread (N is the grid
// block of the scene).
template <typename TexT>
cudaError_t launch_var(const Frame &f, const RenderBwdBufs &b, int N, int batch, TileSched ts, bool persistent,
                       cudaStream_t s) {
    switch (N) {
        case 2: return launch_t<16, 2, TexT, 1, true>(f, b, batch, ts, persistent, s);
        case 4: return launch_t<16, 4, TexT, 1, true>(f, b, batch, ts, persistent, s);
        case 8: return launch_t<16, 8, TexT, 1, true>(f, b, batch, ts, persistent, s);
        case 16: return launch_t<16, 16, TexT, 1, true>(f, b, batch, ts, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int TS, int P>
cudaError_t launch_d(const Frame &f, const RenderBwdBufs &b, int g, int N, int batch, TileSched ts, bool persistent,
                     cudaStream_t s) {
    if (f.group_var[g]) {
        if constexpr (P == 1) {
            if (TS != 16) return cudaErrorInvalidValue;
            switch (f.group_dtype[g]) {
                case GB_F16: return launch_var<__half>(f, b, N, batch, ts, persistent, s);
                case GB_BF16: return launch_var<__nv_bfloat16>(f, b, N, batch, ts, persistent, s);
                default: return launch_var<float>(f, b, N, batch, ts, persistent, s);
            }
        } else {
            return cudaErrorInvalidValue;
        }
    }
    switch (f.group_dtype[g]) {
        case GB_F16: return launch_n<TS, __half, P>(f, b, N, batch, ts, persistent, s);
        case GB_BF16: return launch_n<TS, __nv_bfloat16, P>(f, b, N, batch, ts, persistent, s);
        default: return launch_n<TS, float, P>(f, b, N, batch, ts, persistent, s);
    }
}

}  // namespace bwd

// Launches the backward render of every render group with P pixels per thread.
template <int P>
cudaError_t launch_render_bwd_p(const Frame &f, const RenderBwdBufs &b, int batch, const uint32_t *tile_list,
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
            case 8: e = bwd::launch_d<8, P>(f, b, g, N, batch, ts, persistent, s); break;
            case 16: e = bwd::launch_d<16, P>(f, b, g, N, batch, ts, persistent, s); break;
            case 32: e = bwd::launch_d<32, P>(f, b, g, N, batch, ts, persistent, s); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbill
