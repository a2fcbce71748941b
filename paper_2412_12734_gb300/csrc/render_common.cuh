// Per-tile render helpers shared by the forward and backward kernels.
#pragma once

#include <type_traits>

#include "gbill_internal.cuh"

namespace gbill {

// A staged texel: FP32 grids, and with WIDE any grid, as RGBA float4 (16
// bytes, alpha unused: one 128-bit shared load); otherwise FP16 and BF16 grids
// in their storage type as RGB + pad (8 bytes: one 64-bit load, converted
// exactly to FP32 at use).  The forward stages grids of N <= 4 wide (its
// shared memory has room, and the lookups skip the conversion); the backward
// stages them narrow, for deeper batches in the same shared memory.
template <typename TexT, bool WIDE = false>
using staged_t = typename std::conditional<WIDE || sizeof(TexT) == 4, float4, uint2>::type;

// Bytes of dynamic shared memory for one staged batch: records, footprints,
// colour grids, splat indices, pixel rectangles, warp-block masks and (with
// bwd) record/grid gradient accumulators.
template <int N, typename TexT, bool WIDE = false>
__host__ __device__ inline size_t stage_bytes(int batch, bool bwd) {
    const int texf = N * N * 3;
    size_t b = size_t(batch) * (64 + 48 + sizeof(staged_t<TexT, WIDE>) * N * N + 20);
    if (bwd) b += size_t(batch) * (4 * kRecGrad + 4 * texf);
    return b;
}

// Staged bytes of one batch of the pixel-parallel backward (render_bwd.cuh),
// which adds its gradients to global memory and holds no accumulators in
// shared memory.
template <int N, typename TexT>
__host__ __device__ inline size_t bwd_stage_bytes(int batch) {
    return stage_bytes<N, TexT>(batch, false);
}

// 1 / x through the SFU (max error 1 ulp; flush-to-zero).
__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Footprint of a splat for the warp-block test: alpha = o exp(-rho/2) >=
// 1/255 exactly when rho <= rho_c = 2 ln(255 o), and rho = min(rho_uv,
// rho_lp), so the footprint is the union of the low-pass disk 2 |d|^2 <= rho_c
// and the plane-hit region (a.d)^2 + (b.d)^2 <= rho_c (c.d)^2, d = (dx, dy, 1)
// about the projected centre: q(d) = d^T A d + 2 B.d + C <= 0 with A positive
// definite for a bounded footprint.  rho_c carries a 1/64 relative margin; a
// near-degenerate A (relative cancellation below 2^-10 in a diagonal entry
// or the determinant) marks the splat as "never cull" through an infinite
// disk radius.  Stored per staged splat as three float4:
//   k0 = (A00, A01, A11, C), k1 = (B0, B1, 1/A00, 1/A11), k2 = (e_x, e_y, rho_c/2, 0)
// with e the conic's centre (minimiser of q).
__device__ __forceinline__ void footprint_setup(const float4 &q0, const float4 &q1, float o, float4 *k) {
    k[0] = k[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    k[2] = make_float4(0.0f, 0.0f, INFINITY, 0.0f);
    if (!(o * 255.0f > 1.0f)) return;  // a culled record never reaches a tile; no claim here
    const float rc0 = 2.0f * __logf(255.0f * o);
    const float rc = fmaf(rc0, 1.0f / 64.0f, rc0) + 1.0f / 64.0f;
    const float a0 = q0.x, a1 = q0.y, b0 = q0.z, b1 = q0.w, c0 = q1.x, c1 = q1.y, c2 = q1.z;
    const float p00 = fmaf(a0, a0, b0 * b0), n00 = rc * c0 * c0;
    const float p11 = fmaf(a1, a1, b1 * b1), n11 = rc * c1 * c1;
    const float A00 = p00 - n00, A11 = p11 - n11;
    if (!(A00 > (p00 + n00) * (1.0f / 1024.0f)) || !(A11 > (p11 + n11) * (1.0f / 1024.0f))) return;
    const float A01 = fmaf(a0, a1, b0 * b1) - rc * c0 * c1;
    const float det = A00 * A11 - A01 * A01;
    if (!(det > A00 * A11 * (1.0f / 1024.0f))) return;
    const float B0 = -rc * c0 * c2, B1 = -rc * c1 * c2, Cq = -rc * c2 * c2;
    const float idet = fast_rcp(det);
    k[0] = make_float4(A00, A01, A11, Cq);
    k[1] = make_float4(B0, B1, fast_rcp(A00), fast_rcp(A11));
    k[2] = make_float4((A01 * B1 - A11 * B0) * idet, (A01 * B0 - A00 * B1) * idet, 0.5f * rc, 0.0f);
}

// Whether the pixel centres of the block [bx0, bx0 + 7] x [by0, by0 + BH - 1]
// can hold a pixel with alpha >= 1/255 for a splat with centre record q2,
// pixel rectangle `box` and footprint k (footprint_setup): the block's centre
// rectangle, clipped to `box`, meets the low-pass disk or the plane-hit
// region (minimum of q over the rectangle: at the conic's centre if inside,
// else on one of the four edges, each a clamped 1-D minimum).  Only blocks
// that the per-pixel FP32 test would skip are dropped.
template <int BH>
__device__ __forceinline__ bool block_hits(const float4 &q2, uint2 box, const float4 *k, int bx0, int by0) {
    const int rx0 = max(int(box.x & 0xffffu), bx0), rx1 = min(int(box.y & 0xffffu), bx0 + 7);
    const int ry0 = max(int(box.x >> 16), by0), ry1 = min(int(box.y >> 16), by0 + BH - 1);
    if (rx0 > rx1 || ry0 > ry1) return false;
    const float X0 = (float(rx0) + 0.5f - q2.x) - q2.z, X1 = (float(rx1) + 0.5f - q2.x) - q2.z;
    const float Y0 = (float(ry0) + 0.5f - q2.y) - q2.w, Y1 = (float(ry1) + 0.5f - q2.y) - q2.w;
    const float4 k0 = k[0], k1 = k[1], k2 = k[2];
    // low-pass disk: nearest point of the rectangle to the centre
    const float nx = fminf(fmaxf(0.0f, X0), X1), ny = fminf(fmaxf(0.0f, Y0), Y1);
    if (fmaf(nx, nx, ny * ny) <= k2.z) return true;
    if (k2.x >= X0 && k2.x <= X1 && k2.y >= Y0 && k2.y <= Y1) return true;
    const float A00 = k0.x, A01 = k0.y, A11 = k0.z, Cq = k0.w, B0 = k1.x, B1 = k1.y;
    auto q = [&](float x, float y) {
        return fmaf(x, fmaf(A00, x, 2.0f * fmaf(A01, y, B0)), fmaf(y, fmaf(A11, y, 2.0f * B1), Cq));
    };
    const float yA = fminf(fmaxf(-fmaf(A01, X0, B1) * k1.w, Y0), Y1);
    const float yB = fminf(fmaxf(-fmaf(A01, X1, B1) * k1.w, Y0), Y1);
    const float xA = fminf(fmaxf(-fmaf(A01, Y0, B0) * k1.z, X0), X1);
    const float xB = fminf(fmaxf(-fmaf(A01, Y1, B0) * k1.z, X0), X1);
    const float m = fminf(fminf(q(X0, yA), q(X1, yB)), fminf(q(xA, Y0), q(xB, Y1)));
    return m <= 0.0f;
}

// A staged texel as FP32 RGB (exact for FP16 / BF16 storage).
template <typename T>
__device__ __forceinline__ float4 texel_rgb(const float4 &t, T) {
    return t;
}
__device__ __forceinline__ float4 texel_rgb(const uint2 &t, __half) {
    const float2 rg = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
    return make_float4(rg.x, rg.y, __low2float(*reinterpret_cast<const __half2 *>(&t.y)), 0.0f);
}
__device__ __forceinline__ float4 texel_rgb(const uint2 &t, __nv_bfloat16) {
    const float2 rg = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.x));
    return make_float4(rg.x, rg.y, __low2float(*reinterpret_cast<const __nv_bfloat162 *>(&t.y)), 0.0f);
}

// Loads the records and colour grids of instances [first, first + nb) of a
// tile range into shared memory, and for every splat the mask of the tile's
// 8 x BH warp blocks (row-major, TS/8 per row) that its footprint may touch
// (block_hits); with VAR, the splat's own grid size (1..N) into s_n.  Caller
// synchronizes before and after.
template <int N, int NT, typename TexT, int TS, int BH, bool WIDE = false, bool VAR = false>
__device__ __forceinline__ void stage_batch(const RenderBufs &b, const CamDev &cam, const SceneDev &sc,
                                            uint32_t first, int nb, int tx0, int ty0, float4 *s_rec,
                                            staged_t<TexT, WIDE> *s_tex, int32_t *s_k, uint32_t *s_j,
                                            uint2 *s_box, uint32_t *s_mask, float4 *s_fp, int32_t *s_n = nullptr) {
    constexpr int NN = N * N;
    constexpr int NB = TS * TS / (8 * BH);  // warp blocks per tile: 1 to 32
    static_assert(32 % NB == 0 && NT % 32 == 0, "block masks are gathered within a warp");
    for (int t = threadIdx.x; t < nb; t += NT) {  // a batch deeper than the block: two or more per thread
        const uint32_t j = b.inst_val[first + t];
        const uint32_t r = b.perm[j];
        s_box[t] = b.pbox[r];
        const float4 *rp = reinterpret_cast<const float4 *>(b.rec + r);
        s_rec[4 * t + 0] = rp[0];
        s_rec[4 * t + 1] = rp[1];
        s_rec[4 * t + 2] = rp[2];
        s_rec[4 * t + 3] = rp[3];
        // grid row of the splat: its index in the scene, offset by the
        // camera's block for per-texel SH scenes (evaluated grid per record)
        s_k[t] = int32_t(int64_t(r) - cam.rec_off + cam.tex_row);
        s_j[t] = j;
        if (VAR) s_n[t] = min(max(int(sc.splat_n[int64_t(r) - cam.rec_off]), 1), N);
        float4 k[3];
        footprint_setup(rp[0], rp[1], rp[3].x, k);
        s_fp[3 * t + 0] = k[0];
        s_fp[3 * t + 1] = k[1];
        s_fp[3 * t + 2] = k[2];
    }
    __syncthreads();
    const int t = threadIdx.x;
    for (int base = 0; base < nb * NB; base += NT) {
        const int e = base + t, s = e / NB, w = e - s * NB;
        bool hit = false;
        if (e < nb * NB)
            hit = block_hits<BH>(s_rec[4 * s + 2], s_box[s], s_fp + 3 * s, tx0 + (w % (TS / 8)) * 8,
                                 ty0 + (w / (TS / 8)) * BH);
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        constexpr uint32_t kAll = NB == 32 ? 0xffffffffu : (1u << (NB & 31)) - 1u;
        if (e < nb * NB && w == 0) s_mask[s] = (bal >> ((t & 31) & ~(NB - 1))) & kAll;
    }
    const TexT *tex = static_cast<const TexT *>(sc.tex);
    if constexpr (sizeof(TexT) == 2 && NN % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(tex) & 7u) == 0) {
            // four texels (12 16-bit values, 24 bytes, 8-byte aligned) per step:
            // three 64-bit loads unpacked in registers
            constexpr int NQ = NN / 4;
            const uint2 *raw8 = reinterpret_cast<const uint2 *>(tex);
            for (int e = t; e < nb * NQ; e += NT) {
                const int s = e / NQ, o = e - s * NQ;
                const int64_t g = (int64_t(s_k[s]) * NQ + o) * 3;
                const uint2 a = raw8[g], b2 = raw8[g + 1], c = raw8[g + 2];
                // texel q holds values 3q, 3q + 1, 3q + 2 of h0..h11 = (a.x, a.y, b2.x, b2.y, c.x, c.y)
                const uint2 tx[4] = {make_uint2(a.x, a.y & 0xffffu), make_uint2((a.y >> 16) | (b2.x << 16), b2.x >> 16),
                                     make_uint2(b2.y, c.x & 0xffffu), make_uint2((c.x >> 16) | (c.y << 16), c.y >> 16)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if constexpr (sizeof(staged_t<TexT, WIDE>) == 16) {
                        const float4 f = texel_rgb(tx[q], TexT());
                        s_tex[4 * e + q] = make_float4(f.x, f.y, f.z, 0.0f);
                    } else {
                        s_tex[4 * e + q] = tx[q];
                    }
                }
            }
            return;
        }
    }
    if constexpr (sizeof(TexT) == 4 && NN % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(tex) & 15u) == 0) {
            // four FP32 texels (48 bytes, 16-byte aligned) per step: three 128-bit loads
            constexpr int NQ = NN / 4;
            const float4 *raw16 = reinterpret_cast<const float4 *>(tex);
            for (int e = t; e < nb * NQ; e += NT) {
                const int s = e / NQ, o = e - s * NQ;
                const int64_t g = (int64_t(s_k[s]) * NQ + o) * 3;
                const float4 a = raw16[g], b2 = raw16[g + 1], c = raw16[g + 2];
                s_tex[4 * e + 0] = make_float4(a.x, a.y, a.z, 0.0f);
                s_tex[4 * e + 1] = make_float4(a.w, b2.x, b2.y, 0.0f);
                s_tex[4 * e + 2] = make_float4(b2.z, b2.w, c.x, 0.0f);
                s_tex[4 * e + 3] = make_float4(c.y, c.z, c.w, 0.0f);
            }
            return;
        }
    }
    for (int e = t; e < nb * NN; e += NT) {
        const int s = e / NN, o = e - s * NN;
        const int64_t g = (int64_t(s_k[s]) * NN + o) * 3;
        if constexpr (sizeof(staged_t<TexT, WIDE>) == 16) {
            s_tex[e] = make_float4(load_as_float(tex, g), load_as_float(tex, g + 1), load_as_float(tex, g + 2), 0.0f);
        } else {
            // the stored 16-bit values, unconverted
            const unsigned short *raw = reinterpret_cast<const unsigned short *>(tex);
            s_tex[e] = make_uint2(uint32_t(raw[g]) | (uint32_t(raw[g + 1]) << 16), uint32_t(raw[g + 2]));
        }
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

// The same for a splat whose grid is n x n (1 <= n <= N), stored in rows and
// columns 0..n-1 of its N x N block; kN = (n - 1) / (2 sigma).  For n = 1 the
// cell is texel 0 with zero fractions (the constant colour).
template <int N>
__device__ __forceinline__ Cell<N> grid_cell_n(float u, float v, float sigma, float kN, int n) {
    Cell<N> c;
    const float top = float(n - 1);
    const float up = fminf(fmaxf((u + sigma) * kN, 0.0f), top);
    const float vp = fminf(fmaxf((v + sigma) * kN, 0.0f), top);
    const int iu = max(min(int(up), n - 2), 0), iv = max(min(int(vp), n - 2), 0);
    c.fu = up - float(iu);
    c.fv = vp - float(iv);
    c.base = iu * N + iv;
    return c;
}

// The four texels of a cell: (i_u, i_v), (i_u+1, i_v), (i_u, i_v+1), (i_u+1, i_v+1).
struct Quad {
    float4 c00, c10, c01, c11;
};

template <int N, typename TexT, bool WIDE = false>
__device__ __forceinline__ Quad grid_quad(const staged_t<TexT, WIDE> *g, const Cell<N> &c) {
    Quad q;
    q.c00 = texel_rgb(g[c.base], TexT());
    if (N == 1) {
        q.c10 = q.c01 = q.c11 = q.c00;
    } else {
        q.c10 = texel_rgb(g[c.base + N], TexT());
        q.c01 = texel_rgb(g[c.base + 1], TexT());
        q.c11 = texel_rgb(g[c.base + N + 1], TexT());
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

// Plane hit of the pixel centre (xf, yf) for a record (Record): the offset
// d = (dx, dy) from the projected centre and zeta = adj(T') (d, 1) up to the
// record's scale, so that u = zx / zz, v = zy / zz.
struct Hit {
    float dx, dy, zx, zy, zz;
};

// FP32 evaluation about the centre (every record not flagged precise).
__device__ __forceinline__ Hit plane_hit(float xf, float yf, const float4 &q0, const float4 &q1, const float4 &q2) {
    Hit h;
    h.dx = (xf - q2.x) - q2.z;
    h.dy = (yf - q2.y) - q2.w;
    h.zz = fmaf(q1.x, h.dx, fmaf(q1.y, h.dy, q1.z));
    h.zx = fmaf(q0.x, h.dx, q0.y * h.dy);
    h.zy = fmaf(q0.z, h.dx, q0.w * h.dy);
    return h;
}

// a0 x + a1 y + (l0 x + l1 y + k) with one rounding of the leading sum: the
// product a1 y splits exactly into p + e (FMA), a0 x + p is rounded once (FMA),
// and the low-order terms are added in FP32.
__device__ __forceinline__ float dot2_ext(float a0, float a1, float l0, float l1, float k, float x, float y) {
    const float p = __fmul_rn(a1, y);
    const float e = __fmaf_rn(a1, y, -p);
    const float s = __fmaf_rn(a0, x, p);
    return __fadd_rn(s, __fmaf_rn(l1, y, __fmaf_rn(l0, x, __fadd_rn(e, k))));
}

// Extended-precision evaluation for a flagged record (depth stored negated):
// the offsets from c_hi are exact (c_hi lies on the 1/512-pixel grid), the
// homography entries are the double-float pairs of Record + RecordLo, and
// each zeta component is the sum of its terms with only its own rounding
// left (error-free products and, for zeta_z, an error-free two-sum of the
// m21 dy + m22 part), so u and v carry a few ulps whatever the cancellation
// between the terms.  dx, dy (rounded) serve the low-pass term and the
// adjoints.
__device__ __forceinline__ Hit plane_hit_ext(float xf, float yf, const float4 &q0, const float4 &q1, const float4 &q2,
                                             const RecordLo &L) {
    Hit h;
    const float dxh = __fsub_rn(xf, q2.x), dyh = __fsub_rn(yf, q2.y);
    h.dx = __fsub_rn(dxh, q2.z);
    h.dy = __fsub_rn(dyh, q2.w);
    h.zx = dot2_ext(q0.x, q0.y, L.l0.x, L.l0.y, L.l2.x, dxh, dyh);
    h.zy = dot2_ext(q0.z, q0.w, L.l0.z, L.l0.w, L.l2.y, dxh, dyh);
    const float p = __fmul_rn(q1.y, dyh);
    const float e1 = __fmaf_rn(q1.y, dyh, -p);
    const float t = __fadd_rn(p, q1.z);
    const float bb = __fsub_rn(t, p);
    const float e2 = __fadd_rn(__fsub_rn(p, __fsub_rn(t, bb)), __fsub_rn(q1.z, bb));
    const float sz = __fmaf_rn(q1.x, dxh, t);
    h.zz = __fadd_rn(sz, __fmaf_rn(L.l1.y, dyh, __fmaf_rn(L.l1.x, dxh, __fadd_rn(__fadd_rn(e1, e2), L.l2.z))));
    return h;
}

// Record id of staged splat s (its grid row s_k minus the camera's block offset).
__device__ __forceinline__ int64_t staged_record(const CamDev &cam, int32_t s_k) {
    return int64_t(s_k) - cam.tex_row + cam.rec_off;
}

}  // namespace gbill
