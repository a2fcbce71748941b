// Preprocess (forward and backward) of the textured 2D-Gaussian rasterizer.
//
// Forward:
//   1. preprocess_kernel, one thread per splat looping over its cameras: FP32 tile
//      rectangle and depth key (culling and rectangles are FP32 decisions; the
//      operation sequence is fixed and contraction-free, so the (tile, depth)
//      key list is reproducible bit for bit), and the record's opacity and
//      view-dependent SH colour, added to the grid colour (Sec. 4.2).
//   2. record_kernel, one thread per visible record (after compaction): the
//      rest of the render record, the splat-to-screen homography of Eq. 3
//      composed with the pinhole camera, expressed relative to the projected
//      centre (so its upper-right block vanishes), its adjugate (ray/splat
//      intersection, u = zeta_x / zeta_z) and the centre as a double-float
//      pair.  Near edge-on splats (|det| tiny against its terms) redo the
//      homography and its inverse in FP64.
// Backward, one thread per splat: sums over the scene's cameras the chain from
// the record gradients back to means, quaternions, scales, opacity and SH.
#include <math.h>

#include "gbill_internal.cuh"
#include "sh.cuh"

namespace gbill {
namespace {

// ------------------------------------------------------------------ FP32 ops --
// Single-rounded IEEE operations that the compiler may not fuse or reorder.
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }

// FP32 culling, pixel rectangle and depth of one record.
__device__ bool key_rect(const float p[3], const float q[4], float su, float sv, float o,
                         const CamDev &c, float &z_out, int rect[4]) {
    const float qn2 = fa(fa(fa(fm(q[0], q[0]), fm(q[1], q[1])), fm(q[2], q[2])), fm(q[3], q[3]));
    if (!(qn2 > 0.0f)) return false;
    const float qinv = fdv(1.0f, __fsqrt_rn(qn2));
    const float w = fm(q[0], qinv), x = fm(q[1], qinv), y = fm(q[2], qinv), z = fm(q[3], qinv);
    const float tu0 = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
    const float tu1 = fm(2.0f, fa(fm(x, y), fm(w, z)));
    const float tu2 = fm(2.0f, fs(fm(x, z), fm(w, y)));
    const float tv0 = fm(2.0f, fs(fm(x, y), fm(w, z)));
    const float tv1 = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
    const float tv2 = fm(2.0f, fa(fm(y, z), fm(w, x)));
    const float a0 = fm(su, tu0), a1 = fm(su, tu1), a2 = fm(su, tu2);
    const float b0 = fm(sv, tv0), b1 = fm(sv, tv1), b2 = fm(sv, tv2);
    const float *R = c.R;
    const float A0 = fa(fa(fm(R[0], a0), fm(R[1], a1)), fm(R[2], a2));
    const float A1 = fa(fa(fm(R[3], a0), fm(R[4], a1)), fm(R[5], a2));
    const float A2 = fa(fa(fm(R[6], a0), fm(R[7], a1)), fm(R[8], a2));
    const float B0 = fa(fa(fm(R[0], b0), fm(R[1], b1)), fm(R[2], b2));
    const float B1 = fa(fa(fm(R[3], b0), fm(R[4], b1)), fm(R[5], b2));
    const float B2 = fa(fa(fm(R[6], b0), fm(R[7], b1)), fm(R[8], b2));
    const float P0 = fa(fa(fa(fm(R[0], p[0]), fm(R[1], p[1])), fm(R[2], p[2])), c.t[0]);
    const float P1 = fa(fa(fa(fm(R[3], p[0]), fm(R[4], p[1])), fm(R[5], p[2])), c.t[1]);
    const float P2 = fa(fa(fa(fm(R[6], p[0]), fm(R[7], p[1])), fm(R[8], p[2])), c.t[2]);
    if (!(P2 > c.near_plane)) return false;
    if (!(o >= kAlphaMin)) return false;
    const float xz = fdv(P0, P2), yz = fdv(P1, P2);
    const float t00 = fm(c.fx, fs(A0, fm(A2, xz))), t01 = fm(c.fx, fs(B0, fm(B2, xz)));
    const float t10 = fm(c.fy, fs(A1, fm(A2, yz))), t11 = fm(c.fy, fs(B1, fm(B2, yz)));
    const float t20 = A2, t21 = B2;
    const float d00 = fm(kRhoMax, fa(fm(t00, t00), fm(t01, t01)));
    const float d11 = fm(kRhoMax, fa(fm(t10, t10), fm(t11, t11)));
    const float d02 = fm(kRhoMax, fa(fm(t00, t20), fm(t01, t21)));
    const float d12 = fm(kRhoMax, fa(fm(t10, t20), fm(t11, t21)));
    const float d22 = fs(fm(kRhoMax, fa(fm(t20, t20), fm(t21, t21))), fm(P2, P2));
    if (!(d22 < 0.0f)) return false;
    const float nd = -d22;
    const float ox = fdv(d02, d22), oy = fdv(d12, d22);
    const float hx = fdv(__fsqrt_rn(fa(fm(d02, d02), fm(d00, nd))), nd);
    const float hy = fdv(__fsqrt_rn(fa(fm(d12, d12), fm(d11, nd))), nd);
    const float cx = fa(fm(c.fx, xz), c.cx), cy = fa(fm(c.fy, yz), c.cy);
    float elx = fs(fa(cx, ox), hx), ehx = fa(fa(cx, ox), hx);
    float ely = fs(fa(cy, oy), hy), ehy = fa(fa(cy, oy), hy);
    if (!(elx == elx) || !(ehx == ehx)) { elx = -INFINITY; ehx = INFINITY; }
    if (!(ely == ely) || !(ehy == ehy)) { ely = -INFINITY; ehy = INFINITY; }
    const float lox = fminf(elx, fs(cx, kLowPassRadius)), hix = fmaxf(ehx, fa(cx, kLowPassRadius));
    const float loy = fminf(ely, fs(cy, kLowPassRadius)), hiy = fmaxf(ehy, fa(cy, kLowPassRadius));
    const float fx0 = fmaxf(ceilf(fs(lox, 0.5f)), 0.0f);
    const float fx1 = fminf(floorf(fs(hix, 0.5f)), float(c.width - 1));
    const float fy0 = fmaxf(ceilf(fs(loy, 0.5f)), 0.0f);
    const float fy1 = fminf(floorf(fs(hiy, 0.5f)), float(c.height - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
    rect[0] = int(fx0);
    rect[1] = int(fy0);
    rect[2] = int(fx1);
    rect[3] = int(fy1);
    z_out = P2;
    return true;
}

// ------------------------------------------------------- double-float (FP32) --
// Error-free transformations: Knuth's two-sum, Dekker's fast two-sum and the
// FMA two-product; a double-float carries ~48 significant bits.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    DF p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF p = df_mul_f(b, q1);
    const DF r = df_add(a, DF{-p.hi, -p.lo});
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    DF p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_sqrt(DF a) {
    const float x = sqrtf(a.hi);
    const DF p = two_prod(x, x);
    const DF r = df_add(a, df_neg(p));
    return fast_two_sum(x, r.hi / (2.0f * x));
}
// 2 a in double-float (exact)
__device__ __forceinline__ DF df_twice(DF a) { return DF{2.0f * a.hi, 2.0f * a.lo}; }
// 1 - 2 a
__device__ __forceinline__ DF df_one_minus_twice(DF a) { return df_add(DF{1.0f, 0.0f}, df_neg(df_twice(a))); }
// dot of an FP32 row with a double-float vector
__device__ __forceinline__ DF df_dot_fd(const float *row, const DF v[3]) {
    DF acc = df_mul_f(v[0], row[0]);
    acc = df_add(acc, df_mul_f(v[1], row[1]));
    return df_add(acc, df_mul_f(v[2], row[2]));
}

// dot(row, p) + t in double-float
__device__ __forceinline__ DF df_affine(const float *row, const float p[3], float t) {
    DF acc = two_prod(row[0], p[0]);
    acc = df_add(acc, two_prod(row[1], p[1]));
    acc = df_add(acc, two_prod(row[2], p[2]));
    return df_add(acc, DF{t, 0.0f});
}

__device__ __forceinline__ float load_sh(const SceneDev &s, int64_t i) {
    switch (s.sh_dtype) {
        case GB_F16: return load_as_float(static_cast<const __half *>(s.sh), i);
        case GB_BF16: return load_as_float(static_cast<const __nv_bfloat16 *>(s.sh), i);
        default: return load_as_float(static_cast<const float *>(s.sh), i);
    }
}

// Calls fn(i, c) for the 48 SH coefficients c (index i = 3 m + channel) of
// splat k of a degree-3 scene, read with 128-bit loads: six for 16-bit
// storage, twelve for FP32.  Needs the array 16-byte aligned (sh_vec48).
// Scalar loads of a thread's coefficients, 96 or 192 bytes apart from its
// neighbours', touch 32 sectors per load instruction; the vector loads cut
// the L1 wavefronts of a warp's coefficient reads eightfold.
template <typename F>
__device__ __forceinline__ void for_each_sh48(const SceneDev &s, int64_t k, F &&fn) {
    if (s.sh_dtype == GB_F32) {
        const float4 *src = reinterpret_cast<const float4 *>(static_cast<const float *>(s.sh) + k * 48);
#pragma unroll
        for (int v = 0; v < 12; ++v) {
            const float4 w = src[v];
            fn(4 * v + 0, w.x); fn(4 * v + 1, w.y); fn(4 * v + 2, w.z); fn(4 * v + 3, w.w);
        }
    } else {
        const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const unsigned short *>(s.sh) + k * 48);
        const bool bf = s.sh_dtype == GB_BF16;
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            const uint4 w = src[v];
            const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                float lo, hi;
                if (bf) {
                    lo = __uint_as_float(u[h] << 16);
                    hi = __uint_as_float(u[h] & 0xffff0000u);
                } else {
                    const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&u[h]));
                    lo = t.x;
                    hi = t.y;
                }
                fn(8 * v + 2 * h, lo);
                fn(8 * v + 2 * h + 1, hi);
            }
        }
    }
}

// Whether for_each_sh48 serves the scene: degree 3 and a 16-byte aligned array.
__device__ __forceinline__ bool sh_vec48(const SceneDev &s) {
    return s.D == 3 && (reinterpret_cast<uintptr_t>(s.sh) & 15u) == 0;
}

// ------------------------------------------------------ rotation and frame --
struct Frame3 {
    float tu[3], tv[3];
    float qn[4];
    float qnorm;
};
__device__ __forceinline__ Frame3 tangent_frame(const float q[4]) {
    Frame3 f;
    f.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float inv = 1.0f / f.qnorm;
    for (int i = 0; i < 4; ++i) f.qn[i] = q[i] * inv;
    const float w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
    f.tu[0] = 1.0f - 2.0f * (y * y + z * z);
    f.tu[1] = 2.0f * (x * y + w * z);
    f.tu[2] = 2.0f * (x * z - w * y);
    f.tv[0] = 2.0f * (x * y - w * z);
    f.tv[1] = 1.0f - 2.0f * (x * x + z * z);
    f.tv[2] = 2.0f * (y * z + w * x);
    return f;
}

// Homography block in FP64 for splats seen at a grazing angle, where the
// determinant J = fx fy (n . P) / z of the block cancels: t = (t00, t01, t10,
// t11), m = (m20, m21, m22) = (fy n_x, fx n_y, fx fy n.P / z) / z, each as an
// FP32 pair hi + lo.
__device__ void homography_fp64(const float p[3], const float q[4], float su, float sv,
                                const CamDev &c, DF t[4], DF m[3]) {
    const double qn = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] +
                           (double)q[3] * q[3]);
    const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    const double tu[3] = {1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)};
    const double tv[3] = {2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)};
    double A[3], B[3], P[3], n[3];
    for (int i = 0; i < 3; ++i) {
        const float *r = c.R + 3 * i;
        A[i] = su * ((double)r[0] * tu[0] + (double)r[1] * tu[1] + (double)r[2] * tu[2]);
        B[i] = sv * ((double)r[0] * tv[0] + (double)r[1] * tv[1] + (double)r[2] * tv[2]);
        P[i] = (double)r[0] * p[0] + (double)r[1] * p[1] + (double)r[2] * p[2] + (double)c.t[i];
    }
    // the homography's normal A x B (not s_u s_v R t_w: the camera's FP32 R is
    // orthonormal only to ~1e-8, which a grazing view's n . P would magnify)
    n[0] = A[1] * B[2] - A[2] * B[1];
    n[1] = A[2] * B[0] - A[0] * B[2];
    n[2] = A[0] * B[1] - A[1] * B[0];
    const double iz = 1.0 / P[2], xz = P[0] * iz, yz = P[1] * iz;
    const double tv_[4] = {c.fx * (A[0] - A[2] * xz), c.fx * (B[0] - B[2] * xz), c.fy * (A[1] - A[2] * yz),
                           c.fy * (B[1] - B[2] * yz)};
    const double mv[3] = {c.fy * n[0] * iz, c.fx * n[1] * iz,
                          (double)c.fx * c.fy * (n[0] * P[0] + n[1] * P[1] + n[2] * P[2]) * iz * iz};
    for (int i = 0; i < 4; ++i) {
        t[i].hi = (float)tv_[i];
        t[i].lo = (float)(tv_[i] - (double)t[i].hi);
    }
    for (int i = 0; i < 3; ++i) {
        m[i].hi = (float)mv[i];
        m[i].lo = (float)(mv[i] - (double)m[i].hi);
    }
}

// Conditioning bound of the FP32 plane-hit evaluation about the centre (the
// flag threshold kPreciseKappa).  Over the disk u^2 + v^2 <= r^2 (r^2 = 2 ln
// 255, beyond which alpha < 1/255) the pixel offset is d = T2 (u, v) / w, w =
// t20 u + t21 v + z the hit depth, and zeta_z = J / w (J = t00 t11 - t01 t10
// = m22 z).  The terms summed into zeta_x = t11 d_x - t01 d_y are at most
// (|t11| |row 0| + |t01| |row 1|) r / w, so relative to |zeta_z| the factor w
// cancels; the terms of zeta_z times |u| <= r add r ((|m20| |row 0| + |m21|
// |row 1|) r / |J| + w_max / z).  The bound is the screen-space anisotropy of
// the splat (large for a thin splat seen along its long axis) plus the
// grazing-angle cancellation of zeta_z.
__device__ __forceinline__ float plane_hit_kappa(float t00, float t01, float t10, float t11, float t20, float t21,
                                                 float m20, float m21, float m22, float z) {
    const float r = kLowPassRadius * 1.41421356f;  // sqrt(2 ln 255)
    const float n0 = sqrtf(t00 * t00 + t01 * t01), n1 = sqrtf(t10 * t10 + t11 * t11);
    const float aJ = fabsf(m22) * z;
    const float ku = fmaxf(fabsf(t11) * n0 + fabsf(t01) * n1, fabsf(t10) * n0 + fabsf(t00) * n1);
    const float kz = (fabsf(m20) * n0 + fabsf(m21) * n1) * r;
    const float wmax = z + r * sqrtf(t20 * t20 + t21 * t21);
    const float k = r * (ku + kz) / aJ + r * wmax / z;
    return k == k ? k : INFINITY;  // J = 0: unbounded
}

// --------------------------------------------------------- forward kernel --
// One thread per splat of scene blockIdx.y, looping over the scene's cameras:
// the splat's parameters are read once for all its records (coalesced; the
// SH coefficients stay in L1 across the loop), and each camera's records are
// written coalesced at rec_off + k.
__global__ void __launch_bounds__(256, 4) preprocess_kernel(Frame f, uint32_t *depth_key,
                                                         uint32_t *rec_id, uint2 *rect_out, uint2 *pbox,
                                                         Record *rec_out, Counters *cnt) {
    const int si = blockIdx.y;
    const SceneDev &sc = f.scenes[si];
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool live = k < sc.K;
    float p[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0}, su = 0.0f, sv = 0.0f, o = 0.0f;
    bool finite = false;
    if (live) {
        for (int i = 0; i < 3; ++i) p[i] = sc.means[3 * k + i];
        for (int i = 0; i < 4; ++i) q[i] = sc.quats[4 * k + i];
        su = sc.scales[2 * k];
        sv = sc.scales[2 * k + 1];
        o = sc.opac[k];
        // a splat with a non-finite parameter is culled in every camera and
        // raises error bit 1 (gb_saved_check: GB_ERR_NONFINITE)
        finite = isfinite(su) && isfinite(sv) && isfinite(o);
        for (int i = 0; i < 3; ++i) finite = finite && isfinite(p[i]);
        for (int i = 0; i < 4; ++i) finite = finite && isfinite(q[i]);
        if (!finite) atomicOr(&cnt->error_flags, 2u);
    }
    const int M = (sc.D + 1) * (sc.D + 1);
    for (int ci = 0; ci < f.n_cams; ++ci) {
        const CamDev &cam = f.cams[ci];
        if (cam.scene != si) continue;  // uniform over the block
        const int64_t r = cam.rec_off + k;
        float zkey;
        int pr[4];
        bool valid = finite && key_rect(p, q, su, sv, o, cam, zkey, pr);
        // SH colour, d = (p - campos) / |p - campos|; all 16 basis values
        // (registers), coefficients beyond the scene's degree skipped by a
        // uniform predicate.  Non-finite coefficients cull the record too.
        float rgb[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            float dx = p[0] - cam.campos[0], dy = p[1] - cam.campos[1], dz = p[2] - cam.campos[2];
            const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= dn; dy *= dn; dz *= dn;
            float Y[16];
            sh_basis(3, dx, dy, dz, Y);
            if (sh_vec48(sc)) {
                for_each_sh48(sc, k, [&](int i, float c) { rgb[i % 3] = fmaf(Y[i / 3], c, rgb[i % 3]); });
            } else {
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    if (m < M)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) rgb[ch] += Y[m] * load_sh(sc, (k * M + m) * 3 + ch);
            }
            if (!(isfinite(rgb[0]) && isfinite(rgb[1]) && isfinite(rgb[2]))) {
                atomicOr(&cnt->error_flags, 2u);
                valid = false;
            }
        }
        if (live) {
            if (rec_id) rec_id[r] = uint32_t(r);  // identity values for a sort of every record
            if (!valid) {
                depth_key[r] = 0xFFFFFFFFu;
                rect_out[r] = make_uint2(0u, 0u);
            } else {
                depth_key[r] = __float_as_uint(zkey);
                const int T = f.tile;
                rect_out[r] = make_uint2(uint32_t(pr[0] / T) | (uint32_t(pr[1] / T) << 16),
                                         uint32_t(pr[2] / T) | (uint32_t(pr[3] / T) << 16));
                pbox[r] = make_uint2(uint32_t(pr[0]) | (uint32_t(pr[1]) << 16),
                                     uint32_t(pr[2]) | (uint32_t(pr[3]) << 16));
                // the render record's opacity and SH colour; its homography part
                // (q0..q2) is built by record_kernel for the visible records only
                rec_out[r].q3 = make_float4(o, rgb[0], rgb[1], rgb[2]);
            }
        }
        // warp-aggregated visible count
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if ((threadIdx.x & 31) == 0 && m) atomicAdd(&cnt->n_visible, uint32_t(__popc(m)));
    }
}

// ------------------------------------------------------- record kernel --
// The homography part of the render record (q0..q2) of record r: the whole
// record chain in double-float (~48 bits): unit quaternion, tangent frame,
// camera-space axes A = s_u R t_u, B = s_v R t_v, normal n = A x B, centre P, centre-relative block t and m = (fy n_x, fx n_y, fx fy n.P
// / z) / z.  Only n.P cancels (grazing view); below cos = 1/256 the block is
// redone in FP64.  A record whose conditioning bound passes kPreciseKappa is
// flagged (depth stored negated) and gets its low parts in rec_lo.
__device__ __forceinline__ void record_homography(const Frame &f, int64_t r, Record *rec_out, RecordLo *lo_out) {
    const int ci = camera_of_record(f, r);
    const CamDev &cam = f.cams[ci];
    const SceneDev &sc = f.scenes[cam.scene];
    const int64_t k = r - cam.rec_off;
    float p[3], q[4];
    for (int i = 0; i < 3; ++i) p[i] = sc.means[3 * k + i];
    for (int i = 0; i < 4; ++i) q[i] = sc.quats[4 * k + i];
    const float su = sc.scales[2 * k], sv = sc.scales[2 * k + 1];
    DF qn2 = two_prod(q[0], q[0]);
    for (int i = 1; i < 4; ++i) qn2 = df_add(qn2, two_prod(q[i], q[i]));
    const DF qinv = df_div(DF{1.0f, 0.0f}, df_sqrt(qn2));
    const DF w = df_mul_f(qinv, q[0]), x = df_mul_f(qinv, q[1]), y = df_mul_f(qinv, q[2]),
             zq = df_mul_f(qinv, q[3]);
    const DF xx = df_mul(x, x), yy = df_mul(y, y), zz = df_mul(zq, zq), xy = df_mul(x, y), xzq = df_mul(x, zq),
             yzq = df_mul(y, zq), wx = df_mul(w, x), wy = df_mul(w, y), wz = df_mul(w, zq);
    const DF tu[3] = {df_one_minus_twice(df_add(yy, zz)), df_twice(df_add(xy, wz)), df_twice(df_sub(xzq, wy))};
    const DF tv[3] = {df_twice(df_sub(xy, wz)), df_one_minus_twice(df_add(xx, zz)), df_twice(df_add(yzq, wx))};
    DF A[3], B[3];
    for (int i = 0; i < 3; ++i) {
        const float *row = cam.R + 3 * i;
        A[i] = df_mul_f(df_dot_fd(row, tu), su);
        B[i] = df_mul_f(df_dot_fd(row, tv), sv);
    }
    // normal of the homography, A x B (the camera's FP32 R is orthonormal only
    // to ~1e-8, so s_u s_v R t_w would differ by that, magnified in a grazing n . P)
    const DF nv[3] = {df_sub(df_mul(A[1], B[2]), df_mul(A[2], B[1])), df_sub(df_mul(A[2], B[0]), df_mul(A[0], B[2])),
                      df_sub(df_mul(A[0], B[1]), df_mul(A[1], B[0]))};
    const DF Px = df_affine(cam.R + 0, p, cam.t[0]);
    const DF Py = df_affine(cam.R + 3, p, cam.t[1]);
    const DF Pz = df_affine(cam.R + 6, p, cam.t[2]);
    const DF xz = df_div(Px, Pz), yz = df_div(Py, Pz);
    const DF cxd = df_add(df_mul_f(xz, cam.fx), DF{cam.cx, 0.0f});
    const DF cyd = df_add(df_mul_f(yz, cam.fy), DF{cam.cy, 0.0f});
    const float z = Pz.hi;
    DF np = df_mul(nv[0], Px);
    np = df_add(np, df_mul(nv[1], Py));
    np = df_add(np, df_mul(nv[2], Pz));
    const float nmag = fabsf(nv[0].hi * Px.hi) + fabsf(nv[1].hi * Py.hi) + fabsf(nv[2].hi * Pz.hi);
    DF t[4], m[3];  // t00, t01, t10, t11; m20, m21, m22
    if (fabsf(np.hi) * 256.0f > nmag) {
        t[0] = df_mul_f(df_sub(A[0], df_mul(A[2], xz)), cam.fx);
        t[1] = df_mul_f(df_sub(B[0], df_mul(B[2], xz)), cam.fx);
        t[2] = df_mul_f(df_sub(A[1], df_mul(A[2], yz)), cam.fy);
        t[3] = df_mul_f(df_sub(B[1], df_mul(B[2], yz)), cam.fy);
        m[0] = df_div(df_mul_f(nv[0], cam.fy), Pz);
        m[1] = df_div(df_mul_f(nv[1], cam.fx), Pz);
        m[2] = df_div(df_div(df_mul(np, two_prod(cam.fx, cam.fy)), Pz), Pz);
    } else {
        homography_fp64(p, q, su, sv, cam, t, m);
    }
    // centre: c_hi on the 1/512-pixel grid (exact offsets x + 0.5 - c_hi), c_lo the rest
    const float chx = rintf(cxd.hi * 512.0f) * (1.0f / 512.0f), chy = rintf(cyd.hi * 512.0f) * (1.0f / 512.0f);
    const float clx = __fadd_rn(__fsub_rn(cxd.hi, chx), cxd.lo), cly = __fadd_rn(__fsub_rn(cyd.hi, chy), cyd.lo);
    const float kap = plane_hit_kappa(t[0].hi, t[1].hi, t[2].hi, t[3].hi, A[2].hi, B[2].hi, m[0].hi, m[1].hi, m[2].hi,
                                      z);
    const bool precise = !(kap <= kPreciseKappa);
    Record &R = rec_out[r];
    R.q0 = make_float4(t[3].hi, -t[1].hi, -t[2].hi, t[0].hi);
    R.q1 = make_float4(m[0].hi, m[1].hi, m[2].hi, precise ? -z : z);
    R.q2 = make_float4(chx, chy, clx, cly);
    if (precise) {
        RecordLo &L = lo_out[r];
        L.l0 = make_float4(t[3].lo, -t[1].lo, -t[2].lo, t[0].lo);
        L.l1 = make_float4(m[0].lo, m[1].lo, 0.0f, 0.0f);
        L.l2 = make_float4(-fmaf(t[3].hi, clx, -t[1].hi * cly), -fmaf(-t[2].hi, clx, t[0].hi * cly),
                           m[2].lo - fmaf(m[0].hi, clx, m[1].hi * cly), 0.0f);
    }
}

// One thread per visible record: ids[j] for j < *n_dev (the compacted visible
// records), or, without ids, every record whose depth key is not the culled
// marker.
__global__ void __launch_bounds__(128) record_kernel(Frame f, const uint32_t *ids, const uint32_t *n_dev,
                                                     const uint32_t *depth_key, int64_t max_n, Record *rec_out,
                                                     RecordLo *lo_out) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t n = n_dev ? min(int64_t(*n_dev), max_n) : max_n;
    if (j >= n) return;
    const int64_t r = ids ? int64_t(ids[j]) : j;
    if (!ids && depth_key[r] == 0xFFFFFFFFu) return;
    record_homography(f, r, rec_out, lo_out);
}

// -------------------------------------------------------- backward kernel --
__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// One thread per splat of scene `si`, summing its cameras: the record
// gradient (kRecGrad layout) of each camera through dL/dN = -N^-T H, N = [A B
// P] (N^-1 has rows (B x P, P x A, A x B) / det N), to the centre (plus the
// low-pass projection and depth terms), the scales (-H00 / s_u, -H11 / s_v)
// and a torque A x dL/dA + B x dL/dB of the splat frame, which becomes the
// quaternion gradient 2 (0, tau) q / |q| once summed.  The SH degree D is a
// template parameter so that the per-coefficient accumulators and the basis
// stay in registers.
template <int D>
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(Frame f, int si, const float *rec_grad,
                                                             const int32_t *inv_perm) {
    const SceneDev &sc = f.scenes[si];
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= sc.K) return;
    float p[3], q[4];
    for (int i = 0; i < 3; ++i) p[i] = sc.means[3 * k + i];
    for (int i = 0; i < 4; ++i) q[i] = sc.quats[4 * k + i];
    const float su = sc.scales[2 * k], sv = sc.scales[2 * k + 1];
    const Frame3 fr = tangent_frame(q);
    constexpr int M = (D + 1) * (D + 1);
    float g_p[3] = {0, 0, 0}, g_tau[3] = {0, 0, 0};
    float g_su = 0.0f, g_sv = 0.0f, g_o = 0.0f;
    float g_sh[M][3];
#pragma unroll
    for (int m = 0; m < M; ++m) g_sh[m][0] = g_sh[m][1] = g_sh[m][2] = 0.0f;
    bool seen = false;  // visible in some camera (else every gradient is zero, whatever the parameters)
    for (int ci = 0; ci < f.n_cams; ++ci) {
        const CamDev &cam = f.cams[ci];
        if (cam.scene != si) continue;
        const int32_t j = inv_perm[cam.rec_off + k];
        if (j < 0) continue;
        seen = true;
        float g[kRecGrad];
        const float4 *gp = reinterpret_cast<const float4 *>(rec_grad + int64_t(j) * kRecGrad);
#pragma unroll
        for (int i = 0; i < kRecGrad / 4; ++i) {
            const float4 v = gp[i];
            g[4 * i] = v.x; g[4 * i + 1] = v.y; g[4 * i + 2] = v.z; g[4 * i + 3] = v.w;
        }
        // camera-space frame N = [A B P]
        float A[3], B[3], P[3];
        for (int i = 0; i < 3; ++i) {
            const float *row = cam.R + 3 * i;
            A[i] = su * (row[0] * fr.tu[0] + row[1] * fr.tu[1] + row[2] * fr.tu[2]);
            B[i] = sv * (row[0] * fr.tv[0] + row[1] * fr.tv[1] + row[2] * fr.tv[2]);
            P[i] = row[0] * p[0] + row[1] * p[1] + row[2] * p[2] + cam.t[i];
        }
        float n0[3], n1[3], n2[3];
        cross3(B, P, n0);
        cross3(P, A, n1);
        cross3(A, B, n2);
        const float det = A[0] * n0[0] + A[1] * n0[1] + A[2] * n0[2];
        // det = 0: the plane holds the camera centre, every pair was skipped (H = 0)
        const float idet = det != 0.0f ? 1.0f / det : 0.0f;
        // dL/dA, dL/dB, dL/dP: columns of -N^-T H
        float gN[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                gN[c][i] = -(g[kGH + c] * n0[i] + g[kGH + 3 + c] * n1[i] + g[kGH + 6 + c] * n2[i]) * idet;
        // low-pass branch: centre c = (fx P0 / P2 + cx, fy P1 / P2 + cy); depth P2
        const float iz = 1.0f / P[2];
        const float gcx = g[kGCentreLP] * cam.fx * iz, gcy = g[kGCentreLP + 1] * cam.fy * iz;
        gN[2][0] += gcx;
        gN[2][1] += gcy;
        gN[2][2] += g[kGDepthLP] - (gcx * P[0] + gcy * P[1]) * iz;
        g_su -= g[kGH + 0] / su;
        g_sv -= g[kGH + 4] / sv;
        float ta[3], tb[3];
        cross3(A, gN[0], ta);
        cross3(B, gN[1], tb);
        // back to world space (R^T)
        for (int i = 0; i < 3; ++i) {
            const float r0 = cam.R[i], r1 = cam.R[3 + i], r2 = cam.R[6 + i];
            g_p[i] += r0 * gN[2][0] + r1 * gN[2][1] + r2 * gN[2][2];
            g_tau[i] += r0 * (ta[0] + tb[0]) + r1 * (ta[1] + tb[1]) + r2 * (ta[2] + tb[2]);
        }
        g_o += g[kGOpacity];
        // SH colour
        const float grgb[3] = {g[kGRgb], g[kGRgb + 1], g[kGRgb + 2]};
        float d[3] = {p[0] - cam.campos[0], p[1] - cam.campos[1], p[2] - cam.campos[2]};
        const float dist = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) d[i] /= dist;
        float Y[16], Gs[16][3];
        sh_basis(D, d[0], d[1], d[2], Y);
        sh_basis_grad(D, d[0], d[1], d[2], Gs);
        float gd[3] = {0, 0, 0};
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) g_sh[m][ch] += Y[m] * grgb[ch];
        auto sh_dir = [&](int i, float c) {
            const int m = i / 3, ch = i - 3 * m;
            const float kc = c * grgb[ch];
            gd[0] += kc * Gs[m][0];
            gd[1] += kc * Gs[m][1];
            gd[2] += kc * Gs[m][2];
        };
        if (D == 3 && sh_vec48(sc)) {
            for_each_sh48(sc, k, sh_dir);
        } else {
#pragma unroll
            for (int i = 0; i < 3 * M; ++i) sh_dir(i, load_sh(sc, k * 3 * M + i));
        }
        const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
        for (int i = 0; i < 3; ++i) g_p[i] += (gd[i] - d[i] * dd) / dist;
    }
    if (!seen) {
        // culled everywhere (possibly for non-finite parameters): exact zeros
        if (sc.g_means) for (int i = 0; i < 3; ++i) sc.g_means[3 * k + i] = 0.0f;
        if (sc.g_quats) for (int i = 0; i < 4; ++i) sc.g_quats[4 * k + i] = 0.0f;
        if (sc.g_scales) { sc.g_scales[2 * k] = 0.0f; sc.g_scales[2 * k + 1] = 0.0f; }
        if (sc.g_opac) sc.g_opac[k] = 0.0f;
        if (sc.g_sh)
            for (int m = 0; m < M; ++m)
                for (int ch = 0; ch < 3; ++ch) sc.g_sh[(k * M + m) * 3 + ch] = 0.0f;
        return;
    }
    if (sc.g_means)
        for (int i = 0; i < 3; ++i) sc.g_means[3 * k + i] = g_p[i];
    if (sc.g_quats) {
        // a world rotation delta turns q into (1, delta / 2) q: the gradient of the unit
        // quaternion is 2 (0, tau) q (tangent to the sphere), divided by |q| for the raw one
        const float w = fr.qn[0], x = fr.qn[1], y = fr.qn[2], z = fr.qn[3];
        const float s2 = 2.0f / fr.qnorm;
        sc.g_quats[4 * k + 0] = -s2 * (g_tau[0] * x + g_tau[1] * y + g_tau[2] * z);
        sc.g_quats[4 * k + 1] = s2 * (w * g_tau[0] + g_tau[1] * z - g_tau[2] * y);
        sc.g_quats[4 * k + 2] = s2 * (w * g_tau[1] + g_tau[2] * x - g_tau[0] * z);
        sc.g_quats[4 * k + 3] = s2 * (w * g_tau[2] + g_tau[0] * y - g_tau[1] * x);
    }
    if (sc.g_scales) { sc.g_scales[2 * k] = g_su; sc.g_scales[2 * k + 1] = g_sv; }
    if (sc.g_opac) sc.g_opac[k] = g_o;
    if (sc.g_sh) {
        if (D == 3 && (reinterpret_cast<uintptr_t>(sc.g_sh) & 15u) == 0) {
            // 48 values, 192 bytes: twelve 128-bit stores (scalar stores 192 bytes
            // apart from the neighbouring threads' touch 32 sectors each)
            float4 *dst = reinterpret_cast<float4 *>(sc.g_sh + k * 48);
#pragma unroll
            for (int v = 0; v < 12; ++v) {
                const int i = 4 * v;
                dst[v] = make_float4(g_sh[i / 3][i % 3], g_sh[(i + 1) / 3][(i + 1) % 3], g_sh[(i + 2) / 3][(i + 2) % 3],
                                     g_sh[(i + 3) / 3][(i + 3) % 3]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) sc.g_sh[(k * M + m) * 3 + ch] = g_sh[m][ch];
        }
    }
}

}  // namespace

cudaError_t launch_preprocess(const Frame &f, int64_t max_k, uint32_t *depth_key, uint32_t *rec_id,
                              uint2 *rect, uint2 *pbox, Record *rec, Counters *cnt, cudaStream_t s) {
    if (max_k <= 0) return cudaSuccess;
    dim3 grid(unsigned(ceil_div(max_k, 256)), unsigned(f.n_scenes));
    preprocess_kernel<<<grid, 256, 0, s>>>(f, depth_key, rec_id, rect, pbox, rec, cnt);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_record(const Frame &f, const uint32_t *ids, const uint32_t *n_dev, const uint32_t *depth_key,
                          int64_t max_n, Record *rec, RecordLo *rec_lo, cudaStream_t s) {
    if (max_n <= 0) return cudaSuccess;
    record_kernel<<<unsigned(ceil_div(max_n, 128)), 128, 0, s>>>(f, ids, n_dev, depth_key, max_n, rec, rec_lo);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const Frame &f, int64_t max_k, const float *rec_grad,
                                  const int32_t *inv_perm, cudaStream_t s) {
    if (max_k <= 0) return cudaSuccess;
    for (int si = 0; si < f.n_scenes; ++si) {
        const int64_t K = f.scenes[si].K;
        if (K <= 0) continue;
        const unsigned grid = unsigned(ceil_div(K, 128));
        switch (f.scenes[si].D) {
            case 0: preprocess_bwd_kernel<0><<<grid, 128, 0, s>>>(f, si, rec_grad, inv_perm); break;
            case 1: preprocess_bwd_kernel<1><<<grid, 128, 0, s>>>(f, si, rec_grad, inv_perm); break;
            case 2: preprocess_bwd_kernel<2><<<grid, 128, 0, s>>>(f, si, rec_grad, inv_perm); break;
            default: preprocess_bwd_kernel<3><<<grid, 128, 0, s>>>(f, si, rec_grad, inv_perm); break;
        }
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbill
