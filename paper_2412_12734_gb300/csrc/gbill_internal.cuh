// Internal declarations of the sm_103a rasterizer library.  Nothing here is
// part of the C ABI (include/gbill.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbill.h"

namespace gbill {

constexpr int kMaxCams = GBILL_MAX_CAMERAS;
constexpr int kMaxScenes = GBILL_MAX_SCENES;
constexpr int kMaxGroups = 32;  // distinct (texture size, storage type, per-splat size) of a frame (5 x 3 x 2)

// Constants of the method (Sec. 3.1 Eq. 4 with the 3DGS-lineage clamp and
// cutoffs; the screen-space low-pass of the 2DGS lineage).
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip a splat below this alpha
constexpr float kAlphaMax = 0.99f;          // alpha clamp
constexpr float kTMin = 1e-4f;              // stop before T would drop below
constexpr float kLowPass = 2.0f;            // rho_lp = 2 |x - c|^2 (sigma_lp = sqrt(2)/2 px)
// 2 ln 255: u^2 + v^2 beyond this gives alpha < 1/255 for any o <= 1.
constexpr float kRhoMax = 11.0825270903f;
// sqrt(ln 255): radius of the low-pass disk where 2 r^2 = rho_max.
constexpr float kLowPassRadius = 2.35398885833f;

// Per-camera data, derived on the host from gb_camera.
struct CamDev {
    int32_t width, height, tiles_x, tiles_y;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float campos[3];
    float near_plane;
    int32_t scene;
    int32_t group;      // render group: cameras whose scenes share (tex_n, tex_dtype)
    uint32_t tile_off;  // first global tile id of this camera
    int64_t pix_off;    // first pixel of this camera in the packed outputs
    int64_t rec_off;    // first record (= tile_off-like offset over splats)
    int64_t tex_row;    // grid row of splat k is tex_row + k: 0, or for per-texel SH
                        // scenes the camera's block of evaluated grids
};

struct SceneDev {
    int64_t K;
    const float *means, *quats, *scales, *opac;
    const void *sh;
    const void *tex;
    int32_t D, sh_dtype, N, tex_dtype;  // N, tex: the grid the render reads
    float sigma;
    int32_t mip;                        // mip level (the render reads the filtered grid)
    int32_t tex_sh;                     // per-texel SH degree (the render reads evaluated grids)
    int32_t pad2;
    const uint8_t *splat_n;             // per-splat grid size (null: every splat N)
    float *g_means, *g_quats, *g_scales, *g_opac, *g_sh, *g_tex;
};

// Everything a launch needs about the frame, passed BY VALUE as a kernel
// parameter (no host->device copy, safe under graph capture).
struct Frame {
    int32_t n_cams, n_scenes, tile, flags;
    int64_t n_records;
    int64_t n_pixels;
    uint32_t n_tiles;
    int32_t n_groups;
    float bg[3];
    float pad2;
    int32_t group_N[kMaxGroups], group_dtype[kMaxGroups];
    int32_t group_var[kMaxGroups];  // 1: the group's scenes carry per-splat grid sizes
    uint32_t group_off[kMaxGroups], group_count[kMaxGroups];  // segments of the tile list
    CamDev cams[kMaxCams];
    SceneDev scenes[kMaxScenes];
};

// A projected (splat, camera) record, 64 bytes, written by preprocess and
// read by both render passes.  With the projected centre c moved to the
// origin the splat-to-screen homography T' is lower block triangular:
//   T' = [[t00 t01 0], [t10 t11 0], [t20 t21 t22]],   t22 = centre depth z.
// zeta = adj(T') (dx, dy, 1) / t22 gives the ray/plane hit u = zeta_x/zeta_z,
// v = zeta_y/zeta_z for the pixel offset (dx, dy) = x - c, and the hit depth
// J / zeta_z with J = t00 t11 - t01 t10 = m22 z.
//   q0 = ( t11, -t01, -t10,  t00)           zeta_xy = [[q0.x q0.y][q0.z q0.w]] (dx,dy)
//   q1 = ( m20,  m21,  m22,  z  )           zeta_z  = m20 dx + m21 dy + m22
//   q2 = ( c_hi.x, c_hi.y, c_lo.x, c_lo.y ) c = c_hi + c_lo (double-float centre)
//   q3 = ( o, r_sh, g_sh, b_sh )            opacity and SH colour
//
// The centre is split so that c_hi lies on a 1/512-pixel grid: x + 0.5 - c_hi
// is then exact for |x - c_hi| < 2^15, and c_lo = c - c_hi (|c_lo| <= 2^-10).
// A record whose plane-hit evaluation is ill-conditioned (a thin splat seen
// along its long axis, or one seen at a grazing angle: see kPreciseKappa)
// stores its depth negated (q1.w = -z) and takes the extended-precision
// evaluation of render_common.cuh with its RecordLo.
struct __align__(16) Record {
    float4 q0, q1, q2, q3;
};

// Low parts of a flagged record (48 bytes, indexed like Record): the FP32
// residues of the homography entries, hi + lo = the double-float value, and
// the products of the hi entries with the centre's low part, so that for a
// pixel offset dh = x + 0.5 - c_hi (exact) the plane hit is
//   zeta_x = q0.x dh_x + q0.y dh_y + (l0.x dh_x + l0.y dh_y) + l2.x
//   zeta_y = q0.z dh_x + q0.w dh_y + (l0.z dh_x + l0.w dh_y) + l2.y
//   zeta_z = q1.x dh_x + q1.y dh_y + q1.z + (l1.x dh_x + l1.y dh_y) + l2.z
// up to the dropped lo x lo products.
//   l0 = lo of (t11, -t01, -t10, t00)
//   l1 = (lo m20, lo m21, 0, 0)
//   l2 = (-(q0.x c_lo.x + q0.y c_lo.y), -(q0.z c_lo.x + q0.w c_lo.y),
//         lo m22 - (q1.x c_lo.x + q1.y c_lo.y), 0)
struct __align__(16) RecordLo {
    float4 l0, l1, l2;
};

// A record is flagged for the extended-precision evaluation when its
// conditioning bound exceeds this: kappa bounds, over the part of the
// footprint where the plane hit decides alpha (u^2 + v^2 <= 2 ln 255), the
// ratio of the magnitudes of the terms summed into zeta (times |u|, |v| for
// zeta_z) to |zeta_z|, so an FP32 evaluation about the centre has an error of
// about kappa 2^-24 in u and v.  Below 32 that is < 2e-6.
constexpr float kPreciseKappa = 32.0f;

// Gradient of one record, accumulated by the backward render in the splat's
// own (u, v) frame.  With N = [A | B | P] the camera-space splat frame (A =
// s_u R t_u, B = s_v R t_v, P the centre; Eq. 3 up to the intrinsics K), a
// pixel's plane hit (u, v) solves K N (u, v, 1) ~ (x, y, 1), and for any
// change of the parameters
//   du = -e0 + u e2,  dv = -e1 + v e2,  dw = w e2,   e = N^-1 dN (u, v, 1)
// (w the hit depth).  So the plane-hit part of the gradient is
//   dL/dN = -N^-T H,   H = sum over pairs (u^, v^, W) (x) (u, v, 1),
// W = -(u^ u + v^ v) - w^ w, w^ the depth adjoint of a plane-hit pair: nine
// sums of O(1) multiples of the adjoints (|u|, |v| <= 3.33 where alpha >=
// 1/255), without the cancellation that gradients of the homography entries
// about the centre carry for a thin splat seen along its long axis (there the
// entries' gradients are sums of terms |d| times larger that cancel in the
// parameter chain).  The scale gradients are then -H00 / s_u and -H11 / s_v.
// Slots (16 floats, 4 float4):
//   0..8   H row-major (u^ u, u^ v, u^, v^ u, v^ v, v^, W u, W v, W)
//   9, 10  d c from the screen-space low-pass branch
//   11     sum of the depth adjoints of low-pass pairs (depth = centre z)
//   12     d o;  13..15  d rgb (SH colour)
constexpr int kRecGrad = 16;
constexpr int kGH = 0, kGCentreLP = 9, kGDepthLP = 11, kGOpacity = 12, kGRgb = 13;
constexpr int kRecVals = 16;  // slots the backward render fills

// Device-side counters of one forward.
struct Counters {
    uint32_t n_visible;    // records surviving culling
    uint32_t n_instances;  // (tile, splat) pairs
    uint32_t overflow;     // capacity exceeded
    uint32_t error_flags;  // bit 0: bounded wait timed out; bit 1: non-finite splat culled
    uint32_t work_next;    // persistent render work counter (forward)
    uint32_t work_next_bwd;
    uint32_t pad[2];
    unsigned long long pairs_fwd;    // (pixel, splat) pairs evaluated by render fwd
    unsigned long long pairs_bwd;    // ... and by render bwd
    unsigned long long blend_fwd;    // pairs blended by render fwd
};

// Host-side count of kernels launched by the library (see gb_kernel_launches).
void count_launches(int n);

// ---------------------------------------------------------------- helpers --

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename T>
__device__ __forceinline__ float load_as_float(const T *p, int64_t i);
template <>
__device__ __forceinline__ float load_as_float<float>(const float *p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float load_as_float<__half>(const __half *p, int64_t i) {
    return __half2float(p[i]);
}
template <>
__device__ __forceinline__ float load_as_float<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t i) {
    return __bfloat162float(p[i]);
}

// Binary search of the camera owning global tile id `tile`.
__device__ __forceinline__ int camera_of_tile(const Frame &f, uint32_t tile) {
    int lo = 0, hi = f.n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (f.cams[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Camera of record r (records are camera-major: camera c owns [rec_off, rec_off + K)).
__device__ __forceinline__ int camera_of_record(const Frame &f, int64_t r) {
    int lo = 0, hi = f.n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (f.cams[mid].rec_off <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------- host-side launchers --

// preprocess.cu: culling, key, rectangle, SH colour per record (rec_id, if
// not NULL, receives the identity for a sort of every record)
cudaError_t launch_preprocess(const Frame &f, int64_t max_k, uint32_t *depth_key, uint32_t *rec_id,
                              uint2 *rect, uint2 *pbox, Record *rec, Counters *cnt, cudaStream_t s);
// Homography part (q0..q2) of the render records: of ids[0 .. *n_dev) or,
// with ids NULL, of every record whose depth key is not the culled marker.
cudaError_t launch_record(const Frame &f, const uint32_t *ids, const uint32_t *n_dev, const uint32_t *depth_key,
                          int64_t max_n, Record *rec, RecordLo *rec_lo, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const Frame &f, int64_t max_k, const float *rec_grad,
                                  const int32_t *inv_perm, cudaStream_t s);

// sort.cu
size_t radix_scratch_bytes(int64_t n);
// Visible records (depth key not 0xFFFFFFFF) of [0, n) to the front of
// key_out / id_out in record order (id = record index); pos: n scan slots.
cudaError_t compact_visible(const uint32_t *depth_key, int64_t n, uint32_t *pos, uint32_t *key_out,
                            uint32_t *id_out, void *scratch, size_t scratch_bytes, cudaStream_t s);
cudaError_t radix_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_tmp,
                             uint32_t *vals_tmp, uint32_t *keys_out, uint32_t *vals_out,
                             int64_t max_n, const uint32_t *n_dev, int begin_bit, int end_bit,
                             void *scratch, size_t scratch_bytes, cudaStream_t s);
size_t scan_scratch_bytes(int64_t n);
cudaError_t tile_counts_scan(const Frame &f, const uint32_t *perm, const uint2 *rect, int64_t max_n,
                             const uint32_t *n_dev, uint32_t *offsets, void *scratch,
                             size_t scratch_bytes, Counters *cnt, int64_t capacity, cudaStream_t s);
cudaError_t launch_emit(const Frame &f, const uint32_t *perm, const uint2 *rect,
                        const uint32_t *offsets, int64_t max_n, const Counters *cnt, int64_t capacity,
                        uint32_t *inst_tile, uint32_t *inst_val, cudaStream_t s);
cudaError_t launch_ranges(const uint32_t *tiles_sorted, int64_t max_n, const Counters *cnt,
                          uint2 *ranges, cudaStream_t s);
cudaError_t launch_inverse_perm(const uint32_t *perm, int64_t n_records, const Counters *cnt,
                                int32_t *inv, cudaStream_t s);
cudaError_t launch_export_keys(const Frame &f, const uint32_t *tiles_sorted,
                               const uint32_t *vals_sorted, const uint32_t *perm,
                               const uint32_t *depth_key_by_rec, int64_t n, uint64_t *keys,
                               int64_t *ids, int32_t *cams, cudaStream_t s);

// adam.cu
cudaError_t launch_adam(const gb_adam_tensor *ts, int n, const gb_adam_config &c, int grid_x, cudaStream_t s);

// render_fwd.cu / render_bwd.cu
struct RenderBufs {
    const Record *rec;        // indexed by record id
    const RecordLo *rec_lo;   // indexed by record id; read for flagged records only
    const uint32_t *perm;     // depth-sorted position -> record id
    const uint32_t *inst_val; // sorted instances -> depth-sorted position
    const uint2 *ranges;      // [n_tiles] (begin, end)
    const uint2 *pbox;        // [records] inclusive pixel rectangle (x0 | y0 << 16, x1 | y1 << 16)
    float *rgb, *depth, *alpha;
    float *t_final;           // [n_pixels]
    uint32_t *last;           // [n_pixels] 1 + index in the tile range of the last blended splat
    Counters *cnt;
};
// Which tiles a render launch processes: tile = list[off + i] (or off + i when
// list is null) for i < count; with `work` set, blocks are persistent and pull
// i from that device counter.
struct TileSched {
    const uint32_t *list;
    uint32_t off, count;
    uint32_t *work;
};
cudaError_t launch_render_fwd(const Frame &f, const RenderBufs &b, int batch, const uint32_t *tile_list,
                              uint32_t *work, bool persistent, cudaStream_t s);
cudaError_t launch_tile_list(const Frame &f, const uint2 *ranges, uint32_t *keys, uint32_t *vals, cudaStream_t s);

struct RenderBwdBufs {
    RenderBufs fw;
    const float *d_rgb, *d_depth, *d_alpha;
    float *rec_grad;          // [n_visible, 16], indexed by depth-sorted position
};
// fit2d.cu: image-fitting parameter map, its adjoint, MSE loss and gradient
cudaError_t launch_fit_params(const float *theta, const float *xy, const float *z, const float *log_s,
                              const float *logit, int64_t K, float *quats, float *means, float *scales, float *opac,
                              cudaStream_t s);
cudaError_t launch_fit_params_bwd(const float *theta, const float *log_s, const float *logit, int64_t K,
                                  const float *d_quats, const float *d_means, const float *d_scales,
                                  const float *d_opac, float *d_theta, float *d_xy, float *d_log_s, float *d_logit,
                                  cudaStream_t s);
cudaError_t launch_mse(const float *rgb, const float *target, int64_t n, float *d_rgb, double *loss, cudaStream_t s);

// texsh.cu: per-texel SH grids per (splat, camera) and the backward post-pass
cudaError_t launch_texsh_eval(const Frame &f, int si, int Dt, const void *coef, int dtype, float *out,
                              cudaStream_t s);
cudaError_t launch_texsh_grad(const Frame &f, int si, int Dt, const void *coef, int dtype, const float *grid_grad,
                              float *g_coef, float *g_means, cudaStream_t s);

// mip.cu: box filter of a scene's grids to N >> mip (FP32 out) and its adjoint
cudaError_t launch_mip_filter(const void *src, int dtype, int64_t K, int ns, int mip, float *dst, cudaStream_t s);
cudaError_t launch_mip_grad(const float *gc, int64_t K, int ns, int mip, float *gf, cudaStream_t s);

// ppt = pixels per thread, 1 or 2 (render_bwd.cu, render_bwd2.cu)
cudaError_t launch_render_bwd(const Frame &f, const RenderBwdBufs &b, int batch, int ppt, const uint32_t *tile_list,
                              uint32_t *work, bool persistent, cudaStream_t s);
// render_bwd_sp.cu: the splat-parallel backward (grids of N <= 4, tiles 8 and 16)
bool render_bwd_sp_supported(int tile, int N);
size_t render_bwd_sp_smem(int tile, int N, int dtype, int batch);
cudaError_t launch_render_bwd_sp(const Frame &f, const RenderBwdBufs &b, int batch, const uint32_t *tile_list,
                                 uint32_t *work, bool persistent, cudaStream_t s);
template <int P>
cudaError_t launch_render_bwd_p(const Frame &f, const RenderBwdBufs &b, int batch, const uint32_t *tile_list,
                                uint32_t *work, bool persistent, cudaStream_t s);

}  // namespace gbill
