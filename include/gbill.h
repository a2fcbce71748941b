/*
 * gbill.h -- C ABI of the GB300 (sm_103a) textured 2D-Gaussian-surfel
 * rasterizer ("Gaussian Billboards", arXiv 2412.12734), forward and backward.
 *
 * The library renders oriented 2D Gaussian surfels (Sec. 3.1, Eq. 3-4), each
 * carrying an N x N RGB colour grid sampled bilinearly in its uv plane
 * (Sec. 3.2, Eq. 5, Alg. 2) plus one set of view-dependent SH coefficients
 * added on top (Sec. 4.2), composited front to back (Sec. 3.1, Eq. 2,
 * Alg. 1 fwd).  The backward pass (Alg. 1 bwd, Alg. 2 adj-bilinear) returns
 * gradients for centres, quaternions, scales, opacities, SH coefficients and
 * texels, with the uv adjoint receiving the colour-interpolation term.
 *
 * Conventions shared by every entry point:
 *   - Every array argument is a DEVICE pointer (CUDA global memory) unless the
 *     comment says "host".  The caller owns every input and output buffer; the
 *     library never frees them and never keeps them after a call returns
 *     (except the saved state described at gb_saved_create).
 *   - Floats are IEEE binary32, little endian.  Arrays are dense, row-major,
 *     with the shapes given in brackets.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued on it; calls return before the GPU
 *     finishes unless a comment says the call synchronizes.
 *   - Errors are returned as gb_status; no call aborts, throws or exits.  A
 *     readable message for the last failing call on a context is available
 *     from gb_last_error().  On a non-OK return no output is guaranteed.
 *   - A context is not thread safe: use one context per host thread.
 *
 * Parameter meaning (activated values; logits/log-scales live above the ABI):
 *   means      [K,3]  splat centre p_k in world space                 (Eq. 3)
 *   quats      [K,4]  (w,x,y,z), any nonzero norm; normalised inside; the
 *                     tangents t_u, t_v are the first two columns of its
 *                     rotation matrix                                  (Sec. 3.1)
 *   scales     [K,2]  (s_u, s_v) > 0, linear                           (Eq. 3)
 *   opacities  [K]    o_k in (0,1); alpha = min(0.99, o_k G(u,v))      (Eq. 4)
 *   sh         [K,(D+1)^2,3]  real SH coefficients, degree D <= 3, ordered
 *                     l = 0..D, m = -l..l; colour term added to the grid colour
 *                     (Sec. 4.2), no offset and no clamp
 *   textures   [K,N,N,3] colour grid C_k[i_u][i_v][rgb] spanning
 *                     [-sigma, sigma]^2 of the uv plane, corner aligned, border
 *                     clamped                                        (Eq. 5, Alg. 2)
 *                     or, with per-texel SH, [K,N,N,(Dt+1)^2,3] coefficients
 *                     per texel (Sec. 4.2; gb_scene.tex_sh_degree); a scene
 *                     may also be rendered at a mip level of its grid
 *                     (Sec. 4.1, Fig. 4 f, g; gb_scene.mip_level)
 *
 * Beyond rendering: a fused multi-tensor Adam (gb_adam_step), the image-
 * fitting parameter map, its adjoint and an MSE loss (Sec. 4.1;
 * gb_fit_params, gb_fit_params_backward, gb_mse_loss), an autotuner, and a
 * forward that allocates nothing (gb_render_forward_noalloc).
 */
#ifndef GBILL_H
#define GBILL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBILL_ABI_VERSION 4
#define GBILL_MAX_CAMERAS 64
#define GBILL_MAX_SCENES 16

typedef enum {
    GB_OK = 0,
    GB_ERR_INVALID_ARG = 1, /* a pointer, size, count or option is out of range   */
    GB_ERR_UNSUPPORTED = 2, /* valid request the build does not implement          */
    GB_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the reason)  */
    GB_ERR_CAPACITY = 4,    /* a reserved buffer was too small (no-sync mode)       */
    GB_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (reserved: no
                               kernel of this library waits on another block;
                               persistent blocks take tiles from an atomic
                               counter)                                        */
    GB_ERR_NONFINITE = 6    /* non-finite values were found where none may be       */
} gb_status;

typedef enum { GB_F32 = 0, GB_F16 = 1, GB_BF16 = 2 } gb_dtype;

/* Forward option flags. */
#define GB_FLAG_NO_SYNC 1u /* never synchronize: use the reserved capacity of the
                              saved state, flag overflow on the device (checked by
                              gb_saved_check); required inside CUDA graph capture */
#define GB_FLAG_PERSISTENT 2u /* render with persistent blocks pulling tiles from
                                 a device work counter instead of one block per tile */
#define GB_FLAG_TIMING 4u     /* record CUDA events around every phase of this forward
                                 and of the backward that follows it (see
                                 gb_saved_phase_times); not for use in graph capture */

typedef struct gb_context gb_context;
typedef struct gb_saved gb_saved;

/* One pinhole camera (OpenCV axes: x right, y down, z forward).  Pixel (x,y)
 * has its centre at (x+0.5, y+0.5); (cx, cy) is the principal point in those
 * pixel units.  Host struct. */
typedef struct {
    int32_t width, height;  /* pixels, 1..16384                                 */
    float fx, fy, cx, cy;   /* intrinsics                                        */
    float world_to_cam[12]; /* row-major 3x4 [R | t]; R orthonormal              */
    float near_plane;       /* splats with centre depth <= near are culled       */
    int32_t scene;          /* index into the scenes array of the call           */
} gb_camera;

/* One scene: K splats sharing one texture size and storage type.  Host
 * struct whose array members are device pointers. */
typedef struct {
    int64_t num_splats;       /* K >= 0                                          */
    const float *means;       /* [K,3]                                           */
    const float *quats;       /* [K,4]                                           */
    const float *scales;      /* [K,2]                                           */
    const float *opacities;   /* [K]                                             */
    const void *sh;           /* [K,(D+1)^2,3] of sh_dtype                       */
    const void *textures;     /* [K,N,N,3] of tex_dtype, or with tex_sh_degree   */
                              /* Dt >= 1 [K,N,N,(Dt+1)^2,3]: per-texel SH        */
    int32_t sh_degree;        /* D in 0..3                                       */
    int32_t sh_dtype;         /* gb_dtype                                        */
    int32_t tex_n;            /* N in {1,2,4,8,16}                               */
    int32_t tex_dtype;        /* gb_dtype                                        */
    float sigma;              /* grid extent in uv units (paper default 0.5)     */
    int32_t mip_level;        /* 0: render the N x N grid.  l in 1..log2(N):     */
                              /* render every grid box-filtered to N/2^l x N/2^l */
                              /* (texel = mean of its 2^l x 2^l block; Sec. 4.1, */
                              /* Fig. 4 f, g); gradients still reach the N x N   */
                              /* texels (1/4^l of the coarse texel's gradient).  */
                              /* The filtered grids live in FP32 scratch of the  */
                              /* saved state, sized by a synchronizing forward;  */
                              /* a no-sync forward that needs more fails with    */
                              /* GB_ERR_CAPACITY.                                 */
    int32_t tex_sh_degree;    /* 0: RGB texels.  Dt in 1..3: every texel holds   */
                              /* (Dt+1)^2 SH coefficient triples and shows       */
                              /* sum_lm k_lm Y_lm(d), d the splat's view         */
                              /* direction (Sec. 4.2).  The grids of every       */
                              /* (splat, camera) record are evaluated into FP32  */
                              /* scratch of the saved state (records x N^2 x 3,  */
                              /* sized by a synchronizing forward); gradients    */
                              /* reach the coefficients and, through d, the      */
                              /* means.  Not combined with mip_level.            */
    int32_t reserved;         /* must be 0                                       */
    const uint8_t *splat_tex_n; /* [K] or NULL: per-splat grid size n_k in     */
                              /* 1..tex_n (values outside are clamped to it):  */
                              /* splat k's n_k x n_k grid is rows and columns  */
                              /* 0..n_k-1 of its tex_n x tex_n block, sampled  */
                              /* by Alg. 2 with n_k (the other texels are never */
                              /* read; their gradient is 0).  Needs tex_n >= 2, */
                              /* no mip level or per-texel SH, 16 x 16 tiles and */
                              /* the pixel-parallel backward with one pixel per */
                              /* thread (else GB_ERR_UNSUPPORTED).  The variable */
                              /* grid resolution of Sec. 3.3 and 5.             */
} gb_scene;

/* Gradient outputs of one scene, FP32 device arrays shaped like the inputs.
 * gb_render_backward OVERWRITES them with the sum over that scene's cameras.
 * A NULL member skips that output (its work is still done). */
typedef struct {
    float *d_means, *d_quats, *d_scales, *d_opacities, *d_sh, *d_textures;
} gb_grads;

/* Render options (host struct; NULL = defaults). */
typedef struct {
    int32_t tile_size;   /* tile edge in pixels: 8, 16 or 32 (0 = 16)             */
    int32_t batch_depth; /* splats staged per shared-memory batch of the backward
                            (and of the forward when batch_depth_fwd is 0),
                            0 = automatic; otherwise a multiple of 8 up to the
                            tile's pixels whose staging fits 200 KB of shared
                            memory                                                */
    uint32_t flags;      /* GB_FLAG_*                                             */
    int32_t pixels_per_thread; /* backward: 1, or 2 (two pixels of a column per
                                  thread on the packed FP32x2 pipe); 0 = 1. With 2,
                                  batch_depth is at most tile_size^2 / 2.  (The
                                  forward always runs two pixels per thread,
                                  one for 16 x 16 grids.)                       */
    float background[3]; /* added as T_final * background (default black)        */
    int32_t batch_depth_fwd; /* the forward's batch depth under the same rules;
                                0 = batch_depth, or the forward's own automatic
                                depth when batch_depth is 0 too                */
    int32_t bwd_kernel;  /* backward render loop: 0 = automatic, 1 = pixel-
                            parallel (a lane per pixel, gradients reduced across
                            the warp per splat; pixels_per_thread applies),
                            2 = splat-parallel (a lane per splat, transmittance
                            and colour behind each splat by warp prefix scans
                            over the splats, gradients summed in the lane;
                            grids of N <= 4 on 8 x 8 or 16 x 16 tiles, else
                            GB_ERR_UNSUPPORTED; batch depth a multiple of 8 up
                            to 256).  Automatic is pixel-parallel; the
                            autotuner times both.                             */
} gb_options;

/* Counters of the last forward on a saved state (gb_saved_stats). */
typedef struct {
    int64_t records;     /* (splat, camera) pairs projected                       */
    int64_t visible;     /* records that survived culling                          */
    int64_t instances;   /* (tile, splat) pairs after duplication                  */
    int64_t tiles;       /* tiles over all cameras                                 */
    int64_t pixels;      /* pixels over all cameras                                */
    int64_t capacity;    /* reserved instance capacity                             */
    int32_t overflow;    /* nonzero if a no-sync forward ran out of capacity       */
    int32_t error_flags; /* device error bits (bit 0: bounded wait timed out;
                            bit 1: a splat with a non-finite mean, quaternion,
                            scale, opacity or SH colour was culled)            */
    int64_t pairs_fwd;   /* (pixel, splat) pairs evaluated by the last forward     */
    int64_t pairs_bwd;   /* (pixel, splat) pairs evaluated by the last backward    */
    int64_t blended_fwd;      /* pairs blended by the last forward            */
    int64_t contributing_bwd; /* pairs whose adjoints the last backward computed:
                                 the blended pairs of its forward (0 before a
                                 backward)                                    */
} gb_stats;

/* Phases timed under GB_FLAG_TIMING, in the order gb_saved_phase_times
 * returns them. */
typedef enum {
    GB_PHASE_PREPROCESS = 0, /* grid pre-passes (mip filter, per-texel SH grids);
                                culling, FP32 rectangle, depth key, SH colour;
                                compaction of the visible records and their
                                homography records                           */
    GB_PHASE_DEPTH_SORT,     /* radix sort of the visible records by depth        */
    GB_PHASE_COUNT_SCAN,     /* exclusive scan of per-record tile counts          */
    GB_PHASE_EMIT,           /* (tile, splat) duplication                         */
    GB_PHASE_TILE_SORT,      /* stable radix sort of instances by tile            */
    GB_PHASE_RANGES,         /* per-tile [begin, end)                             */
    GB_PHASE_RENDER_FWD,     /* per-tile front-to-back render                     */
    GB_PHASE_BWD_SETUP,      /* gradient buffers zeroed, inverse permutation      */
    GB_PHASE_RENDER_BWD,     /* per-tile back-to-front adjoint; mip-filter adjoint */
    GB_PHASE_PREPROCESS_BWD, /* chain to means, quats, scales, opacity, SH;
                                per-texel SH coefficient and centre gradients */
    GB_PHASE_COUNT
} gb_phase;

/* ---------------------------------------------------------------- contexts -- */

/* Creates a context bound to CUDA device `device` (made current on the calling
 * thread).  The context owns the scratch memory of the sort (grown on demand
 * with cudaMalloc).  *out receives the handle; GB_ERR_CUDA if the device is
 * missing. */
gb_status gb_context_create(int32_t device, gb_context **out);

/* Frees the context and its scratch after synchronizing the device.  NULL is a
 * no-op.  Saved states created from it must be destroyed first. */
gb_status gb_context_destroy(gb_context *ctx);

/* Message of the last failing call on `ctx` (static storage owned by the
 * context; valid until the next call on it).  Never NULL. */
const char *gb_last_error(const gb_context *ctx);

/* Name of a status code.  Never NULL. */
const char *gb_status_string(gb_status status);

/* ------------------------------------------------------------- saved state -- */

/* A saved state holds everything the backward pass needs from one forward:
 * projected records, the depth permutation, the sorted (tile, splat) list,
 * the tile ranges and per-pixel final transmittance and last-contributor
 * index (the backward recomputes each pixel's transmittances from these,
 * Alg. 1 bwd).  It is created empty and grows on demand with cudaMalloc in
 * synchronizing forwards; it is overwritten by every forward that uses it.
 * It must not be shared by two forwards in flight. */
gb_status gb_saved_create(gb_context *ctx, gb_saved **out);
gb_status gb_saved_destroy(gb_saved *saved);

/* Pre-sizes a saved state so that GB_FLAG_NO_SYNC forwards (e.g. inside a CUDA
 * graph capture) never allocate: `records` = sum over cameras of the scene's
 * splat count, `instances` = (tile, splat) pairs, `pixels` and `tiles` over
 * all cameras.  Synchronizes the device.  A forward recorded on the state
 * stays valid: buffers that grow keep their contents, so its backward may
 * follow the reserve.  Growing moves the buffers, so a CUDA graph captured
 * on the state before the reserve must be captured again. */
gb_status gb_saved_reserve(gb_saved *saved, int64_t records, int64_t instances, int64_t pixels,
                           int64_t tiles);

/* Copies the counters of the last forward into *out (host); synchronizes the
 * saved state's last stream. */
gb_status gb_saved_stats(gb_saved *saved, gb_stats *out);

/* Synchronizes and returns GB_ERR_CAPACITY if the last no-sync forward ran out
 * of instance capacity (its outputs are then invalid; reserve more and rerun),
 * GB_ERR_TIMEOUT if a bounded device wait gave up, GB_ERR_NONFINITE if the last
 * forward culled splats with a non-finite mean, quaternion, scale, opacity or
 * SH colour (the rest of the frame is rendered as if they were absent; texel
 * values are not checked), else GB_OK. */
gb_status gb_saved_check(gb_saved *saved);

/* Durations in milliseconds (host array ms[GB_PHASE_COUNT]) of the phases of
 * the last forward run with GB_FLAG_TIMING and of the backward after it
 * (entries of a pass not run are -1).  Synchronizes. */
gb_status gb_saved_phase_times(gb_saved *saved, float *ms, int32_t cap);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts), for launch accounting. */
uint64_t gb_kernel_launches(void);

/* Copies the projected records of the last forward to HOST memory for
 * inspection: rec[r][16] for record r = (camera c, splat k), r = sum of the
 * splat counts of the scenes of cameras 0..c-1, plus k.  Layout per record:
 * t11, -t01, -t10, t00, m20, m21, m22, z, c_hi.x, c_hi.y, c_lo.x, c_lo.y, o,
 * r, g, b, where T' = [[t00 t01 0][t10 t11 0][t20 t21 z]] is the splat-to-
 * screen homography with the projected centre c moved to the origin and
 * (m20, m21, m22) = third row of adj(T') / z; a pixel at offset (dx, dy) from
 * c hits the splat at u = (t11 dx - t01 dy) / (m20 dx + m21 dy + m22), v =
 * (t00 dy - t10 dx) / (same).  c = c_hi + c_lo with c_hi on the 1/512-pixel
 * grid.  Every field is the FP32 rounding of its double-float value.  A record
 * whose plane-hit evaluation is ill-conditioned (a thin splat seen along its
 * long axis, or a grazing one) stores z negated and is evaluated in extended
 * precision from its low parts: rec_lo[r][12] (host, nullable) receives them,
 * lo(t11), -lo(t01), -lo(t10), lo(t00), lo(m20), lo(m21), 0, 0, then the
 * centre terms -(t11 c_lo.x - t01 c_lo.y), -(t00 c_lo.y - t10 c_lo.x),
 * lo(m22) - (m20 c_lo.x + m21 c_lo.y), 0 (zeros for other records).
 * visible[r] = 1 if the record survived culling (other rows are undefined).
 * `cap` = records the host arrays hold.  Synchronizes. */
gb_status gb_saved_export_records(gb_saved *saved, float *rec, float *rec_lo, uint8_t *visible, int64_t cap,
                                  int64_t *count);

/* Copies the sorted instance list of the last forward to HOST arrays: keys[i]
 * = (global tile id << 32) | bits(FP32 centre depth), ids[i] = splat index
 * within its scene, cams[i] = camera index.  Global tile ids number the tiles
 * of camera 0 first (row-major, ceil(W/tile) per row), then camera 1, ...
 * `cap` is the host capacity; *count receives the instance count (arrays are
 * filled up to min(count, cap)).  Synchronizes.  Used by parity tests. */
gb_status gb_saved_export_keys(gb_saved *saved, uint64_t *keys, int64_t *ids, int32_t *cams,
                               int64_t cap, int64_t *count);

/* ----------------------------------------------------------------- render -- */

/* Forward render of all cameras (Alg. 1 fwd; Eq. 2-5).
 *   scenes  host array [n_scenes] (1..GBILL_MAX_SCENES)
 *   cams    host array [n_cams]   (1..GBILL_MAX_CAMERAS); cams[i].scene indexes scenes
 *   rgb     [P,3]  P = sum over cameras of W*H; camera i's pixels start at
 *                  sum_{j<i} W_j H_j, row-major within a camera
 *   depth   [P]    sum_i z_i alpha_i T_i (z_i: plane-hit depth, or centre
 *                  depth where the screen-space low-pass is the larger)
 *   alpha   [P]    1 - T_final
 * Steps on `stream`: preprocess (homography, FP32 tile rectangle, depth key),
 * depth radix sort, tile-count scan, (tile, splat) duplication, tile radix
 * sort, tile ranges, per-tile render.  Unless GB_FLAG_NO_SYNC is set the
 * call synchronizes once (to size the instance list) and may grow `saved`.
 * Returns GB_ERR_INVALID_ARG for bad sizes/pointers/options,
 * GB_ERR_UNSUPPORTED for tex_n not in {1,2,4,8,16} or sh_degree > 3,
 * GB_ERR_CAPACITY when the frame has 0xF0000000 or more (tile, splat)
 * instances (a synchronizing forward; a no-sync forward flags it for
 * gb_saved_check like any instance count above its reservation). */
gb_status gb_render_forward(gb_context *ctx, gb_saved *saved, const gb_scene *scenes,
                            int32_t n_scenes, const gb_camera *cams, int32_t n_cams,
                            const gb_options *opt, float *rgb, float *depth, float *alpha,
                            void *stream);

/* Backward of the last forward on `saved` (Alg. 1 bwd, Alg. 2 adj-bilinear).
 *   d_rgb   [P,3] dL/drgb (required); d_depth [P], d_alpha [P] (nullable)
 *   grads   host array [n_scenes] of gb_grads (device pointers), overwritten
 *           with the gradient summed over each scene's cameras.
 * The scene parameter arrays passed to the forward must be unchanged.
 * Enqueued on `stream`, never synchronizes.  It reads what the forward wrote
 * into `saved`: use the forward's stream, or order `stream` after it (an
 * event), as for any dependent CUDA work. */
gb_status gb_render_backward(gb_context *ctx, gb_saved *saved, const float *d_rgb,
                             const float *d_depth, const float *d_alpha, const gb_grads *grads,
                             int32_t n_scenes, void *stream);

/* ------------------------------------------------------------------ adam -- */

/* One tensor of a fused Adam step (the optimiser of Sec. 3.3).  All pointers
 * are device pointers of n elements; param, m and v are FP32 and updated in
 * place; grad is read.  shadow (nullable) receives the updated parameter in
 * shadow_dtype (FP16/BF16 storage read by the renderer, or FP32). */
typedef struct {
    float *param;
    const float *grad;
    float *m, *v;
    void *shadow;
    int32_t shadow_dtype; /* gb_dtype */
    int32_t reserved;     /* must be 0 */
    int64_t n;
} gb_adam_tensor;

/* Adam hyper-parameters; step is the 1-based iteration used for the bias
 * corrections 1 - beta^step. */
typedef struct {
    float lr, beta1, beta2, eps;
    int32_t step;
    int32_t reserved; /* must be 0 */
} gb_adam_config;

/* m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), in FP32, for every
 * element of up to 16 tensors in one launch on `stream` (host array `tensors`).
 * GB_ERR_INVALID_ARG for bad counts, null pointers, beta outside [0,1),
 * step < 1. */
gb_status gb_adam_step(gb_context *ctx, const gb_adam_tensor *tensors, int32_t n_tensors,
                       const gb_adam_config *cfg, void *stream);

/* ------------------------------------------------------ no allocation -- */

/* Forward render for callers that cannot allocate device memory: code that
 * runs where cudaMalloc is unavailable or forbidden (a host with a fixed
 * device-memory budget handed out by someone else, a plug-in that must not
 * touch the allocator, a caller that owns all memory it uses).  There is no
 * counterpart in the paper; it is the forward of gb_render_forward (same
 * arguments and outputs, no saved state, so no backward after it) with every
 * scratch buffer taken from one fixed device array of about 36 MB compiled
 * into the library; every GPU that loads the library holds that array until
 * the process exits.
 * Limits per call: 131,072 records (splats x cameras), 524,288 (tile, splat)
 * instances, 1,048,576 pixels, 8,192 tiles; beyond them the call returns
 * GB_ERR_CAPACITY with a message and renders nothing.  GB_FLAG_TIMING and
 * GB_FLAG_PERSISTENT, and scenes with a mip_level or per-texel SH, are
 * rejected (GB_ERR_UNSUPPORTED).
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.
 * The call synchronizes `stream` once to check the instance count.  Every
 * call shares the one array, which keeps the previous call's contents: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialized by the caller. */
gb_status gb_render_forward_noalloc(gb_context *ctx, const gb_scene *scenes, int32_t n_scenes,
                                    const gb_camera *cams, int32_t n_cams, const gb_options *opt,
                                    float *rgb, float *depth, float *alpha, void *stream);

/* --------------------------------------------------------- image fitting -- */

/* Image fitting (Sec. 4.1): one camera looks down +z at splats that face it
 * and may only turn about the view axis.  A splat's raw parameters are an
 * angle theta [K], a position xy [K,2] in its plane at depth z [K],
 * log-scales [K,2] and an opacity logit [K] (FP32 device arrays).  This
 * writes the activated parameters gb_scene takes:
 *   quats     = (cos(theta/2), 0, 0, sin(theta/2))   [K,4]
 *   means     = (x, y, z)                              [K,3]
 *   scales    = exp(log_scales)                        [K,2]
 *   opacities = 1 / (1 + exp(-logit))                  [K]
 * All pointers are device arrays of K >= 0 rows; no allocation, no sync. */
gb_status gb_fit_params(gb_context *ctx, int64_t K, const float *theta, const float *xy, const float *z,
                        const float *log_scales, const float *logit_opacities, float *quats, float *means,
                        float *scales, float *opacities, void *stream);

/* Adjoint of gb_fit_params: from the renderer's gradients of the activated
 * parameters (d_quats [K,4], d_means [K,3], d_scales [K,2], d_opacities [K],
 * e.g. the gb_grads of gb_render_backward) to the raw parameters'
 * (d_theta [K], d_xy [K,2], d_log_scales [K,2], d_logit_opacities [K],
 * overwritten).  The z gradient is not formed (the planes stay fixed). */
gb_status gb_fit_params_backward(gb_context *ctx, int64_t K, const float *theta, const float *log_scales,
                                 const float *logit_opacities, const float *d_quats, const float *d_means,
                                 const float *d_scales, const float *d_opacities, float *d_theta, float *d_xy,
                                 float *d_log_scales, float *d_logit_opacities, void *stream);

/* Mean squared error over n values (e.g. n = 3 x pixels of an rgb image):
 * *loss = mean (rgb - target)^2, a device FP64 scalar overwritten on
 * `stream` (summed in FP64); d_rgb (device, nullable) = 2 (rgb - target) / n,
 * the upstream gradient for gb_render_backward.  No allocation, no sync. */
gb_status gb_mse_loss(gb_context *ctx, const float *rgb, const float *target, int64_t n, float *d_rgb,
                      double *loss, void *stream);

/* ---------------------------------------------------------------- tuning -- */

/* Autotuner: times forward + backward of this frame for every candidate
 * (tile_size 8, 16 and 32; batch_depth 8, 16, 24, 32, 48, 64, 88, 128, 184,
 * 256 where it fits the tile and the shared-memory budget; pixels_per_thread
 * 1 and 2; the forward at its automatic depth; the splat-parallel backward where it
 * applies, listed with pixels_per_thread 3), then, at the fastest of those,
 * times the forward alone at every
 * batch_depth_fwd candidate (listed with pixels_per_thread 0 and the forward's
 * time), and writes the fastest options to *best (flags and
 * background are copied from *base, which may be NULL).  Each candidate runs
 * once untimed (which may grow `saved`) and then `reps` timed repetitions
 * (1..100) with dL/drgb = 1 for every pixel.  The call allocates its own
 * output, upstream-gradient and parameter-gradient buffers with cudaMalloc and
 * frees them before returning; it synchronizes the device.  ms (host array of
 * `cap` floats, nullable) receives the mean time per candidate in the order
 * tried, tiles/batches (host, nullable) the candidate's options;
 * *n_candidates (nullable) the number tried. */
gb_status gb_autotune(gb_context *ctx, gb_saved *saved, const gb_scene *scenes, int32_t n_scenes,
                      const gb_camera *cams, int32_t n_cams, const gb_options *base, int32_t reps,
                      gb_options *best, float *ms, int32_t *tiles, int32_t *batches, int32_t *ppts,
                      int32_t cap, int32_t *n_candidates);

#ifdef __cplusplus
}
#endif

#endif /* GBILL_H */
