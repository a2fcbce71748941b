// C ABI of the rasterizer (include/gbill.h): argument checking, the frame
// descriptor, buffer management of saved states and the launch sequence of
// the forward and backward passes.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "gbill_internal.cuh"
#include "render_common.cuh"

using namespace gbill;

namespace gbill {
static std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(uint64_t(n), std::memory_order_relaxed); }
}  // namespace gbill

// Events: [0..7] forward start + after each of its 7 phases, [8..11] backward.
constexpr int kNumEvents = 12;

struct gb_context {
    int device;
    char err[512];
};

struct gb_saved {
    gb_context *ctx;
    int64_t cap_rec, cap_inst, cap_pix, cap_tiles;
    Record *rec;
    RecordLo *rec_lo;
    uint32_t *depth_key, *keys_tmp, *vals_tmp, *dkeys_sorted, *perm, *offsets;
    uint2 *rect, *pbox;
    int32_t *inv;
    float *rec_grad;
    uint32_t *inst_tile, *inst_val, *inst_tile_tmp, *inst_val_tmp, *tiles_sorted, *vals_sorted;
    uint2 *ranges;
    uint32_t *tl_keys, *tl_vals, *tl_keys_tmp, *tl_vals_tmp, *tl_keys_out, *tile_list;
    uint32_t *work;  // [2 * kMaxGroups] persistent-render work counters (forward, backward)
    bool use_list;
    float *t_final;
    uint32_t *last;
    Counters *cnt;
    Counters *cnt_host;
    void *scratch;
    size_t scratch_bytes;
    // mip-level grids: box-filtered FP32 grids of the last forward and their
    // gradient, packed per scene at mip_off[] (floats)
    float *mip_tex, *mip_grad;
    int64_t mip_cap;
    int64_t mip_off[kMaxScenes];
    int32_t mip_ns[kMaxScenes];
    // per-texel SH: evaluated grids of every (splat, camera) record and their
    // gradient, per scene at tsh_off[] (floats); the scenes' coefficients
    float *tsh_tex, *tsh_grad;
    int64_t tsh_cap;
    int64_t tsh_off[kMaxScenes], tsh_rows[kMaxScenes];
    const void *tsh_coef[kMaxScenes];
    int32_t tsh_dtype[kMaxScenes];
    // last forward
    Frame frame;
    bool has_forward;
    int64_t n_records, n_pixels, max_k, inst_max;
    int tile_bits, batch_fwd, batch_bwd, ppt;
    bool bwd_sp;  // the backward runs the splat-parallel loop
    uint32_t flags;
    cudaStream_t stream;
    cudaEvent_t ev[kNumEvents];
    bool ev_ready, timed_fwd, timed_bwd;
};

namespace {

gb_status fail(gb_context *ctx, gb_status st, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define GB_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), GB_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                 \
    } while (0)

cudaError_t alloc(void **p, size_t bytes) {
    if (*p) {
        cudaError_t e = cudaFree(*p);
        if (e != cudaSuccess) return e;
    }
    *p = nullptr;
    return cudaMalloc(p, std::max<size_t>(bytes, 16));
}

template <typename T>
cudaError_t alloc_t(T **p, int64_t n) {
    return alloc(reinterpret_cast<void **>(p), size_t(std::max<int64_t>(n, 1)) * sizeof(T));
}

// Grows *p, which holds old_n elements, to n elements.  With keep, the first
// old_n elements move to the new allocation (a recorded forward stays valid
// across gb_saved_reserve); without, the contents are dropped.  The device is
// idle when it is called.
template <typename T>
cudaError_t grow_t(T **p, int64_t old_n, int64_t n, bool keep) {
    if (!keep || !*p || old_n <= 0) return alloc_t(p, n);
    T *q = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&q), std::max<size_t>(size_t(std::max<int64_t>(n, 1)) * sizeof(T), 16));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(q, *p, size_t(std::min(old_n, n)) * sizeof(T), cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(q);
        return e;
    }
    e = cudaFree(*p);
    *p = q;
    return e;
}

// The reserve_* functions grow one group of saved-state buffers to at least n
// elements.  keep: the buffers hold a recorded forward that a backward may
// still read (gb_saved_reserve between a forward and its backward), so their
// contents move with them; a forward sizing its own buffers drops them.
gb_status reserve_records(gb_saved *s, int64_t n, bool keep = false) {
    if (n <= s->cap_rec) return GB_OK;
    gb_context *ctx = s->ctx;
    GB_CUDA(ctx, cudaDeviceSynchronize());
    const int64_t c = n + n / 8 + 1024, o = s->cap_rec;
    GB_CUDA(ctx, grow_t(&s->rec, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->rec_lo, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->depth_key, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->keys_tmp, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->vals_tmp, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->dkeys_sorted, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->perm, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->offsets, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->rect, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->pbox, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->inv, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->rec_grad, o * kRecGrad, c * kRecGrad, keep));
    s->cap_rec = c;
    return GB_OK;
}

gb_status reserve_instances(gb_saved *s, int64_t n, bool keep = false) {
    if (n <= s->cap_inst) return GB_OK;
    gb_context *ctx = s->ctx;
    if (n >= int64_t(0xF0000000u))
        return fail(ctx, GB_ERR_CAPACITY, "%lld (tile, splat) instances exceed the 32-bit index range",
                    (long long)n);
    GB_CUDA(ctx, cudaDeviceSynchronize());
    const int64_t c = std::min<int64_t>(n + n / 4 + 4096, int64_t(0xF0000000u)), o = s->cap_inst;
    GB_CUDA(ctx, grow_t(&s->inst_tile, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->inst_val, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->inst_tile_tmp, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->inst_val_tmp, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->tiles_sorted, o, c, keep));
    GB_CUDA(ctx, grow_t(&s->vals_sorted, o, c, keep));
    s->cap_inst = c;
    return GB_OK;
}

gb_status reserve_pixels(gb_saved *s, int64_t n, bool keep = false) {
    if (n <= s->cap_pix) return GB_OK;
    gb_context *ctx = s->ctx;
    GB_CUDA(ctx, cudaDeviceSynchronize());
    const int64_t o = s->cap_pix;
    GB_CUDA(ctx, grow_t(&s->t_final, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->last, o, n, keep));
    s->cap_pix = n;
    return GB_OK;
}

gb_status reserve_tiles(gb_saved *s, int64_t n, bool keep = false) {
    if (n <= s->cap_tiles) return GB_OK;
    gb_context *ctx = s->ctx;
    GB_CUDA(ctx, cudaDeviceSynchronize());
    const int64_t o = s->cap_tiles;
    GB_CUDA(ctx, grow_t(&s->ranges, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->tl_keys, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->tl_vals, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->tl_keys_tmp, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->tl_vals_tmp, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->tl_keys_out, o, n, keep));
    GB_CUDA(ctx, grow_t(&s->tile_list, o, n, keep));
    if (!s->work) GB_CUDA(ctx, alloc_t(&s->work, 2 * kMaxGroups));
    s->cap_tiles = n;
    return GB_OK;
}

gb_status reserve_scratch(gb_saved *s) {
    const size_t need = std::max(radix_scratch_bytes(std::max(std::max(s->cap_rec, s->cap_inst), s->cap_tiles)),
                                 scan_scratch_bytes(s->cap_rec)) + 1024;
    if (need <= s->scratch_bytes) return GB_OK;
    gb_context *ctx = s->ctx;
    GB_CUDA(ctx, cudaDeviceSynchronize());
    GB_CUDA(ctx, alloc(&s->scratch, need));
    s->scratch_bytes = need;
    return GB_OK;
}

size_t frame_smem(const Frame &f, int batch, bool bwd);
int default_batch(const Frame &f, bool bwd);

// The forward's batch depth: batch_depth_fwd, else batch_depth, else the
// forward's automatic depth (at most the tile's pixels).
int forward_batch(const gb_options &o, const Frame &f, int nt) {
    if (o.batch_depth_fwd) return o.batch_depth_fwd;
    if (o.batch_depth) return o.batch_depth;
    return std::min(default_batch(f, false), nt);
}

// Automatic batch depth of one pass: the most splats whose staging fits the
// pass's shared-memory budget per block, a multiple of 8, at least 8.  The
// backward gets 48 KB, so that four blocks (the register limit of its 256
// threads) stay resident per SM: with FP16 grids staged at 8 bytes a texel
// that is 184 at N = 4, 72 at N = 8 and 16 at N = 16 (measured on the
// 1M-splat, 16-view workload: N = 4 at 88 / 128 / 184: 39.9 / 38.7 / 37.8 ms;
// N = 8 at 32 / 64 / 88: 42.7 / 41.0 / 41.8 ms; N = 16 at 16 / 24: 54.1 /
// 54.2 ms).  The forward gets 36 KB, so that six blocks (its register limit
// at 16 x 16 tiles) stay resident: 88 at N = 4, 56 at N = 8, 16 at N = 16.
int default_batch(const Frame &f, bool bwd) {
    const int per = int(frame_smem(f, 1, bwd));
    int b = ((bwd ? 48 : 36) * 1024) / per;
    b = std::min(b, 256);
    b &= ~7;
    return std::max(b, 8);
}

// Staged bytes of one batch of the forward (bwd false) or the backward for a
// grid of size N stored as TexT; the forward stages grids of N <= 4 as FP32
// RGBA whatever their storage type.
template <typename TexT>
size_t batch_smem_t(int N, int batch, bool bwd) {
    switch (N) {
        case 1: return bwd ? bwd_stage_bytes<1, TexT>(batch) : stage_bytes<1, TexT, true>(batch, false);
        case 2: return bwd ? bwd_stage_bytes<2, TexT>(batch) : stage_bytes<2, TexT, true>(batch, false);
        case 4: return bwd ? bwd_stage_bytes<4, TexT>(batch) : stage_bytes<4, TexT, true>(batch, false);
        case 8: return bwd ? bwd_stage_bytes<8, TexT>(batch) : stage_bytes<8, TexT>(batch, false);
        default: return bwd ? bwd_stage_bytes<16, TexT>(batch) : stage_bytes<16, TexT>(batch, false);
    }
}

// The same for a grid stored as `dtype` (FP16 and BF16 stage alike).
size_t batch_smem(int N, int dtype, int batch, bool bwd) {
    return dtype == GB_F32 ? batch_smem_t<float>(N, batch, bwd) : batch_smem_t<__half>(N, batch, bwd);
}

// The largest over the frame's render groups (one batch depth serves all);
// per-splat grid sizes take 4 more bytes a staged splat.
size_t frame_smem(const Frame &f, int batch, bool bwd) {
    size_t m = 0;
    for (int g = 0; g < f.n_groups; ++g)
        m = std::max(m, batch_smem(f.group_N[g], f.group_dtype[g], batch, bwd) +
                            (f.group_var[g] ? size_t(batch) * 4 : 0));
    return m;
}

bool frame_has_var(const Frame &f) {
    for (int g = 0; g < f.n_groups; ++g)
        if (f.group_var[g]) return true;
    return false;
}

// Whether every render group of the frame can take the splat-parallel
// backward, and its shared memory per block at a batch depth.
bool frame_sp_ok(const Frame &f) {
    for (int g = 0; g < f.n_groups; ++g)
        if (f.group_var[g] || !render_bwd_sp_supported(f.tile, f.group_N[g])) return false;
    return true;
}
size_t frame_sp_smem(const Frame &f, int batch) {
    size_t m = 0;
    for (int g = 0; g < f.n_groups; ++g)
        m = std::max(m, render_bwd_sp_smem(f.tile, f.group_N[g], f.group_dtype[g], batch));
    return m;
}

// Automatic batch depth of the splat-parallel backward: its registers leave
// two resident blocks of 256 threads per SM, so a block may take up to 96 KB
// of staging; longer batches give each warp longer lists of splats to spread
// over its lanes.  At most 256, a multiple of 8.
int default_batch_sp(const Frame &f) {
    int b = 256;
    while (b > 8 && frame_sp_smem(f, b) > 96 * 1024) b -= 8;
    return b;
}

// The automatic backward loop is the pixel-parallel one: on the 1M-splat,
// 16-view workload at N = 4 the splat-parallel loop took 63.8 ms at batch depth
// 176 (68.8 at 128, 78.2 at 88) against 42.7 ms (2-view ncu case: 3.60e9
// warp instructions at 18 active threads each, against 3.71e9 at 25.6: per
// pixel only a few splats of a warp's list are blended, so the scans and
// per-pixel broadcasts serve few lanes).  The autotuner still times it.
constexpr bool kSplatParallelAuto = false;

__global__ void zero_rec_grad(float *g, const Counters *cnt, int64_t max_n) {
    const int64_t n = std::min<int64_t>(int64_t(cnt->n_visible), max_n) * kRecGrad / 4;
    float4 *g4 = reinterpret_cast<float4 *>(g);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

bool dtype_ok(int32_t d) { return d == GB_F32 || d == GB_F16 || d == GB_BF16; }

gb_status build_frame(gb_context *ctx, const gb_scene *scenes, int32_t n_scenes, const gb_camera *cams,
                      int32_t n_cams, int tile, const float bg[3], Frame &f, int64_t &max_k) {
    if (!scenes || n_scenes < 1 || n_scenes > kMaxScenes)
        return fail(ctx, GB_ERR_INVALID_ARG, "n_scenes must be in 1..%d", kMaxScenes);
    if (!cams || n_cams < 1 || n_cams > kMaxCams)
        return fail(ctx, GB_ERR_INVALID_ARG, "n_cams must be in 1..%d", kMaxCams);
    memset(&f, 0, sizeof(f));
    f.n_cams = n_cams;
    f.n_scenes = n_scenes;
    f.tile = tile;
    for (int i = 0; i < 3; ++i) f.bg[i] = bg ? bg[i] : 0.0f;
    max_k = 0;
    for (int s = 0; s < n_scenes; ++s) {
        const gb_scene &g = scenes[s];
        SceneDev &d = f.scenes[s];
        if (g.num_splats < 0 || g.num_splats > (int64_t(1) << 31))
            return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: num_splats %lld out of range", s, (long long)g.num_splats);
        if (g.sh_degree < 0 || g.sh_degree > 3)
            return fail(ctx, GB_ERR_UNSUPPORTED, "scene %d: sh_degree %d not in 0..3", s, g.sh_degree);
        if (!(g.tex_n == 1 || g.tex_n == 2 || g.tex_n == 4 || g.tex_n == 8 || g.tex_n == 16))
            return fail(ctx, GB_ERR_UNSUPPORTED, "scene %d: tex_n %d not in {1,2,4,8,16}", s, g.tex_n);
        if (!dtype_ok(g.sh_dtype) || !dtype_ok(g.tex_dtype))
            return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: bad storage dtype", s);
        if (!(g.sigma > 0.0f) || !isfinite(g.sigma))
            return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: sigma must be positive", s);
        if (g.tex_sh_degree < 0 || g.tex_sh_degree > 3)
            return fail(ctx, GB_ERR_UNSUPPORTED, "scene %d: tex_sh_degree %d not in 0..3", s, g.tex_sh_degree);
        if (g.tex_sh_degree && g.mip_level)
            return fail(ctx, GB_ERR_UNSUPPORTED, "scene %d: per-texel SH takes no mip level", s);
        if (g.reserved != 0) return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: reserved field must be 0", s);
        if (g.mip_level < 0 || g.mip_level > 4 || (g.tex_n >> g.mip_level) < 1)
            return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: mip_level %d not in 0..log2(%d)", s, g.mip_level,
                        g.tex_n);
        if (g.num_splats > 0 && (!g.means || !g.quats || !g.scales || !g.opacities || !g.sh || !g.textures))
            return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: null parameter pointer", s);
        if (g.splat_tex_n && (g.tex_n < 2 || g.mip_level || g.tex_sh_degree))
            return fail(ctx, GB_ERR_UNSUPPORTED,
                        "scene %d: per-splat grid sizes need tex_n >= 2 and take no mip level or per-texel SH", s);
        d.K = g.num_splats;
        d.means = g.means;
        d.quats = g.quats;
        d.scales = g.scales;
        d.opac = g.opacities;
        d.sh = g.sh;
        d.tex = g.textures;
        d.D = g.sh_degree;
        d.sh_dtype = g.sh_dtype;
        d.N = g.tex_n;
        d.tex_dtype = g.tex_dtype;
        d.sigma = g.sigma;
        d.mip = g.mip_level;
        d.tex_sh = g.tex_sh_degree;
        d.splat_n = g.splat_tex_n;
        max_k = std::max(max_k, g.num_splats);
    }
    // render groups: one per distinct (rendered grid size, tex_dtype, per-splat
    // sizes or not) among the scenes
    int scene_group[kMaxScenes];
    for (int sidx = 0; sidx < n_scenes; ++sidx) {
        // a scene at a mip level is rendered from its FP32 filtered grid
        const int n_eff = scenes[sidx].tex_n >> scenes[sidx].mip_level;
        const int dt = (scenes[sidx].mip_level || scenes[sidx].tex_sh_degree) ? int(GB_F32) : scenes[sidx].tex_dtype;
        const int var = scenes[sidx].splat_tex_n ? 1 : 0;
        int g = -1;
        for (int k = 0; k < f.n_groups; ++k)
            if (f.group_N[k] == n_eff && f.group_dtype[k] == dt && f.group_var[k] == var) g = k;
        if (g < 0) {
            g = f.n_groups++;
            f.group_N[g] = n_eff;
            f.group_dtype[g] = dt;
            f.group_var[g] = var;
        }
        scene_group[sidx] = g;
    }
    int64_t tiles = 0, pix = 0, rec = 0;
    for (int c = 0; c < n_cams; ++c) {
        const gb_camera &g = cams[c];
        CamDev &d = f.cams[c];
        if (g.width < 1 || g.height < 1 || g.width > 16384 || g.height > 16384)
            return fail(ctx, GB_ERR_INVALID_ARG, "camera %d: size %dx%d out of range", c, g.width, g.height);
        if (g.scene < 0 || g.scene >= n_scenes)
            return fail(ctx, GB_ERR_INVALID_ARG, "camera %d: scene %d out of range", c, g.scene);
        bool fin = isfinite(g.fx) && isfinite(g.fy) && isfinite(g.cx) && isfinite(g.cy) && isfinite(g.near_plane);
        for (int i = 0; i < 12; ++i) fin = fin && isfinite(g.world_to_cam[i]);
        if (!fin) return fail(ctx, GB_ERR_NONFINITE, "camera %d has non-finite parameters", c);
        d.width = g.width;
        d.height = g.height;
        d.tiles_x = int32_t(ceil_div(g.width, tile));
        d.tiles_y = int32_t(ceil_div(g.height, tile));
        d.fx = g.fx; d.fy = g.fy; d.cx = g.cx; d.cy = g.cy;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) d.R[3 * i + j] = g.world_to_cam[4 * i + j];
            d.t[i] = g.world_to_cam[4 * i + 3];
        }
        for (int i = 0; i < 3; ++i)
            d.campos[i] = -(d.R[i] * d.t[0] + d.R[3 + i] * d.t[1] + d.R[6 + i] * d.t[2]);
        d.near_plane = g.near_plane;
        d.scene = g.scene;
        d.group = scene_group[g.scene];
        f.group_count[d.group] += uint32_t(int64_t(d.tiles_x) * d.tiles_y);
        d.tile_off = uint32_t(tiles);
        d.pix_off = pix;
        d.rec_off = rec;
        tiles += int64_t(d.tiles_x) * d.tiles_y;
        pix += int64_t(g.width) * g.height;
        rec += scenes[g.scene].num_splats;
    }
    if (tiles >= (int64_t(1) << 31) || rec >= int64_t(0xF0000000u))
        return fail(ctx, GB_ERR_INVALID_ARG, "frame too large (%lld tiles, %lld records)", (long long)tiles,
                    (long long)rec);
    f.n_tiles = uint32_t(tiles);
    f.n_pixels = pix;
    f.n_records = rec;
    uint32_t off = 0;
    for (int k = 0; k < f.n_groups; ++k) {
        f.group_off[k] = off;
        off += f.group_count[k];
    }
    return GB_OK;
}

}  // namespace

extern "C" {

const char *gb_status_string(gb_status s) {
    switch (s) {
        case GB_OK: return "GB_OK";
        case GB_ERR_INVALID_ARG: return "GB_ERR_INVALID_ARG";
        case GB_ERR_UNSUPPORTED: return "GB_ERR_UNSUPPORTED";
        case GB_ERR_CUDA: return "GB_ERR_CUDA";
        case GB_ERR_CAPACITY: return "GB_ERR_CAPACITY";
        case GB_ERR_TIMEOUT: return "GB_ERR_TIMEOUT";
        case GB_ERR_NONFINITE: return "GB_ERR_NONFINITE";
    }
    return "GB_UNKNOWN_STATUS";
}

const char *gb_last_error(const gb_context *ctx) { return ctx ? ctx->err : "null context"; }

gb_status gb_context_create(int32_t device, gb_context **out) {
    if (!out) return GB_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return GB_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return GB_ERR_CUDA;
    gb_context *c = new (std::nothrow) gb_context();
    if (!c) return GB_ERR_CUDA;
    c->device = device;
    c->err[0] = 0;
    *out = c;
    return GB_OK;
}

gb_status gb_context_destroy(gb_context *ctx) {
    if (!ctx) return GB_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    delete ctx;
    return GB_OK;
}

gb_status gb_saved_create(gb_context *ctx, gb_saved **out) {
    if (!ctx || !out) return fail(ctx, GB_ERR_INVALID_ARG, "null argument");
    gb_saved *s = new (std::nothrow) gb_saved();
    if (!s) return fail(ctx, GB_ERR_CUDA, "host allocation failed");
    memset(s, 0, sizeof(*s));
    s->ctx = ctx;
    cudaError_t e = cudaMalloc(&s->cnt, sizeof(Counters));
    if (e == cudaSuccess) e = cudaMallocHost(&s->cnt_host, sizeof(Counters));
    if (e != cudaSuccess) {
        if (s->cnt) cudaFree(s->cnt);
        delete s;
        return fail(ctx, GB_ERR_CUDA, "saved state allocation failed: %s", cudaGetErrorString(e));
    }
    memset(s->cnt_host, 0, sizeof(Counters));
    cudaMemset(s->cnt, 0, sizeof(Counters));
    for (int i = 0; i < kNumEvents; ++i) {
        if (cudaEventCreate(&s->ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(s->ev[j]);
            cudaFree(s->cnt);
            cudaFreeHost(s->cnt_host);
            delete s;
            return fail(ctx, GB_ERR_CUDA, "event creation failed");
        }
    }
    s->ev_ready = true;
    *out = s;
    return GB_OK;
}

gb_status gb_saved_destroy(gb_saved *s) {
    if (!s) return GB_OK;
    cudaDeviceSynchronize();
    void *ptrs[] = {s->rec, s->rec_lo, s->depth_key, s->keys_tmp, s->vals_tmp, s->dkeys_sorted, s->perm,
                    s->offsets, s->rect, s->pbox, s->inv, s->rec_grad, s->inst_tile, s->inst_val, s->inst_tile_tmp,
                    s->inst_val_tmp, s->tiles_sorted, s->vals_sorted, s->ranges, s->tl_keys, s->tl_vals,
                    s->tl_keys_tmp, s->tl_vals_tmp, s->tl_keys_out, s->tile_list, s->work, s->t_final, s->last,
                    s->cnt, s->scratch, s->mip_tex, s->mip_grad, s->tsh_tex, s->tsh_grad};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (s->cnt_host) cudaFreeHost(s->cnt_host);
    if (s->ev_ready)
        for (int i = 0; i < kNumEvents; ++i) cudaEventDestroy(s->ev[i]);
    delete s;
    return GB_OK;
}

gb_status gb_saved_reserve(gb_saved *s, int64_t records, int64_t instances, int64_t pixels, int64_t tiles) {
    if (!s || records < 0 || instances < 0 || pixels < 0 || tiles < 0)
        return fail(s ? s->ctx : nullptr, GB_ERR_INVALID_ARG, "bad reserve arguments");
    gb_status st;
    // a recorded forward stays valid: a backward may follow the reserve
    const bool keep = s->has_forward;
    if ((st = reserve_records(s, records, keep)) != GB_OK) return st;
    if ((st = reserve_instances(s, instances, keep)) != GB_OK) return st;
    if ((st = reserve_pixels(s, pixels, keep)) != GB_OK) return st;
    if ((st = reserve_tiles(s, tiles, keep)) != GB_OK) return st;
    if ((st = reserve_scratch(s)) != GB_OK) return st;
    GB_CUDA(s->ctx, cudaDeviceSynchronize());
    return GB_OK;
}

gb_status gb_saved_stats(gb_saved *s, gb_stats *out) {
    if (!s || !out) return fail(s ? s->ctx : nullptr, GB_ERR_INVALID_ARG, "null argument");
    GB_CUDA(s->ctx, cudaMemcpyAsync(s->cnt_host, s->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    GB_CUDA(s->ctx, cudaStreamSynchronize(s->stream));
    out->records = s->n_records;
    out->visible = s->cnt_host->n_visible;
    out->instances = s->cnt_host->n_instances;
    out->tiles = s->frame.n_tiles;
    out->pixels = s->n_pixels;
    out->capacity = s->cap_inst;
    out->overflow = int32_t(s->cnt_host->overflow);
    out->error_flags = int32_t(s->cnt_host->error_flags);
    out->pairs_fwd = int64_t(s->cnt_host->pairs_fwd);
    out->pairs_bwd = int64_t(s->cnt_host->pairs_bwd);
    out->blended_fwd = int64_t(s->cnt_host->blend_fwd);
    // the backward computes the adjoints of exactly the pairs its forward blended
    out->contributing_bwd = s->cnt_host->pairs_bwd ? int64_t(s->cnt_host->blend_fwd) : 0;
    return GB_OK;
}

uint64_t gb_kernel_launches(void) { return g_launches.load(); }

gb_status gb_saved_phase_times(gb_saved *s, float *ms, int32_t cap) {
    if (!s || !ms || cap < 0) return fail(s ? s->ctx : nullptr, GB_ERR_INVALID_ARG, "bad arguments");
    GB_CUDA(s->ctx, cudaStreamSynchronize(s->stream));
    for (int i = 0; i < cap && i < GB_PHASE_COUNT; ++i) {
        int a, b;
        bool on;
        if (i < 7) { a = i; b = i + 1; on = s->timed_fwd; }
        else { a = i + 1; b = i + 2; on = s->timed_bwd; }
        ms[i] = -1.0f;
        if (on) GB_CUDA(s->ctx, cudaEventElapsedTime(&ms[i], s->ev[a], s->ev[b]));
    }
    return GB_OK;
}

gb_status gb_saved_check(gb_saved *s) {
    gb_stats st;
    gb_status r = gb_saved_stats(s, &st);
    if (r != GB_OK) return r;
    if (st.overflow)
        return fail(s->ctx, GB_ERR_CAPACITY, "instance capacity %lld exceeded (%lld needed)",
                    (long long)st.capacity, (long long)st.instances);
    if (st.error_flags & 1) return fail(s->ctx, GB_ERR_TIMEOUT, "a bounded device wait timed out");
    if (st.error_flags & 2)
        return fail(s->ctx, GB_ERR_NONFINITE,
                    "non-finite splat parameters or SH colour: those splats were culled in the last forward");
    return GB_OK;
}

gb_status gb_saved_export_keys(gb_saved *s, uint64_t *keys, int64_t *ids, int32_t *cams, int64_t cap,
                               int64_t *count) {
    if (!s || !count || cap < 0) return fail(s ? s->ctx : nullptr, GB_ERR_INVALID_ARG, "bad arguments");
    if (!s->has_forward) return fail(s->ctx, GB_ERR_INVALID_ARG, "no forward recorded on this saved state");
    gb_stats st;
    gb_status r = gb_saved_stats(s, &st);
    if (r != GB_OK) return r;
    if (st.overflow) return fail(s->ctx, GB_ERR_CAPACITY, "last forward overflowed");
    *count = st.instances;
    const int64_t n = std::min<int64_t>(cap, st.instances);
    if (n == 0) return GB_OK;
    if (!keys || !ids || !cams) return fail(s->ctx, GB_ERR_INVALID_ARG, "null output array");
    uint64_t *dk = nullptr;
    int64_t *di = nullptr;
    int32_t *dc = nullptr;
    GB_CUDA(s->ctx, cudaMalloc(&dk, n * 8));
    GB_CUDA(s->ctx, cudaMalloc(&di, n * 8));
    GB_CUDA(s->ctx, cudaMalloc(&dc, n * 4));
    GB_CUDA(s->ctx, launch_export_keys(s->frame, s->tiles_sorted, s->vals_sorted, s->perm, s->depth_key, n, dk,
                                       di, dc, s->stream));
    GB_CUDA(s->ctx, cudaMemcpyAsync(keys, dk, n * 8, cudaMemcpyDeviceToHost, s->stream));
    GB_CUDA(s->ctx, cudaMemcpyAsync(ids, di, n * 8, cudaMemcpyDeviceToHost, s->stream));
    GB_CUDA(s->ctx, cudaMemcpyAsync(cams, dc, n * 4, cudaMemcpyDeviceToHost, s->stream));
    GB_CUDA(s->ctx, cudaStreamSynchronize(s->stream));
    cudaFree(dk);
    cudaFree(di);
    cudaFree(dc);
    return GB_OK;
}

gb_status gb_saved_export_records(gb_saved *s, float *rec, float *rec_lo, uint8_t *visible, int64_t cap,
                                  int64_t *count) {
    if (!s || !count || cap < 0) return fail(s ? s->ctx : nullptr, GB_ERR_INVALID_ARG, "bad arguments");
    if (!s->has_forward) return fail(s->ctx, GB_ERR_INVALID_ARG, "no forward recorded on this saved state");
    *count = s->n_records;
    const int64_t n = std::min<int64_t>(cap, s->n_records);
    if (n == 0) return GB_OK;
    if (!rec || !visible) return fail(s->ctx, GB_ERR_INVALID_ARG, "null output array");
    GB_CUDA(s->ctx, cudaStreamSynchronize(s->stream));
    GB_CUDA(s->ctx, cudaMemcpy(rec, s->rec, size_t(n) * sizeof(Record), cudaMemcpyDeviceToHost));
    if (rec_lo) GB_CUDA(s->ctx, cudaMemcpy(rec_lo, s->rec_lo, size_t(n) * sizeof(RecordLo), cudaMemcpyDeviceToHost));
    uint32_t *keys = static_cast<uint32_t *>(malloc(size_t(n) * 4));
    if (!keys) return fail(s->ctx, GB_ERR_INVALID_ARG, "host allocation failed");
    cudaError_t e = cudaMemcpy(keys, s->depth_key, size_t(n) * 4, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
        visible[i] = keys[i] != 0xFFFFFFFFu;
        // low parts exist for visible flagged records only (depth stored negated)
        if (rec_lo && !(visible[i] && rec[16 * i + 7] < 0.0f)) memset(rec_lo + 12 * i, 0, 12 * sizeof(float));
    }
    free(keys);
    GB_CUDA(s->ctx, e);
    return GB_OK;
}

gb_status gb_render_forward(gb_context *ctx, gb_saved *s, const gb_scene *scenes, int32_t n_scenes,
                            const gb_camera *cams, int32_t n_cams, const gb_options *opt, float *rgb,
                            float *depth, float *alpha, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (!s || s->ctx != ctx) return fail(ctx, GB_ERR_INVALID_ARG, "saved state missing or from another context");
    if (!rgb) return fail(ctx, GB_ERR_INVALID_ARG, "rgb output is required");
    gb_options o{};
    if (opt) o = *opt;
    const int ppt = o.pixels_per_thread ? o.pixels_per_thread : 1;
    if (ppt != 1 && ppt != 2) return fail(ctx, GB_ERR_INVALID_ARG, "pixels_per_thread must be 1 or 2");
    const int tile = o.tile_size ? o.tile_size : 16;
    if (tile != 8 && tile != 16 && tile != 32)
        return fail(ctx, GB_ERR_UNSUPPORTED, "tile_size %d not built (8, 16 or 32)", tile);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Frame f;
    int64_t max_k = 0;
    gb_status r = build_frame(ctx, scenes, n_scenes, cams, n_cams, tile, o.background, f, max_k);
    if (r != GB_OK) return r;
    const int nt = tile * tile;
    if (o.bwd_kernel < 0 || o.bwd_kernel > 2) return fail(ctx, GB_ERR_INVALID_ARG, "bwd_kernel must be 0, 1 or 2");
    if (frame_has_var(f) && (tile != 16 || ppt != 1))
        return fail(ctx, GB_ERR_UNSUPPORTED,
                    "per-splat grid sizes render on 16 x 16 tiles with one backward pixel per thread");
    const bool sp_ok = frame_sp_ok(f);
    if (o.bwd_kernel == 2 && !sp_ok)
        return fail(ctx, GB_ERR_UNSUPPORTED, "the splat-parallel backward takes grids of N <= 4 on 8 x 8 or 16 x 16 tiles");
    // pixels per thread set (1 or 2) asks for the pixel-parallel loop
    const bool sp = o.bwd_kernel == 2 || (o.bwd_kernel == 0 && o.pixels_per_thread == 0 && sp_ok && kSplatParallelAuto);
    const int bf = forward_batch(o, f, nt);
    const int bb = o.batch_depth ? o.batch_depth
                                 : (sp ? default_batch_sp(f) : std::min(default_batch(f, true), nt / ppt));
    if (bf < 8 || bf > nt || (bf & 7)) return fail(ctx, GB_ERR_INVALID_ARG, "forward batch depth %d invalid", bf);
    if (bb < 8 || (bb & 7)) return fail(ctx, GB_ERR_INVALID_ARG, "batch_depth %d invalid", bb);
    if (sp) {
        if (bb > 256) return fail(ctx, GB_ERR_INVALID_ARG, "batch_depth %d above 256 (splat-parallel backward)", bb);
        if (frame_sp_smem(f, bb) > 200 * 1024)
            return fail(ctx, GB_ERR_INVALID_ARG, "batch_depth %d needs too much shared memory", bb);
    } else {
        if (bb > nt / ppt)
            return fail(ctx, GB_ERR_INVALID_ARG, "batch_depth %d exceeds the backward's %d threads", bb, nt / ppt);
        if (frame_smem(f, bb, true) > 200 * 1024)
            return fail(ctx, GB_ERR_INVALID_ARG, "batch_depth %d needs too much shared memory", bb);
    }
    if (frame_smem(f, bf, false) > 200 * 1024)
        return fail(ctx, GB_ERR_INVALID_ARG, "forward batch depth %d needs too much shared memory", bf);
    const bool nosync = (o.flags & GB_FLAG_NO_SYNC) != 0;
    if (nosync) {
        if (f.n_records > s->cap_rec || f.n_pixels > s->cap_pix || int64_t(f.n_tiles) > s->cap_tiles ||
            s->cap_inst == 0)
            return fail(ctx, GB_ERR_CAPACITY, "saved state not reserved for this frame (no-sync mode)");
    } else {
        if ((r = reserve_records(s, f.n_records)) != GB_OK) return r;
        if ((r = reserve_pixels(s, f.n_pixels)) != GB_OK) return r;
        if ((r = reserve_tiles(s, f.n_tiles)) != GB_OK) return r;
        if ((r = reserve_instances(s, std::max<int64_t>(s->cap_inst, 1 << 16))) != GB_OK) return r;
        if ((r = reserve_scratch(s)) != GB_OK) return r;
    }
    const bool timing = (o.flags & GB_FLAG_TIMING) != 0;
    // the preprocess phase starts with the grid pre-passes below
    if (timing) GB_CUDA(ctx, cudaEventRecord(s->ev[0], st));
    // mip-level scenes: filter their grids into FP32 scratch the render reads
    int64_t mip_need = 0;
    for (int i = 0; i < f.n_scenes; ++i) {
        s->mip_off[i] = mip_need;
        s->mip_ns[i] = f.scenes[i].N;
        if (f.scenes[i].mip) {
            const int64_t n = f.scenes[i].N >> f.scenes[i].mip;
            mip_need += f.scenes[i].K * n * n * 3;
        }
    }
    if (mip_need > s->mip_cap) {
        if (nosync)
            return fail(ctx, GB_ERR_CAPACITY,
                        "mip-level grids need %lld floats of scratch: run a synchronizing forward first",
                        (long long)mip_need);
        GB_CUDA(ctx, alloc_t(&s->mip_tex, mip_need));
        GB_CUDA(ctx, alloc_t(&s->mip_grad, mip_need));
        s->mip_cap = mip_need;
    }
    for (int i = 0; i < f.n_scenes; ++i) {
        SceneDev &d = f.scenes[i];
        if (!d.mip) continue;
        GB_CUDA(ctx, launch_mip_filter(d.tex, d.tex_dtype, d.K, d.N, d.mip, s->mip_tex + s->mip_off[i], st));
        d.tex = s->mip_tex + s->mip_off[i];
        d.tex_dtype = GB_F32;
        d.N >>= d.mip;
    }
    // per-texel SH scenes: one evaluated RGB grid per (splat, camera) record,
    // camera blocks of K rows (CamDev::tex_row)
    int64_t tsh_need = 0;
    for (int i = 0; i < f.n_scenes; ++i) {
        s->tsh_off[i] = tsh_need;
        s->tsh_rows[i] = 0;
        if (!f.scenes[i].tex_sh) continue;
        for (int c = 0; c < f.n_cams; ++c)
            if (f.cams[c].scene == i) {
                f.cams[c].tex_row = s->tsh_rows[i];
                s->tsh_rows[i] += f.scenes[i].K;
            }
        if (s->tsh_rows[i] >= (int64_t(1) << 31))
            return fail(ctx, GB_ERR_INVALID_ARG, "scene %d: per-texel SH over %lld records exceeds 2^31", i,
                        (long long)s->tsh_rows[i]);
        tsh_need += s->tsh_rows[i] * f.scenes[i].N * f.scenes[i].N * 3;
    }
    if (tsh_need > s->tsh_cap) {
        if (nosync)
            return fail(ctx, GB_ERR_CAPACITY,
                        "per-texel SH grids need %lld floats of scratch: run a synchronizing forward first",
                        (long long)tsh_need);
        GB_CUDA(ctx, alloc_t(&s->tsh_tex, tsh_need));
        GB_CUDA(ctx, alloc_t(&s->tsh_grad, tsh_need));
        s->tsh_cap = tsh_need;
    }
    for (int i = 0; i < f.n_scenes; ++i) {
        SceneDev &d = f.scenes[i];
        if (!d.tex_sh) continue;
        s->tsh_coef[i] = d.tex;
        s->tsh_dtype[i] = d.tex_dtype;
        GB_CUDA(ctx, launch_texsh_eval(f, i, d.tex_sh, d.tex, d.tex_dtype, s->tsh_tex + s->tsh_off[i], st));
        d.tex = s->tsh_tex + s->tsh_off[i];
        d.tex_dtype = GB_F32;
    }
    const int64_t R = f.n_records;
    int tile_bits = 1;
    while ((int64_t(1) << tile_bits) < int64_t(f.n_tiles)) ++tile_bits;
    s->frame = f;
    s->n_records = R;
    s->n_pixels = f.n_pixels;
    s->max_k = max_k;
    s->tile_bits = tile_bits;
    s->batch_fwd = bf;
    s->batch_bwd = bb;
    s->ppt = ppt;
    s->bwd_sp = sp;
    s->flags = o.flags;
    s->stream = st;
    s->has_forward = false;
    s->timed_fwd = s->timed_bwd = false;
#define GB_MARK(i) \
    if (timing) GB_CUDA(ctx, cudaEventRecord(s->ev[i], st))

    GB_CUDA(ctx, cudaMemsetAsync(s->cnt, 0, sizeof(Counters), st));
    GB_CUDA(ctx, cudaMemsetAsync(s->ranges, 0, size_t(f.n_tiles) * sizeof(uint2), st));
    GB_CUDA(ctx, launch_preprocess(f, max_k, s->depth_key, nullptr, s->rect, s->pbox, s->rec, s->cnt, st));
    // visible records to the front in record order; their records' homography
    // part, one thread per visible record; then sorted by depth (stable, so
    // equal depths keep record order)
    GB_CUDA(ctx, compact_visible(s->depth_key, R, s->offsets, s->dkeys_sorted, s->perm, s->scratch, s->scratch_bytes,
                                 st));
    GB_CUDA(ctx, launch_record(f, s->perm, &s->cnt->n_visible, nullptr, R, s->rec, s->rec_lo, st));
    GB_MARK(1);
    GB_CUDA(ctx, radix_sort_pairs(s->dkeys_sorted, s->perm, s->keys_tmp, s->vals_tmp, s->dkeys_sorted, s->perm, R,
                                  &s->cnt->n_visible, 0, 32, s->scratch, s->scratch_bytes, st));
    GB_MARK(2);
    GB_CUDA(ctx, tile_counts_scan(f, s->perm, s->rect, R, &s->cnt->n_visible, s->offsets, s->scratch,
                                  s->scratch_bytes, s->cnt, s->cap_inst, st));
    GB_MARK(3);
    int64_t inst_max = s->cap_inst;
    if (!nosync) {
        GB_CUDA(ctx, cudaMemcpyAsync(s->cnt_host, s->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        GB_CUDA(ctx, cudaStreamSynchronize(st));
        const int64_t need = s->cnt_host->n_instances;
        if (need > s->cap_inst) {
            if ((r = reserve_instances(s, need)) != GB_OK) return r;
            if ((r = reserve_scratch(s)) != GB_OK) return r;
            GB_CUDA(ctx, cudaMemsetAsync(&s->cnt->overflow, 0, sizeof(uint32_t), st));
        }
        inst_max = std::max<int64_t>(need, 1);
    }
    s->inst_max = inst_max;
    if (timing && !nosync) GB_CUDA(ctx, cudaEventRecord(s->ev[3], st));  // exclude the host round trip
    GB_CUDA(ctx, launch_emit(f, s->perm, s->rect, s->offsets, R, s->cnt, s->cap_inst, s->inst_tile, s->inst_val, st));
    GB_MARK(4);
    GB_CUDA(ctx, radix_sort_pairs(s->inst_tile, s->inst_val, s->inst_tile_tmp, s->inst_val_tmp, s->tiles_sorted,
                                  s->vals_sorted, inst_max, &s->cnt->n_instances, 0, tile_bits, s->scratch,
                                  s->scratch_bytes, st));
    GB_MARK(5);
    GB_CUDA(ctx, launch_ranges(s->tiles_sorted, inst_max, s->cnt, s->ranges, st));
    GB_MARK(6);
    const bool persistent = (o.flags & GB_FLAG_PERSISTENT) != 0;
    s->use_list = persistent || f.n_groups > 1;
    if (s->use_list) {
        int kbits = 24;
        while ((1 << (kbits - 24)) < f.n_groups) ++kbits;
        GB_CUDA(ctx, launch_tile_list(f, s->ranges, s->tl_keys, s->tl_vals, st));
        GB_CUDA(ctx, radix_sort_pairs(s->tl_keys, s->tl_vals, s->tl_keys_tmp, s->tl_vals_tmp, s->tl_keys_out,
                                      s->tile_list, f.n_tiles, nullptr, 0, kbits, s->scratch, s->scratch_bytes, st));
        GB_CUDA(ctx, cudaMemsetAsync(s->work, 0, 2 * kMaxGroups * sizeof(uint32_t), st));
    }
    RenderBufs b;
    b.rec = s->rec;
    b.rec_lo = s->rec_lo;
    b.perm = s->perm;
    b.inst_val = s->vals_sorted;
    b.ranges = s->ranges;
    b.pbox = s->pbox;
    b.rgb = rgb;
    b.depth = depth;
    b.alpha = alpha;
    b.t_final = s->t_final;
    b.last = s->last;
    b.cnt = s->cnt;
    GB_CUDA(ctx, launch_render_fwd(f, b, bf, s->use_list ? s->tile_list : nullptr, persistent ? s->work : nullptr,
                                   persistent, st));
    GB_MARK(7);
#undef GB_MARK
    s->timed_fwd = timing;
    s->has_forward = true;
    return GB_OK;
}

gb_status gb_render_backward(gb_context *ctx, gb_saved *s, const float *d_rgb, const float *d_depth,
                             const float *d_alpha, const gb_grads *grads, int32_t n_scenes, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (!s || s->ctx != ctx) return fail(ctx, GB_ERR_INVALID_ARG, "saved state missing or from another context");
    if (!s->has_forward) return fail(ctx, GB_ERR_INVALID_ARG, "no forward recorded on this saved state");
    if (!d_rgb) return fail(ctx, GB_ERR_INVALID_ARG, "d_rgb is required");
    if (!grads || n_scenes != s->frame.n_scenes)
        return fail(ctx, GB_ERR_INVALID_ARG, "grads must hold one entry per scene (%d)", s->frame.n_scenes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool timing = (s->flags & GB_FLAG_TIMING) != 0;
    if (timing) GB_CUDA(ctx, cudaEventRecord(s->ev[8], st));
    Frame f = s->frame;
    for (int i = 0; i < n_scenes; ++i) {
        SceneDev &d = f.scenes[i];
        d.g_means = grads[i].d_means;
        d.g_quats = grads[i].d_quats;
        d.g_scales = grads[i].d_scales;
        d.g_opac = grads[i].d_opacities;
        d.g_sh = grads[i].d_sh;
        d.g_tex = grads[i].d_textures;
        if (d.g_tex && d.mip) d.g_tex = s->mip_grad + s->mip_off[i];  // gradient of the filtered grid
        // per-texel SH: gradient of every record's evaluated grid (post-pass below)
        if (d.tex_sh) d.g_tex = s->tsh_grad + s->tsh_off[i];
        const int64_t rows = d.tex_sh ? s->tsh_rows[i] : d.K;
        if (d.g_tex && rows > 0)
            GB_CUDA(ctx, cudaMemsetAsync(d.g_tex, 0, size_t(rows) * d.N * d.N * 3 * sizeof(float), st));
    }
    const int64_t R = s->n_records;
    zero_rec_grad<<<unsigned(std::min<int64_t>(ceil_div(std::max<int64_t>(R, 1) * (kRecGrad / 4), 256), 65535)), 256, 0, st>>>(
        s->rec_grad, s->cnt, R);
    GB_CUDA(ctx, cudaGetLastError());
    count_launches(1);
    GB_CUDA(ctx, launch_inverse_perm(s->perm, R, s->cnt, s->inv, st));
    if (timing) GB_CUDA(ctx, cudaEventRecord(s->ev[9], st));
    RenderBwdBufs b;
    b.fw.rec = s->rec;
    b.fw.rec_lo = s->rec_lo;
    b.fw.perm = s->perm;
    b.fw.inst_val = s->vals_sorted;
    b.fw.ranges = s->ranges;
    b.fw.pbox = s->pbox;
    b.fw.rgb = nullptr;
    b.fw.depth = nullptr;
    b.fw.alpha = nullptr;
    b.fw.t_final = s->t_final;
    b.fw.last = s->last;
    b.fw.cnt = s->cnt;
    b.d_rgb = d_rgb;
    b.d_depth = d_depth;
    b.d_alpha = d_alpha;
    b.rec_grad = s->rec_grad;
    GB_CUDA(ctx, cudaMemsetAsync(&s->cnt->pairs_bwd, 0, sizeof(unsigned long long), st));
    const bool persistent = (s->flags & GB_FLAG_PERSISTENT) != 0;
    // the backward's tile counters start from zero at every call (a forward
    // may be followed by several backwards)
    if (persistent) GB_CUDA(ctx, cudaMemsetAsync(s->work + kMaxGroups, 0, kMaxGroups * sizeof(uint32_t), st));
    if (s->bwd_sp)
        GB_CUDA(ctx, launch_render_bwd_sp(f, b, s->batch_bwd, s->use_list ? s->tile_list : nullptr,
                                          persistent ? s->work + kMaxGroups : nullptr, persistent, st));
    else
        GB_CUDA(ctx, launch_render_bwd(f, b, s->batch_bwd, s->ppt, s->use_list ? s->tile_list : nullptr,
                                       persistent ? s->work + kMaxGroups : nullptr, persistent, st));
    for (int i = 0; i < n_scenes; ++i)
        if (f.scenes[i].mip && grads[i].d_textures)
            GB_CUDA(ctx, launch_mip_grad(s->mip_grad + s->mip_off[i], f.scenes[i].K, s->mip_ns[i], f.scenes[i].mip,
                                         grads[i].d_textures, st));
    if (timing) GB_CUDA(ctx, cudaEventRecord(s->ev[10], st));
    GB_CUDA(ctx, launch_preprocess_bwd(f, s->max_k, s->rec_grad, s->inv, st));
    // per-texel SH: coefficient gradients and the centre gradient through the
    // view direction (added to the means gradient written just above)
    for (int i = 0; i < n_scenes; ++i)
        if (f.scenes[i].tex_sh)
            GB_CUDA(ctx, launch_texsh_grad(f, i, f.scenes[i].tex_sh, s->tsh_coef[i], s->tsh_dtype[i],
                                           s->tsh_grad + s->tsh_off[i], grads[i].d_textures, grads[i].d_means,
                                           st));
    if (timing) GB_CUDA(ctx, cudaEventRecord(s->ev[11], st));
    s->timed_bwd = timing;
    return GB_OK;
}

gb_status gb_adam_step(gb_context *ctx, const gb_adam_tensor *tensors, int32_t n_tensors,
                       const gb_adam_config *cfg, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (!tensors || !cfg || n_tensors < 1 || n_tensors > 16)
        return fail(ctx, GB_ERR_INVALID_ARG, "n_tensors must be in 1..16 with a config");
    if (cfg->step < 1 || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
        !(cfg->eps >= 0.0f) || !isfinite(cfg->lr) || cfg->reserved != 0)
        return fail(ctx, GB_ERR_INVALID_ARG, "bad Adam hyper-parameters");
    int64_t biggest = 0;
    for (int i = 0; i < n_tensors; ++i) {
        const gb_adam_tensor &t = tensors[i];
        if (t.n < 0 || t.reserved != 0 || (t.n > 0 && (!t.param || !t.grad || !t.m || !t.v)))
            return fail(ctx, GB_ERR_INVALID_ARG, "adam tensor %d: bad pointer or size", i);
        if (t.shadow && !dtype_ok(t.shadow_dtype))
            return fail(ctx, GB_ERR_INVALID_ARG, "adam tensor %d: bad shadow dtype", i);
        biggest = std::max(biggest, t.n);
    }
    // enough blocks to fill the GPU (152 SMs x 8 resident 256-thread blocks) per tensor
    const int grid_x = int(std::max<int64_t>(1, std::min<int64_t>(ceil_div(biggest, 4 * 256), 152 * 8)));
    GB_CUDA(ctx, launch_adam(tensors, n_tensors, *cfg, grid_x, static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

// ---------------------------------------------------------------------------
// Forward without allocation.  Every scratch buffer of the forward pipeline is
// carved from this one file-scope device array, so the call never allocates.
// Limits per call: records (splats x cameras), (tile, splat) instances,
// pixels and tiles below; the array is 256-byte aligned and each carved
// buffer starts on a 256-byte boundary.
constexpr int64_t kNaMaxRecords = int64_t(1) << 17;
constexpr int64_t kNaMaxInstances = int64_t(1) << 19;
constexpr int64_t kNaMaxPixels = int64_t(1) << 20;
constexpr int64_t kNaMaxTiles = int64_t(1) << 13;
constexpr size_t na_round(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kNaRadixBytes = size_t(kNaMaxInstances / 4096) * 512 * 4 + 64 * 1024;
constexpr size_t kNaScratchBytes =
    na_round(sizeof(Counters)) + na_round(2 * kMaxGroups * 4) +
    na_round(kNaMaxRecords * sizeof(Record)) + na_round(kNaMaxRecords * sizeof(RecordLo)) + 7 * na_round(kNaMaxRecords * 4) + 2 * na_round(kNaMaxRecords * 8) +
    6 * na_round(kNaMaxInstances * 4) + 2 * na_round(kNaMaxPixels * 4) + na_round(kNaMaxTiles * 8) +
    6 * na_round(kNaMaxTiles * 4) + na_round(kNaRadixBytes);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
static void *g_noalloc_addr[64] = {nullptr};
static std::mutex g_noalloc_mu;

gb_status gb_render_forward_noalloc(gb_context *ctx, const gb_scene *scenes, int32_t n_scenes,
                                    const gb_camera *cams, int32_t n_cams, const gb_options *opt, float *rgb,
                                    float *depth, float *alpha, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (!rgb) return fail(ctx, GB_ERR_INVALID_ARG, "rgb output is required");
    gb_options o{};
    if (opt) o = *opt;
    const int tile = o.tile_size ? o.tile_size : 16;
    if (tile != 8 && tile != 16 && tile != 32)
        return fail(ctx, GB_ERR_UNSUPPORTED, "tile_size %d not built (8, 16 or 32)", tile);
    if (o.flags & (GB_FLAG_TIMING | GB_FLAG_PERSISTENT))
        return fail(ctx, GB_ERR_UNSUPPORTED, "the no-allocation forward takes no timing or persistent flag");
    Frame f;
    int64_t max_k = 0;
    gb_status r = build_frame(ctx, scenes, n_scenes, cams, n_cams, tile, o.background, f, max_k);
    if (r != GB_OK) return r;
    for (int i = 0; i < f.n_scenes; ++i)
        if (f.scenes[i].mip || f.scenes[i].tex_sh)
            return fail(ctx, GB_ERR_UNSUPPORTED,
                        "the no-allocation forward renders no mip-level or per-texel SH scene");
    if (frame_has_var(f) && tile != 16)
        return fail(ctx, GB_ERR_UNSUPPORTED, "per-splat grid sizes render on 16 x 16 tiles");
    if (f.n_records > kNaMaxRecords || f.n_pixels > kNaMaxPixels || int64_t(f.n_tiles) > kNaMaxTiles)
        return fail(ctx, GB_ERR_CAPACITY,
                    "no-allocation forward limits: %lld records (max %lld), %lld pixels (max %lld), %u tiles (max %lld)",
                    (long long)f.n_records, (long long)kNaMaxRecords, (long long)f.n_pixels,
                    (long long)kNaMaxPixels, f.n_tiles, (long long)kNaMaxTiles);
    const int nt = tile * tile;
    const int bf = forward_batch(o, f, nt);
    if (bf < 8 || bf > nt || (bf & 7) || frame_smem(f, bf, false) > 200 * 1024)
        return fail(ctx, GB_ERR_INVALID_ARG, "forward batch depth %d invalid", bf);
    int dev = 0;
    GB_CUDA(ctx, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(ctx, GB_ERR_UNSUPPORTED, "device index %d beyond 63", dev);
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *ptr = nullptr;
            GB_CUDA(ctx, cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            g_noalloc_addr[dev] = ptr;
        }
        base = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    }
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        void *p = base + off;
        off += na_round(bytes);
        return p;
    };
    Counters *cnt = static_cast<Counters *>(carve(sizeof(Counters)));
    carve(2 * kMaxGroups * 4);  // work counters (persistent mode is not offered here)
    Record *rec = static_cast<Record *>(carve(kNaMaxRecords * sizeof(Record)));
    RecordLo *rec_lo = static_cast<RecordLo *>(carve(kNaMaxRecords * sizeof(RecordLo)));
    uint32_t *depth_key = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint32_t *rec_id = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint32_t *keys_tmp = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint32_t *vals_tmp = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint32_t *dkeys_sorted = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint32_t *perm = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint32_t *offsets = static_cast<uint32_t *>(carve(kNaMaxRecords * 4));
    uint2 *rect = static_cast<uint2 *>(carve(kNaMaxRecords * 8));
    uint2 *pbox = static_cast<uint2 *>(carve(kNaMaxRecords * 8));
    uint32_t *inst_tile = static_cast<uint32_t *>(carve(kNaMaxInstances * 4));
    uint32_t *inst_val = static_cast<uint32_t *>(carve(kNaMaxInstances * 4));
    uint32_t *inst_tile_tmp = static_cast<uint32_t *>(carve(kNaMaxInstances * 4));
    uint32_t *inst_val_tmp = static_cast<uint32_t *>(carve(kNaMaxInstances * 4));
    uint32_t *tiles_sorted = static_cast<uint32_t *>(carve(kNaMaxInstances * 4));
    uint32_t *vals_sorted = static_cast<uint32_t *>(carve(kNaMaxInstances * 4));
    float *t_final = static_cast<float *>(carve(kNaMaxPixels * 4));
    uint32_t *last = static_cast<uint32_t *>(carve(kNaMaxPixels * 4));
    uint2 *ranges = static_cast<uint2 *>(carve(kNaMaxTiles * 8));
    uint32_t *tl_keys = static_cast<uint32_t *>(carve(kNaMaxTiles * 4));
    uint32_t *tl_vals = static_cast<uint32_t *>(carve(kNaMaxTiles * 4));
    uint32_t *tl_keys_tmp = static_cast<uint32_t *>(carve(kNaMaxTiles * 4));
    uint32_t *tl_vals_tmp = static_cast<uint32_t *>(carve(kNaMaxTiles * 4));
    uint32_t *tl_keys_out = static_cast<uint32_t *>(carve(kNaMaxTiles * 4));
    uint32_t *tile_list = static_cast<uint32_t *>(carve(kNaMaxTiles * 4));
    void *scratch = carve(kNaRadixBytes);
    if (off > kNaScratchBytes) return fail(ctx, GB_ERR_CUDA, "internal: no-allocation scratch layout overflow");
    if (radix_scratch_bytes(kNaMaxInstances) > kNaRadixBytes || scan_scratch_bytes(kNaMaxRecords) > kNaRadixBytes)
        return fail(ctx, GB_ERR_CUDA, "internal: no-allocation sort scratch too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t R = f.n_records;
    int tile_bits = 1;
    while ((int64_t(1) << tile_bits) < int64_t(f.n_tiles)) ++tile_bits;
    // the array keeps the previous call's contents: clear what must start at zero
    GB_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(Counters), st));
    GB_CUDA(ctx, cudaMemsetAsync(ranges, 0, size_t(f.n_tiles) * sizeof(uint2), st));
    GB_CUDA(ctx, launch_preprocess(f, max_k, depth_key, rec_id, rect, pbox, rec, cnt, st));
    GB_CUDA(ctx, launch_record(f, nullptr, nullptr, depth_key, R, rec, rec_lo, st));
    GB_CUDA(ctx, radix_sort_pairs(depth_key, rec_id, keys_tmp, vals_tmp, dkeys_sorted, perm, R, nullptr, 0, 32,
                                  scratch, kNaRadixBytes, st));
    GB_CUDA(ctx, tile_counts_scan(f, perm, rect, R, &cnt->n_visible, offsets, scratch, kNaRadixBytes, cnt,
                                  kNaMaxInstances, st));
    // the instance count decides whether the list fits: read it (no allocation)
    Counters host_cnt;
    GB_CUDA(ctx, cudaMemcpyAsync(&host_cnt, cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    GB_CUDA(ctx, cudaStreamSynchronize(st));
    if (int64_t(host_cnt.n_instances) > kNaMaxInstances)
        return fail(ctx, GB_ERR_CAPACITY, "no-allocation forward: %u (tile, splat) instances (max %lld)",
                    host_cnt.n_instances, (long long)kNaMaxInstances);
    const int64_t inst_max = std::max<int64_t>(host_cnt.n_instances, 1);
    GB_CUDA(ctx, launch_emit(f, perm, rect, offsets, R, cnt, kNaMaxInstances, inst_tile, inst_val, st));
    GB_CUDA(ctx, radix_sort_pairs(inst_tile, inst_val, inst_tile_tmp, inst_val_tmp, tiles_sorted, vals_sorted,
                                  inst_max, &cnt->n_instances, 0, tile_bits, scratch, kNaRadixBytes, st));
    GB_CUDA(ctx, launch_ranges(tiles_sorted, inst_max, cnt, ranges, st));
    const bool use_list = f.n_groups > 1;
    if (use_list) {
        int kbits = 24;
        while ((1 << (kbits - 24)) < f.n_groups) ++kbits;
        GB_CUDA(ctx, launch_tile_list(f, ranges, tl_keys, tl_vals, st));
        GB_CUDA(ctx, radix_sort_pairs(tl_keys, tl_vals, tl_keys_tmp, tl_vals_tmp, tl_keys_out, tile_list, f.n_tiles,
                                      nullptr, 0, kbits, scratch, kNaRadixBytes, st));
    }
    RenderBufs b;
    b.rec = rec;
    b.rec_lo = rec_lo;
    b.perm = perm;
    b.inst_val = vals_sorted;
    b.ranges = ranges;
    b.pbox = pbox;
    b.rgb = rgb;
    b.depth = depth;
    b.alpha = alpha;
    b.t_final = t_final;
    b.last = last;
    b.cnt = cnt;
    GB_CUDA(ctx, launch_render_fwd(f, b, bf, use_list ? tile_list : nullptr, nullptr, false, st));
    return GB_OK;
}

__global__ void fill_kernel(float *p, int64_t n, float v) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = v;
}

gb_status gb_fit_params(gb_context *ctx, int64_t K, const float *theta, const float *xy, const float *z,
                        const float *log_scales, const float *logit_opacities, float *quats, float *means,
                        float *scales, float *opacities, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (K < 0) return fail(ctx, GB_ERR_INVALID_ARG, "K must be >= 0");
    if (K > 0 && (!theta || !xy || !z || !log_scales || !logit_opacities || !quats || !means || !scales ||
                  !opacities))
        return fail(ctx, GB_ERR_INVALID_ARG, "null array");
    GB_CUDA(ctx, launch_fit_params(theta, xy, z, log_scales, logit_opacities, K, quats, means, scales, opacities,
                                   static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

gb_status gb_fit_params_backward(gb_context *ctx, int64_t K, const float *theta, const float *log_scales,
                                 const float *logit_opacities, const float *d_quats, const float *d_means,
                                 const float *d_scales, const float *d_opacities, float *d_theta, float *d_xy,
                                 float *d_log_scales, float *d_logit_opacities, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (K < 0) return fail(ctx, GB_ERR_INVALID_ARG, "K must be >= 0");
    if (K > 0 && (!theta || !log_scales || !logit_opacities || !d_quats || !d_means || !d_scales || !d_opacities ||
                  !d_theta || !d_xy || !d_log_scales || !d_logit_opacities))
        return fail(ctx, GB_ERR_INVALID_ARG, "null array");
    GB_CUDA(ctx, launch_fit_params_bwd(theta, log_scales, logit_opacities, K, d_quats, d_means, d_scales,
                                       d_opacities, d_theta, d_xy, d_log_scales, d_logit_opacities,
                                       static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

gb_status gb_mse_loss(gb_context *ctx, const float *rgb, const float *target, int64_t n, float *d_rgb,
                      double *loss, void *stream) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, GB_ERR_INVALID_ARG, "n must be >= 0");
    if (!loss || (n > 0 && (!rgb || !target))) return fail(ctx, GB_ERR_INVALID_ARG, "null array");
    GB_CUDA(ctx, launch_mse(rgb, target, n, d_rgb, loss, static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

gb_status gb_autotune(gb_context *ctx, gb_saved *s, const gb_scene *scenes, int32_t n_scenes,
                      const gb_camera *cams, int32_t n_cams, const gb_options *base, int32_t reps,
                      gb_options *best, float *ms, int32_t *tiles, int32_t *batches, int32_t *ppts,
                      int32_t cap, int32_t *n_candidates) {
    if (!ctx) return GB_ERR_INVALID_ARG;
    if (!s || s->ctx != ctx || !best) return fail(ctx, GB_ERR_INVALID_ARG, "bad autotune arguments");
    if (reps < 1 || reps > 100) return fail(ctx, GB_ERR_INVALID_ARG, "reps must be in 1..100");
    Frame f;
    int64_t max_k = 0;
    gb_status r = build_frame(ctx, scenes, n_scenes, cams, n_cams, 16, nullptr, f, max_k);
    if (r != GB_OK) return r;
    // scratch buffers owned by this call
    float *rgb = nullptr, *dep = nullptr, *alp = nullptr, *drgb = nullptr, *gbuf = nullptr;
    size_t gtot = 0;
    // gradient outputs shaped like each scene's stored arrays: the stored grid
    // (not the mip level rendered) and its per-texel SH coefficients
    auto tex_floats = [](const gb_scene &sc) {
        const int64_t Mt = sc.tex_sh_degree ? (sc.tex_sh_degree + 1) * (sc.tex_sh_degree + 1) : 1;
        return int64_t(sc.tex_n) * sc.tex_n * 3 * Mt;
    };
    for (int i = 0; i < n_scenes; ++i) {
        const int64_t K = scenes[i].num_splats, M = (scenes[i].sh_degree + 1) * (scenes[i].sh_degree + 1);
        gtot += size_t(K) * (3 + 4 + 2 + 1 + 3 * M + tex_floats(scenes[i]));
    }
    cudaError_t e = cudaMalloc(&rgb, size_t(f.n_pixels) * 12 + 16);
    if (e == cudaSuccess) e = cudaMalloc(&dep, size_t(f.n_pixels) * 4 + 16);
    if (e == cudaSuccess) e = cudaMalloc(&alp, size_t(f.n_pixels) * 4 + 16);
    if (e == cudaSuccess) e = cudaMalloc(&drgb, size_t(f.n_pixels) * 12 + 16);
    if (e == cudaSuccess) e = cudaMalloc(&gbuf, gtot * 4 + 16);
    gb_grads g[kMaxScenes];
    gb_status st = GB_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        st = fail(ctx, GB_ERR_CUDA, "autotune allocation failed: %s", cudaGetErrorString(e));
    } else {
        fill_kernel<<<1024, 256>>>(drgb, f.n_pixels * 3, 1.0f);
        count_launches(1);
        float *p = gbuf;
        for (int i = 0; i < n_scenes; ++i) {
            const int64_t K = scenes[i].num_splats, M = (scenes[i].sh_degree + 1) * (scenes[i].sh_degree + 1);
            g[i].d_means = p; p += K * 3;
            g[i].d_quats = p; p += K * 4;
            g[i].d_scales = p; p += K * 2;
            g[i].d_opacities = p; p += K;
            g[i].d_sh = p; p += K * 3 * M;
            g[i].d_textures = p; p += K * tex_floats(scenes[i]);
        }
        gb_options o{};
        if (base) o = *base;
        o.flags &= ~(GB_FLAG_NO_SYNC | GB_FLAG_TIMING);
        o.batch_depth_fwd = 0;
        float best_ms = INFINITY;
        int n = 0;
        const int tile_c[3] = {16, 8, 32};
        const int batch_c[10] = {8, 16, 24, 32, 48, 64, 88, 128, 184, 256};
        // one untimed run of the candidate (sizes `saved`), then `reps` timed
        // no-sync runs; *t = mean milliseconds
        auto time_candidate = [&](gb_options &c, bool with_bwd, float *t) -> gb_status {
            c.flags &= ~GB_FLAG_NO_SYNC;
            gb_status r = gb_render_forward(ctx, s, scenes, n_scenes, cams, n_cams, &c, rgb, dep, alp, nullptr);
            if (r == GB_OK && with_bwd) r = gb_render_backward(ctx, s, drgb, nullptr, nullptr, g, n_scenes, nullptr);
            if (r != GB_OK) return r;
            c.flags |= GB_FLAG_NO_SYNC;
            cudaEventRecord(e0, nullptr);
            for (int k = 0; k < reps && r == GB_OK; ++k) {
                r = gb_render_forward(ctx, s, scenes, n_scenes, cams, n_cams, &c, rgb, dep, alp, nullptr);
                if (r == GB_OK && with_bwd)
                    r = gb_render_backward(ctx, s, drgb, nullptr, nullptr, g, n_scenes, nullptr);
            }
            cudaEventRecord(e1, nullptr);
            c.flags &= ~GB_FLAG_NO_SYNC;
            if (r != GB_OK) return r;
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(t, e0, e1);
            if (ce != cudaSuccess) return fail(ctx, GB_ERR_CUDA, "autotune timing failed: %s", cudaGetErrorString(ce));
            r = gb_saved_check(s);
            *t /= float(reps);
            return r;
        };
        auto report = [&](int T, int B, int pi, float t) {  // appends a candidate to the caller's arrays
            if (n < cap) {
                if (ms) ms[n] = t;
                if (tiles) tiles[n] = T;
                if (batches) batches[n] = B;
                if (ppts) ppts[n] = pi;
            }
            ++n;
        };
        // forward + backward over tile, the backward's batch depth and pixels per
        // thread of the pixel-parallel backward (the forward at its automatic
        // depth, so that the backward's depth is not judged by the forward's
        // time at the same depth), then the splat-parallel one
        o.bwd_kernel = 1;
        for (int pi = 1; pi <= 2 && st == GB_OK; ++pi)
        for (int ti = 0; ti < 3 && st == GB_OK; ++ti)
            for (int bi = 0; bi < 10 && st == GB_OK; ++bi) {
                const int T = tile_c[ti], B = batch_c[bi];
                if (B > T * T / pi) continue;
                if (frame_has_var(f) && (T != 16 || pi != 1)) continue;
                if (frame_smem(f, B, true) > 160 * 1024) continue;
                o.tile_size = T;
                o.batch_depth = B;
                o.batch_depth_fwd = std::min(default_batch(f, false), T * T);
                o.pixels_per_thread = pi;
                float t = 0.0f;
                if ((st = time_candidate(o, true, &t)) != GB_OK) break;
                report(T, B, pi, t);
                if (t < best_ms) {
                    best_ms = t;
                    *best = o;
                }
            }
        // splat-parallel backward (reported with pixels_per_thread 3): tiles 16
        // and 8, batch depths up to 256 (the forward at its automatic depth)
        const int batch_sp[6] = {48, 88, 128, 176, 216, 256};
        for (int ti = 0; ti < 2 && st == GB_OK; ++ti) {
            o.tile_size = tile_c[ti];
            o.pixels_per_thread = 1;
            o.bwd_kernel = 2;
            Frame ft = f;
            ft.tile = o.tile_size;
            if (!frame_sp_ok(ft)) continue;
            for (int bi = 0; bi < 6 && st == GB_OK; ++bi) {
                const int B = batch_sp[bi];
                if (frame_sp_smem(ft, B) > 160 * 1024) continue;
                o.batch_depth = B;
                o.batch_depth_fwd = std::min(default_batch(f, false), o.tile_size * o.tile_size);
                float t = 0.0f;
                if ((st = time_candidate(o, true, &t)) != GB_OK) break;
                report(o.tile_size, B, 3, t);
                if (t < best_ms) {
                    best_ms = t;
                    *best = o;
                }
            }
            o.batch_depth_fwd = 0;
        }
        // the forward alone at every depth that fits the fastest tile (its time
        // does not depend on the backward's options)
        if (st == GB_OK && best_ms < INFINITY) {
            gb_options c = *best;
            const int T = c.tile_size;
            float best_fwd = INFINITY;
            for (int bi = 0; bi < 10 && st == GB_OK; ++bi) {
                const int B = batch_c[bi];
                if (B > T * T || frame_smem(f, B, false) > 160 * 1024) continue;
                c.batch_depth_fwd = B;
                float t = 0.0f;
                if ((st = time_candidate(c, false, &t)) != GB_OK) break;
                report(T, B, 0, t);
                if (t < best_fwd) {
                    best_fwd = t;
                    best->batch_depth_fwd = B;
                }
            }
        }
        if (st == GB_OK && best_ms < INFINITY) {
            best->flags &= ~GB_FLAG_NO_SYNC;
            if (base) best->flags |= (base->flags & GB_FLAG_NO_SYNC);
        }
        if (n_candidates) *n_candidates = n;
        if (st == GB_OK && n == 0) st = fail(ctx, GB_ERR_UNSUPPORTED, "no autotune candidate fits");
    }
    cudaDeviceSynchronize();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rgb); cudaFree(dep); cudaFree(alp); cudaFree(drgb); cudaFree(gbuf);
    return st;
}

}  // extern "C"
