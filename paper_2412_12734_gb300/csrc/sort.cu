// Sorting and bookkeeping kernels: stable LSD radix sort of (u32 key, u32
// value) pairs, exclusive scan, (tile, splat) instance duplication, per-tile
// ranges.  Element counts may live on the device (kernels are launched for a
// capacity and read the true count), so no host round trip is needed between
// preprocess and render.
#include "gbill_internal.cuh"

namespace gbill {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;  // 32-key rounds per warp
constexpr int kWarpTile = 32 * kSortRounds;
constexpr int kSortTile = kWarpTile * kSortWarps;  // 4096 keys per block
constexpr int kMaxRadixBits = 9;                   // digits of 8 or 9 bits

__device__ __forceinline__ uint32_t load_n(const uint32_t *n_dev, int64_t max_n) {
    return n_dev ? uint32_t(min(int64_t(*n_dev), max_n)) : uint32_t(max_n);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Per-block digit histogram, written digit-major: hist[d * nblocks + block].
template <int BITS>
__global__ void __launch_bounds__(kSortThreads) radix_upsweep(const uint32_t *keys, int64_t max_n,
                                                              const uint32_t *n_dev, int shift,
                                                              uint32_t mask, uint32_t *hist) {
    constexpr int kRadix = 1 << BITS;
    __shared__ uint32_t h[kRadix];
    const uint32_t n = load_n(n_dev, max_n);
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = int64_t(blockIdx.x) * kSortTile + int64_t(warp) * kWarpTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool act = idx < n;
        const uint32_t am = __ballot_sync(0xffffffffu, act);
        if (act) {
            const uint32_t d = (keys[idx] >> shift) & mask;
            const uint32_t peers = __match_any_sync(am, d);
            if ((peers & lanemask_lt()) == 0) atomicAdd(&h[d], uint32_t(__popc(peers)));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) hist[int64_t(i) * gridDim.x + blockIdx.x] = h[i];
}

// Stable scatter: warp w owns keys [w*512, (w+1)*512) of the block tile and
// ranks them in order with warp-match; per-digit warp counts are then
// prefix-summed over warps so earlier warps come first.
template <int BITS>
__global__ void __launch_bounds__(kSortThreads) radix_downsweep(
    const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out, uint32_t *vals_out,
    int64_t max_n, const uint32_t *n_dev, int shift, uint32_t mask, const uint32_t *offs) {
    constexpr int kRadix = 1 << BITS;
    // per-warp digit counts, later the block's keys in local (digit, input) order
    __shared__ uint32_t wcount[kSortWarps * kRadix > kSortTile ? kSortWarps * kRadix : kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t goff[kRadix];  // the block's first global position per digit
    __shared__ uint32_t loc[kRadix];   // the block's first local position per digit
    const uint32_t n = load_n(n_dev, max_n);
    const int64_t blk_base = int64_t(blockIdx.x) * kSortTile;
    if (blk_base >= n) return;  // uniform per block
    const int nblk = int(int64_t(n) - blk_base < int64_t(kSortTile) ? int64_t(n) - blk_base : int64_t(kSortTile));
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) wcount[i] = 0;
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) goff[i] = offs[int64_t(i) * gridDim.x + blockIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = blk_base + int64_t(warp) * kWarpTile;
    uint32_t k_[kSortRounds], v_[kSortRounds], rank_[kSortRounds];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool act = idx < n;
        const uint32_t am = __ballot_sync(0xffffffffu, act);
        rank_[r] = 0xffffffffu;
        if (act) {
            k_[r] = keys_in[idx];
            v_[r] = vals_in[idx];
            const uint32_t d = (k_[r] >> shift) & mask;
            const uint32_t peers = __match_any_sync(am, d);
            const uint32_t before = wcount[warp * kRadix + d];
            rank_[r] = before + __popc(peers & lt);
            __syncwarp(am);
            if ((peers & lt) == 0) wcount[warp * kRadix + d] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps (the warp's first slot within the
    // digit's run) and the digit's block total
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcount[w * kRadix + d];
            wcount[w * kRadix + d] = run;
            run += c;
        }
        loc[d] = run;
    }
    __syncthreads();
    // exclusive prefix over digits of the block totals: each thread sums its
    // kRadix / kSortThreads consecutive digits, then a warp scan and the warps'
    // totals
    {
        constexpr int PER = kRadix / kSortThreads;
        static_assert(PER >= 1 && PER * kSortThreads == kRadix, "digits per thread");
        __shared__ uint32_t wsum[kSortWarps];
        uint32_t c[PER], tsum = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            c[i] = loc[threadIdx.x * PER + i];
            tsum += c[i];
        }
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t excl = x - tsum;
        for (int w = 0; w < warp; ++w) excl += wsum[w];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            loc[threadIdx.x * PER + i] = excl;
            excl += c[i];
        }
    }
    __syncthreads();
    uint32_t lpos[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r)
        if (rank_[r] != 0xffffffffu) {
            const uint32_t d = (k_[r] >> shift) & mask;
            lpos[r] = loc[d] + wcount[warp * kRadix + d] + rank_[r];
        }
    __syncthreads();  // the counts are read; their array now takes the keys
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r)
        if (rank_[r] != 0xffffffffu) {
            wcount[lpos[r]] = k_[r];
            s_vals[lpos[r]] = v_[r];
        }
    __syncthreads();
    // in local order: consecutive threads write consecutive positions of a
    // digit's run (coalesced)
    for (int p = threadIdx.x; p < nblk; p += kSortThreads) {
        const uint32_t k = wcount[p];
        const uint32_t d = (k >> shift) & mask;
        const uint32_t pos = goff[d] + uint32_t(p) - loc[d];
        keys_out[pos] = k;
        vals_out[pos] = s_vals[p];
    }
}

// ----------------------------------------------------------------- scan --
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

struct LoadArray {
    const uint32_t *a;
    __device__ uint32_t operator()(int64_t i) const { return a[i]; }
};

// Tile count of the j-th depth-sorted record: rectangle area in tiles.
struct LoadTileCount {
    const uint32_t *perm;
    const uint2 *rect;
    __device__ uint32_t operator()(int64_t j) const {
        const uint2 r = rect[perm[j]];
        const uint32_t nx = (r.y & 0xffffu) - (r.x & 0xffffu) + 1u;
        const uint32_t ny = (r.y >> 16) - (r.x >> 16) + 1u;
        return nx * ny;
    }
};

// Exclusive scan over the block's threads, in the type T (uint32_t for the
// radix histograms, uint64_t for tile counts, whose totals may pass 2^32).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total) {
    __shared__ T wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < kScanThreads / 32 ? wsum[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    const T before = warp ? wsum[warp - 1] : T(0);
    *total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__device__ __forceinline__ uint32_t saturate32(uint64_t x) {
    return x > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(x);
}

// Every partial sum is formed in 64 bits: one block holds 4,096 counts of up
// to 2^32 - 1 each, so its total, the running offsets and the frame total can
// all pass 2^32.  Block sums and offsets are stored saturated at 2^32 - 1;
// such a frame sets the overflow flag (its total exceeds any capacity), and
// every emit past the capacity is skipped.
template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_reduce(Load ld, int64_t max_n, const uint32_t *n_dev,
                                                            uint32_t *block_sums) {
    const uint32_t n = load_n(n_dev, max_n);
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    uint64_t s = 0;
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += ld(base + i);
    uint64_t tot;
    block_exclusive_scan<uint64_t>(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = saturate32(tot);
}

// Single block: exclusive scan of the block sums in place (64-bit running
// sums, stored saturated); the total to *total and the counters.
__global__ void __launch_bounds__(kScanThreads) scan_block_sums(uint32_t *sums, int64_t nb, uint32_t *total,
                                                                Counters *cnt, int64_t capacity) {
    uint64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = i < nb ? uint64_t(sums[i]) : 0ull;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan<uint64_t>(v, &tot);
        if (i < nb) sums[i] = saturate32(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        const uint32_t sat = saturate32(carry);
        if (total) *total = sat;
        if (cnt) {
            cnt->n_instances = sat;
            if (carry > uint64_t(capacity)) cnt->overflow = 1u;
        }
    }
}

template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_downsweep(Load ld, int64_t max_n, const uint32_t *n_dev,
                                                               const uint32_t *block_sums, uint32_t *out) {
    const uint32_t n = load_n(n_dev, max_n);
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? ld(base + i) : 0u;
        s += v[i];
    }
    uint64_t tot;
    uint64_t run = uint64_t(block_sums[blockIdx.x]) + block_exclusive_scan<uint64_t>(s, &tot);
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = saturate32(run);
        run += v[i];
    }
}

template <class Load>
cudaError_t exclusive_scan(Load ld, int64_t max_n, const uint32_t *n_dev, uint32_t *out, uint32_t *total,
                           void *scratch, size_t scratch_bytes, Counters *cnt, int64_t capacity,
                           cudaStream_t s) {
    const int64_t nb = ceil_div(max_n, kScanTile);
    if (nb <= 0) return cudaSuccess;
    if (scratch_bytes < size_t(nb) * sizeof(uint32_t)) return cudaErrorInvalidValue;
    uint32_t *sums = static_cast<uint32_t *>(scratch);
    scan_reduce<<<unsigned(nb), kScanThreads, 0, s>>>(ld, max_n, n_dev, sums);
    scan_block_sums<<<1, kScanThreads, 0, s>>>(sums, nb, total, cnt, capacity);
    scan_downsweep<<<unsigned(nb), kScanThreads, 0, s>>>(ld, max_n, n_dev, sums, out);
    count_launches(3);
    return cudaGetLastError();
}

// ---------------------------------------------------------- duplication --
__global__ void __launch_bounds__(256) emit_kernel(Frame f, const uint32_t *perm, const uint2 *rect,
                                                   const uint32_t *offsets, int64_t max_n,
                                                   const Counters *cnt, int64_t capacity,
                                                   uint32_t *inst_tile, uint32_t *inst_val) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= min(int64_t(cnt->n_visible), max_n)) return;
    const uint32_t r = perm[j];
    const int ci = camera_of_record(f, r);
    const CamDev &cam = f.cams[ci];
    const uint2 rc = rect[r];
    const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu, y1 = rc.y >> 16;
    int64_t o = offsets[j];
    if (o + int64_t(x1 - x0 + 1) * (y1 - y0 + 1) > capacity) return;  // overflow flagged by the scan
    for (uint32_t y = y0; y <= y1; ++y)
        for (uint32_t x = x0; x <= x1; ++x) {
            inst_tile[o] = cam.tile_off + y * uint32_t(cam.tiles_x) + x;
            inst_val[o] = uint32_t(j);
            ++o;
        }
}

__global__ void ranges_kernel(const uint32_t *tiles, int64_t max_n, const Counters *cnt, uint2 *ranges) {
    const int64_t n = min(int64_t(cnt->n_instances), max_n);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = tiles[i];
    if (i == 0 || tiles[i - 1] != t) ranges[t].x = uint32_t(i);
    if (i == n - 1 || tiles[i + 1] != t) ranges[t].y = uint32_t(i + 1);
}

// inv[perm[j]] = j for the visible records (the caller preset inv to -1).
__global__ void inverse_perm_kernel(const uint32_t *perm, int64_t n_records, const Counters *cnt, int32_t *inv) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= min(int64_t(cnt->n_visible), n_records)) return;
    inv[perm[j]] = int32_t(j);
}

// Visible records (depth key not the culled marker) in record order.
struct LoadVisible {
    const uint32_t *key;
    __device__ uint32_t operator()(int64_t i) const { return key[i] != 0xFFFFFFFFu ? 1u : 0u; }
};

__global__ void compact_kernel(const uint32_t *key, const uint32_t *pos, int64_t n, uint32_t *key_out,
                               uint32_t *id_out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = key[i];
    if (k != 0xFFFFFFFFu) {
        key_out[pos[i]] = k;
        id_out[pos[i]] = uint32_t(i);
    }
}

__global__ void export_keys_kernel(Frame f, const uint32_t *tiles, const uint32_t *vals, const uint32_t *perm,
                                   const uint32_t *depth_key, int64_t n, uint64_t *keys, int64_t *ids,
                                   int32_t *cams) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t r = perm[vals[i]];
    const int ci = camera_of_record(f, r);
    keys[i] = (uint64_t(tiles[i]) << 32) | depth_key[r];
    ids[i] = int64_t(r) - f.cams[ci].rec_off;
    cams[i] = ci;
}

// Sort key of a tile: its render group, then instance count, largest first.
__global__ void tile_key_kernel(Frame f, const uint2 *ranges, uint32_t *keys, uint32_t *vals) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= f.n_tiles) return;
    const int ci = camera_of_tile(f, t);
    const uint2 r = ranges[t];
    const uint32_t cost = min(r.y - r.x, 0xFFFFFFu);
    keys[t] = (uint32_t(f.cams[ci].group) << 24) | (0xFFFFFFu - cost);
    vals[t] = t;
}

}  // namespace

cudaError_t launch_tile_list(const Frame &f, const uint2 *ranges, uint32_t *keys, uint32_t *vals, cudaStream_t s) {
    if (f.n_tiles == 0) return cudaSuccess;
    tile_key_kernel<<<unsigned(ceil_div(f.n_tiles, 256)), 256, 0, s>>>(f, ranges, keys, vals);
    count_launches(1);
    return cudaGetLastError();
}

size_t radix_scratch_bytes(int64_t n) {
    const int64_t nb = ceil_div(n, kSortTile);
    const int64_t h = nb * (int64_t(1) << kMaxRadixBits);
    return size_t(h) * sizeof(uint32_t) + size_t(ceil_div(h, kScanTile) + 1) * sizeof(uint32_t) + 256;
}

size_t scan_scratch_bytes(int64_t n) { return size_t(ceil_div(n, kScanTile) + 1) * sizeof(uint32_t); }

cudaError_t radix_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_tmp,
                             uint32_t *vals_tmp, uint32_t *keys_out, uint32_t *vals_out, int64_t max_n,
                             const uint32_t *n_dev, int begin_bit, int end_bit, void *scratch,
                             size_t scratch_bytes, cudaStream_t s) {
    if (max_n <= 0) return cudaSuccess;
    const int64_t nb = ceil_div(max_n, kSortTile);
    if (scratch_bytes < radix_scratch_bytes(max_n)) return cudaErrorInvalidValue;
    uint32_t *hist = static_cast<uint32_t *>(scratch);
    uint32_t *scan_tmp = hist + nb * (int64_t(1) << kMaxRadixBits);
    const size_t scan_bytes = scratch_bytes - size_t(nb << kMaxRadixBits) * sizeof(uint32_t);
    const int bits = end_bit - begin_bit;
    if (bits <= 0) {
        if (keys_out == keys_in) return cudaSuccess;
        cudaMemcpyAsync(keys_out, keys_in, size_t(max_n) * 4, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals_out, vals_in, size_t(max_n) * 4, cudaMemcpyDeviceToDevice, s);
        return cudaGetLastError();
    }
    // fewest passes of at most 9 bits, the bits spread evenly (17 -> 9 + 8, 32 -> 4 x 8)
    const int passes = (bits + kMaxRadixBits - 1) / kMaxRadixBits;
    // the last pass writes keys_out; with the input there, pass 0 must not
    if (keys_in == keys_out && (passes & 1)) return cudaErrorInvalidValue;
    const uint32_t *ki = keys_in, *vi = vals_in;
    int shift = begin_bit;
    for (int p = 0; p < passes; ++p) {
        const int w = bits / passes + (p < bits % passes ? 1 : 0);
        const uint32_t mask = (1u << w) - 1u;
        uint32_t *ko = ((passes - p) & 1) ? keys_out : keys_tmp;
        uint32_t *vo = ((passes - p) & 1) ? vals_out : vals_tmp;
        const int64_t h = nb << (w > 8 ? 9 : 8);
        if (w > 8) radix_upsweep<9><<<unsigned(nb), kSortThreads, 0, s>>>(ki, max_n, n_dev, shift, mask, hist);
        else radix_upsweep<8><<<unsigned(nb), kSortThreads, 0, s>>>(ki, max_n, n_dev, shift, mask, hist);
        cudaError_t e = exclusive_scan(LoadArray{hist}, h, nullptr, hist, nullptr, scan_tmp, scan_bytes,
                                       nullptr, 0, s);
        if (e != cudaSuccess) return e;
        if (w > 8)
            radix_downsweep<9><<<unsigned(nb), kSortThreads, 0, s>>>(ki, vi, ko, vo, max_n, n_dev, shift, mask, hist);
        else
            radix_downsweep<8><<<unsigned(nb), kSortThreads, 0, s>>>(ki, vi, ko, vo, max_n, n_dev, shift, mask, hist);
        count_launches(2);
        ki = ko;
        vi = vo;
        shift += w;
    }
    return cudaGetLastError();
}

cudaError_t compact_visible(const uint32_t *depth_key, int64_t n, uint32_t *pos, uint32_t *key_out,
                            uint32_t *id_out, void *scratch, size_t scratch_bytes, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = exclusive_scan(LoadVisible{depth_key}, n, nullptr, pos, nullptr, scratch, scratch_bytes, nullptr,
                                   0, s);
    if (e != cudaSuccess) return e;
    compact_kernel<<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(depth_key, pos, n, key_out, id_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t tile_counts_scan(const Frame &f, const uint32_t *perm, const uint2 *rect, int64_t max_n,
                             const uint32_t *n_dev, uint32_t *offsets, void *scratch, size_t scratch_bytes,
                             Counters *cnt, int64_t capacity, cudaStream_t s) {
    (void)f;
    return exclusive_scan(LoadTileCount{perm, rect}, max_n, n_dev, offsets, nullptr, scratch, scratch_bytes,
                          cnt, capacity, s);
}

cudaError_t launch_emit(const Frame &f, const uint32_t *perm, const uint2 *rect, const uint32_t *offsets,
                        int64_t max_n, const Counters *cnt, int64_t capacity, uint32_t *inst_tile,
                        uint32_t *inst_val, cudaStream_t s) {
    if (max_n <= 0) return cudaSuccess;
    emit_kernel<<<unsigned(ceil_div(max_n, 256)), 256, 0, s>>>(f, perm, rect, offsets, max_n, cnt, capacity,
                                                              inst_tile, inst_val);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t *tiles_sorted, int64_t max_n, const Counters *cnt, uint2 *ranges,
                          cudaStream_t s) {
    if (max_n <= 0) return cudaSuccess;
    ranges_kernel<<<unsigned(ceil_div(max_n, 256)), 256, 0, s>>>(tiles_sorted, max_n, cnt, ranges);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_inverse_perm(const uint32_t *perm, int64_t n_records, const Counters *cnt, int32_t *inv,
                                cudaStream_t s) {
    if (n_records <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(inv, 0xFF, size_t(n_records) * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    inverse_perm_kernel<<<unsigned(ceil_div(n_records, 256)), 256, 0, s>>>(perm, n_records, cnt, inv);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_export_keys(const Frame &f, const uint32_t *tiles_sorted, const uint32_t *vals_sorted,
                               const uint32_t *perm, const uint32_t *depth_key_by_rec, int64_t n,
                               uint64_t *keys, int64_t *ids, int32_t *cams, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    export_keys_kernel<<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(f, tiles_sorted, vals_sorted, perm,
                                                                  depth_key_by_rec, n, keys, ids, cams);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gbill
