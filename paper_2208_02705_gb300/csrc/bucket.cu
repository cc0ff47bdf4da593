// Bucketing of samples by field (counting sort: histogram, exclusive scan,
// scatter) so that each tiny MLP is evaluated over a contiguous run of its
// own samples: the concurrent queries of many MLPs of Sec. "Real-time
// Rendering Speedup" done as one grouped evaluation.  The scan also cuts
// every field's run into tiles for the MLP kernels.
#include "internal.cuh"

namespace roam {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Iterates the valid samples of a round.  Slot layout: 32 consecutive live
// rays share a 32-wide column per sample index k (see slot_of); a warp covers
// one (ray group, k) pair, so reads of cnt and recs coalesce.
struct SlotIter {
    const uint32_t *cnt;
    const uint32_t *recs;
    uint32_t n_live;
    uint32_t R;
    __device__ uint64_t total() const { return (uint64_t)((n_live + 31u) >> 5) * R * 32u; }
    // slot ids fit in 32 bits (the round size is chosen so), so the column
    // arithmetic stays 32-bit
    // (the record is read whether or not slot s holds one -- every slot
    // below total() lies inside the slot array -- so that it and the
    // ray's count are loaded side by side, not one after the other)
    __device__ bool valid(uint64_t s, uint32_t &key) const
    {
        const uint32_t lane = (uint32_t)(s & 31u);
        const uint32_t col = (uint32_t)(s >> 5);
        const uint32_t q = group_of(col, R);
        const uint32_t k = col - q * R;
        const uint32_t i = q * 32u + lane;
        const uint32_t rec = __ldg(recs + s);
        if (i >= n_live || k >= __ldg(cnt + i)) return false;
        key = rec >> 16;
        return true;
    }
};

__global__ void __launch_bounds__(512) k_hist(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count,
                                              uint32_t n_fixed, int R, const uint16_t *keys16, int n_fields,
                                              uint32_t *hist, Counters *ctr)
{
    extern __shared__ uint32_t sh[];
    for (int f = threadIdx.x; f < n_fields; f += blockDim.x) sh[f] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (keys16) {
        for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_fixed; s += stride) {
            const uint32_t key = keys16[s];
            if (key < (uint32_t)n_fields) atomicAdd(&sh[key], 1u);
            else atomicOr(&ctr->status, kStatusBadLabel);
        }
    } else {
        SlotIter it{cnt, recs, live_count ? *live_count : n_fixed, (uint32_t)R};
        const uint64_t tot = it.total();
        for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < tot; s += stride) {
            uint32_t key;
            if (it.valid(s, key)) atomicAdd(&sh[key], 1u);
        }
    }
    __syncthreads();
    for (int f = threadIdx.x; f < n_fields; f += blockDim.x)
        if (sh[f]) atomicAdd(&hist[f], sh[f]);
}

__device__ __forceinline__ uint32_t ntiles_of(uint32_t h, int tile, int group)
{
    const uint32_t t = (h + (uint32_t)tile - 1u) / (uint32_t)tile;
    return (t + (uint32_t)group - 1u) / (uint32_t)group * (uint32_t)group;
}

// the padding group of field f: its class's own, else the call's
__device__ __forceinline__ int group_of_field(const ClassBounds &cb, int f, int group)
{
    int c = 0;
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (f >= cb.first[k]) c = k;
    return cb.group[c] > 0 ? cb.group[c] : group;
}

// One block: offsets = exclusive scan of hist; tiles of `tile` samples per
// field, the tile count of every non-empty field rounded up to a multiple of
// its group (its class's, else `group`; trailing tiles empty) so that groups
// of tiles never mix fields; resets hist for the next use.
__global__ void __launch_bounds__(1024) k_scan(uint32_t *hist, int n_fields, int tile, int group, uint32_t *offsets,
                                               uint32_t *cursor, Tile *tiles, uint32_t *tile_off_out, Counters *ctr,
                                               ClassBounds cb)
{
    __shared__ uint32_t warp_a[32], warp_b[32];
    extern __shared__ uint32_t tile_off[];   // [n_fields + 1]
    const int per = (n_fields + blockDim.x - 1) / blockDim.x;
    const int f0 = threadIdx.x * per;
    uint32_t cs = 0, ts = 0, hit = 0;
    for (int q = 0; q < per; ++q) {
        const int f = f0 + q;
        if (f < n_fields) {
            const uint32_t h = hist[f];
            cs += h;
            ts += ntiles_of(h, tile, group_of_field(cb, f, group));
            hit += h > 0;
        }
    }
    // block scans of (cs, ts)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t a = cs, b = ts;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(kFull, a, o), yb = __shfl_up_sync(kFull, b, o);
        if (lane >= o) { a += ya; b += yb; }
    }
    if (lane == 31) { warp_a[wid] = a; warp_b[wid] = b; }
    __syncthreads();
    if (wid == 0) {
        uint32_t sa = lane < (int)(blockDim.x >> 5) ? warp_a[lane] : 0u;
        uint32_t sb = lane < (int)(blockDim.x >> 5) ? warp_b[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ya = __shfl_up_sync(kFull, sa, o), yb = __shfl_up_sync(kFull, sb, o);
            if (lane >= o) { sa += ya; sb += yb; }
        }
        warp_a[lane] = sa;
        warp_b[lane] = sb;
    }
    __syncthreads();
    uint32_t ea = a - cs + (wid > 0 ? warp_a[wid - 1] : 0u);
    uint32_t eb = b - ts + (wid > 0 ? warp_b[wid - 1] : 0u);
    const uint32_t total = warp_a[(blockDim.x >> 5) - 1];
    const uint32_t total_tiles = warp_b[(blockDim.x >> 5) - 1];
    for (int q = 0; q < per; ++q) {
        const int f = f0 + q;
        if (f < n_fields) {
            const uint32_t h = hist[f];
            offsets[f] = ea;
            cursor[f] = ea;
            tile_off[f] = eb;
            ea += h;
            eb += ntiles_of(h, tile, group_of_field(cb, f, group));
        }
    }
    if (threadIdx.x == 0) {
        offsets[n_fields] = total;
        tile_off[n_fields] = total_tiles;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) ctr->class_tiles[c] = tile_off[min(max(cb.first[c], 0), n_fields)];
    // field hit counts (warp reduce then atomics)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hit += __shfl_down_sync(kFull, hit, o);
    if (lane == 0 && hit) atomicAdd(&ctr->fields_hit, hit);
    __syncthreads();
    // tile descriptors: tile t belongs to the last field whose first tile is <= t
    // (written here, or by the scatter's whole grid when tile_off_out is set)
    if (tile_off_out)
        for (int f = threadIdx.x; f <= n_fields; f += blockDim.x) tile_off_out[f] = tile_off[f];
    for (uint32_t t = threadIdx.x; t < (tile_off_out ? 0u : total_tiles); t += blockDim.x) {
        int lo = 0, hi = n_fields - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        // skip fields with no tiles (equal tile_off): the search lands on the last one
        const uint32_t k = t - tile_off[lo];
        const uint32_t h = offsets[lo + 1] - offsets[lo];
        Tile tl;
        tl.field = (uint32_t)lo;
        tl.start = offsets[lo] + k * (uint32_t)tile;
        tl.count = h > k * (uint32_t)tile ? min((uint32_t)tile, h - k * (uint32_t)tile) : 0u;
        tl.pad = 0;
        tiles[t] = tl;
    }
    __syncthreads();
    for (int q = 0; q < per; ++q) {
        const int f = f0 + q;
        if (f < n_fields) hist[f] = 0;
    }
    if (threadIdx.x == 0) {
        ctr->n_tiles = total_tiles;
        ctr->n_samples += total;
    }
}

__device__ __forceinline__ void scatter_one(bool valid, uint32_t key, uint32_t value, uint32_t *cursor,
                                            uint32_t *sorted)
{
    const unsigned active = __ballot_sync(kFull, valid);
    if (valid) {
        const unsigned peers = __match_any_sync(active, key);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&cursor[key], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        sorted[base + __popc(peers & ((1u << lane) - 1u))] = value;
    }
}

__global__ void __launch_bounds__(512) k_scatter(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count,
                                                 uint32_t n_fixed, int R, const uint16_t *keys16, int n_fields,
                                                 uint32_t *cursor, uint32_t *sorted)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (keys16) {
        const uint64_t tot = ((uint64_t)n_fixed + 31u) & ~31ull;
        for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < tot; s += stride) {
            const uint32_t key = s < n_fixed ? keys16[s] : 0u;
            const bool v = s < n_fixed && key < (uint32_t)n_fields;
            scatter_one(v, key, (uint32_t)s, cursor, sorted);
        }
    } else {
        SlotIter it{cnt, recs, live_count ? *live_count : n_fixed, (uint32_t)R};
        const uint64_t tot = it.total();
        for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < tot; s += stride) {
            uint32_t key = 0;
            const bool v = it.valid(s, key);
            scatter_one(v, key, (uint32_t)s, cursor, sorted);
        }
    }
}

// tile t of the list: the last field whose first tile is <= t
__device__ __forceinline__ Tile tile_record(uint32_t t, const uint32_t *tile_off, const uint32_t *offsets, int n_fields,
                                            int tile)
{
    int lo = 0, hi = n_fields - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_off + mid) <= t) lo = mid; else hi = mid - 1;
    }
    const uint32_t k = t - __ldg(tile_off + lo);
    const uint32_t o0 = __ldg(offsets + lo), h = __ldg(offsets + lo + 1) - o0;
    Tile tl;
    tl.field = (uint32_t)lo;
    tl.start = o0 + k * (uint32_t)tile;
    tl.count = h > k * (uint32_t)tile ? min((uint32_t)tile, h - k * (uint32_t)tile) : 0u;
    tl.pad = 0;
    return tl;
}

// Scatter with block-level aggregation: a block takes kItems x blockDim
// consecutive samples, ranks them within their field in shared memory,
// reserves each touched field's range with one global atomic, then writes;
// the whole grid also writes the tile records from the scan's tile offsets.
constexpr int kItems = 8;
constexpr int kMaxFieldsBlk = 6144;     // two shared counters per field within 48 KB

__global__ void __launch_bounds__(512) k_scatter_blk(const uint32_t *cnt, const uint32_t *recs,
                                                     const uint32_t *live_count, uint32_t n_fixed, int R,
                                                     const uint16_t *keys16, int n_fields, uint32_t *cursor,
                                                     uint32_t *sorted, const uint32_t *tile_off,
                                                     const uint32_t *offsets, Tile *tiles, int tile, Counters *ctr)
{
    extern __shared__ uint32_t sh[];
    uint32_t *cnt_s = sh, *base_s = sh + n_fields;
    for (int f = threadIdx.x; f < n_fields; f += blockDim.x) cnt_s[f] = 0u;
    __syncthreads();
    SlotIter it{cnt, recs, live_count ? *live_count : n_fixed, (uint32_t)R};
    const uint64_t tot = keys16 ? (uint64_t)n_fixed : it.total();
    const uint64_t chunk = (uint64_t)blockDim.x * kItems;
    for (uint64_t c0 = (uint64_t)blockIdx.x * chunk; c0 < tot; c0 += (uint64_t)gridDim.x * chunk) {
        uint32_t key[kItems], loc[kItems];
        bool v[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint64_t s = c0 + (uint64_t)i * blockDim.x + threadIdx.x;
            key[i] = 0u;
            v[i] = false;
            if (s < tot) {
                if (keys16) {
                    key[i] = keys16[s];
                    v[i] = key[i] < (uint32_t)n_fields;
                    if (!v[i]) atomicOr(&ctr->status, kStatusBadLabel);
                } else {
                    v[i] = it.valid(s, key[i]);
                }
            }
            if (v[i]) loc[i] = atomicAdd(&cnt_s[key[i]], 1u);
        }
        __syncthreads();
        for (int f = threadIdx.x; f < n_fields; f += blockDim.x) {
            const uint32_t n = cnt_s[f];
            if (n) {
                base_s[f] = atomicAdd(&cursor[f], n);
                cnt_s[f] = 0u;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (v[i]) sorted[base_s[key[i]] + loc[i]] = (uint32_t)(c0 + (uint64_t)i * blockDim.x + threadIdx.x);
        __syncthreads();
    }
    const uint32_t n_tiles = ctr->n_tiles;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
        tiles[t] = tile_record(t, tile_off, offsets, n_fields, tile);
}

void scan_and_scatter(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count, uint32_t n_fixed, int R,
                      int group, const uint16_t *keys16, int n_fields, int tile, const BucketBufs &b, Counters *ctr,
                      int grid, cudaStream_t s, ClassBounds cb)
{
    const bool blk = b.tile_off != nullptr && n_fields <= kMaxFieldsBlk;
    k_scan<<<1, 1024, (size_t)(n_fields + 1) * sizeof(uint32_t), s>>>(b.hist, n_fields, tile, group < 1 ? 1 : group,
                                                                       b.offsets, b.cursor, b.tiles,
                                                                       blk ? b.tile_off : nullptr, ctr, cb);
    if (blk)
        k_scatter_blk<<<grid, 512, 2 * (size_t)n_fields * sizeof(uint32_t), s>>>(
            cnt, recs, live_count, n_fixed, R, keys16, n_fields, b.cursor, b.sorted, b.tile_off, b.offsets, b.tiles,
            tile, ctr);
    else
        k_scatter<<<grid, 512, 0, s>>>(cnt, recs, live_count, n_fixed, R, keys16, n_fields, b.cursor, b.sorted);
}

}  // namespace

void launch_bucket(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count, uint32_t n_fixed,
                   int R, int group, const uint16_t *keys16, int n_fields, int tile,
                   const BucketBufs &b, Counters *ctr, int grid, cudaStream_t s, ClassBounds cb)
{
    const size_t sh = (size_t)n_fields * sizeof(uint32_t);
    k_hist<<<grid, 512, sh, s>>>(cnt, recs, live_count, n_fixed, R, keys16, n_fields, b.hist, ctr);
    scan_and_scatter(cnt, recs, live_count, n_fixed, R, group, keys16, n_fields, tile, b, ctr, grid, s, cb);
}

void launch_bucket_ready(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count, uint32_t n_fixed,
                         int R, int group, int n_fields, int tile, const BucketBufs &b, Counters *ctr, int grid,
                         cudaStream_t s, ClassBounds cb)
{
    scan_and_scatter(cnt, recs, live_count, n_fixed, R, group, nullptr, n_fields, tile, b, ctr, grid, s, cb);
}

}  // namespace roam
