// Adaptive assignment of the occupied voxels to n networks (Alg. 1 stage
// II, Sec. "Adaptive Radiance Fields Slimming and Fine-tuning"): network k
// takes the smallest unassigned voxel (lexicographic (z, y, x), i.e. the
// smallest linear index) as its anchor plus the s - 1 unassigned voxels
// nearest to it (squared distance in voxel units, ties to the smaller linear
// index), s = S / n; the last network takes what remains.
//
// The networks are built one after the other (each depends on the voxels
// the earlier ones took); within a network everything is data parallel:
//   k_hist_select  per digit of the 47-bit key (squared distance << 27 |
//                  rank), a histogram of the candidates matching the digits
//                  fixed so far (shared-memory bins, then global atomics);
//                  the block that finishes last picks the bin holding the
//                  wanted rank, growing the key prefix by one digit (4
//                  digits of 12 bits)
//   k_take_anchor  every unassigned voxel whose key is <= the selected key
//                  joins the network; the block that finishes last finds the
//                  next network's anchor (the first unassigned voxel from a
//                  cursor; k_anchor for the first network)
// Five launches per network, with no waiting between blocks: the serial
// parts run in whichever block finishes last (a counter of finished blocks).
// Keys are unique (the rank is part of them), so exactly s voxels are taken.
// All state stays on the device: no host synchronisation per network.
#include "internal.cuh"

namespace roam {

namespace {

constexpr int kDigitBits = 12;
constexpr int kBins = 1 << kDigitBits;
constexpr int kRankBits = 27;               // ranks below 2^27 (512^3 grids hold < 2^27 occupied voxels)
constexpr uint16_t kFree = 0xffffu;

struct AssignState {
    uint32_t cursor;       // every rank before it is assigned
    uint32_t anchor;       // rank of the current anchor
    uint32_t ax, ay, az;   // its voxel coordinates
    uint32_t rank_left;    // rank still to locate within the current prefix
    unsigned long long prefix;   // key digits fixed so far
    uint32_t status;
    uint32_t done;               // blocks finished in the current launch (the last one does the serial part)
};

__global__ void k_occupied_list(const uint32_t *bits, const uint32_t *prefix, int64_t n_words, uint32_t *vox)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = bits[w];
        uint32_t r = prefix[w];
        while (word) {
            const int b = __ffs(word) - 1;
            vox[r++] = (uint32_t)(w * 32 + b);
            word &= word - 1u;
        }
    }
}

// the first unassigned voxel from the cursor: the new anchor (one block)
__device__ void find_anchor(const uint16_t *field, uint32_t S, const uint32_t *vox, int gx, int gy, AssignState *st,
                            uint32_t s_minus_1)
{
    __shared__ uint32_t found;
    if (threadIdx.x == 0) found = 0xffffffffu;
    __syncthreads();
    for (uint32_t base = st->cursor; base < S; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        if (i < S && __ldcg(&field[i]) == kFree) atomicMin(&found, i);     // past L1: other blocks just wrote
        __syncthreads();
        if (found != 0xffffffffu) break;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint32_t a = found;
        st->cursor = a;
        st->anchor = a;
        if (a < S) {
            const uint32_t v = vox[a];
            st->ax = v % (uint32_t)gx;
            st->ay = (v / (uint32_t)gx) % (uint32_t)gy;
            st->az = v / ((uint32_t)gx * (uint32_t)gy);
        } else {
            st->status = 1u;
        }
        st->rank_left = s_minus_1;
        st->prefix = 0ull;
    }
}

__global__ void __launch_bounds__(1024) k_anchor(const uint16_t *field, uint32_t S, const uint32_t *vox, int gx,
                                                 int gy, AssignState *st, uint32_t s_minus_1)
{
    find_anchor(field, S, vox, gx, gy, st, s_minus_1);
}

// true in the one block that finishes last (after every block's global
// writes of this launch are visible)
__device__ __forceinline__ bool last_block(AssignState *st)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ unsigned long long key_of(const AssignState &st, uint32_t v, uint32_t rank, int gx, int gy)
{
    const int x = (int)(v % (uint32_t)gx), y = (int)((v / (uint32_t)gx) % (uint32_t)gy),
              z = (int)(v / ((uint32_t)gx * (uint32_t)gy));
    const long long dx = x - (int)st.ax, dy = y - (int)st.ay, dz = z - (int)st.az;
    const unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
    return (d2 << kRankBits) | rank;
}

// Histogram of digit `pass` (0 = most significant) of the keys matching the
// prefix (shared-memory bins, then global atomics); then, in the block that
// finishes last, the select: the bin holding rank_left extends the prefix by
// one digit (512 threads, 8 bins each), and the histogram is cleared.
__global__ void __launch_bounds__(512) k_hist_select(const uint16_t *field, uint32_t S, const uint32_t *vox, int gx,
                                                     int gy, AssignState *st, int pass, uint32_t *hist)
{
    __shared__ uint32_t sh[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    {
        const AssignState sv = *st;
        const int shift = (3 - pass) * kDigitBits;
        // eight candidates per thread per round, their loads issued together
        // (one dependent load after another per voxel would leave the SMs
        // waiting on L2 latency)
        constexpr int kU = 8;
        const uint32_t stride = gridDim.x * blockDim.x;
        for (uint32_t i0 = sv.cursor + blockIdx.x * blockDim.x + threadIdx.x; i0 < S; i0 += kU * stride) {
            uint16_t fv[kU];
            uint32_t vv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t i = i0 + (uint32_t)u * stride;
                fv[u] = i < S ? field[i] : (uint16_t)0;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t i = i0 + (uint32_t)u * stride;
                vv[u] = fv[u] == kFree && i < S ? vox[i] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t i = i0 + (uint32_t)u * stride;
                if (fv[u] != kFree || i >= S) continue;
                const unsigned long long k = key_of(sv, vv[u], i, gx, gy);
                if (pass > 0 && (k >> (shift + kDigitBits)) != sv.prefix) continue;
                atomicAdd(&sh[(k >> shift) & (kBins - 1)], 1u);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
    if (!last_block(st)) return;
    // select: the bin holding rank_left (hist read from L2, where the atomics landed)
    const int t = threadIdx.x;
    const uint32_t want = st->rank_left;
    uint32_t c[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { c[q] = __ldcg(&hist[8 * t + q]); sum += c[q]; }
    uint32_t *part = sh;                      // reuse: the block's histogram is flushed
    __syncthreads();
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 512; o <<= 1) {
        const uint32_t v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const uint32_t before = t > 0 ? part[t - 1] : 0u;
    if (want >= before && want < part[t]) {
        uint32_t acc = before;
        for (int q = 0; q < 8; ++q) {
            if (want < acc + c[q]) {
                st->prefix = (st->prefix << kDigitBits) | (unsigned long long)(8 * t + q);
                st->rank_left = want - acc;
                break;
            }
            acc += c[q];
        }
    }
    if (t == 511 && want >= part[511]) st->status = 1u;      // fewer candidates than asked for
#pragma unroll
    for (int q = 0; q < 8; ++q) hist[8 * t + q] = 0u;
    if (t == 0) st->done = 0u;
}

// every unassigned voxel whose key is <= the selected key joins network
// `net`; then, in the block that finishes last, the next network's anchor
__global__ void __launch_bounds__(1024) k_take_anchor(uint16_t *field, uint32_t S, const uint32_t *vox, int gx, int gy,
                                                      AssignState *st, uint16_t net, uint32_t s_minus_1)
{
    {
        const AssignState sv = *st;
        const unsigned long long thr = sv.prefix;
        for (uint32_t i = sv.cursor + blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
            if (field[i] != kFree) continue;
            if (key_of(sv, vox[i], i, gx, gy) <= thr) field[i] = net;
        }
    }
    if (!last_block(st)) return;
    if (threadIdx.x == 0) st->done = 0u;
    find_anchor(field, S, vox, gx, gy, st, s_minus_1);
}

__global__ void k_take_rest(uint16_t *field, uint32_t S, uint16_t net)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x)
        if (field[i] == kFree) field[i] = net;
}

__global__ void k_boxes(const uint16_t *field, uint32_t S, const uint32_t *vox, int gx, int gy, int32_t *boxes)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        const uint32_t v = vox[i];
        const int x = (int)(v % (uint32_t)gx), y = (int)((v / (uint32_t)gx) % (uint32_t)gy),
                  z = (int)(v / ((uint32_t)gx * (uint32_t)gy));
        int32_t *b = boxes + 6 * (int64_t)field[i];
        atomicMin(&b[0], x); atomicMin(&b[1], y); atomicMin(&b[2], z);
        atomicMax(&b[3], x + 1); atomicMax(&b[4], y + 1); atomicMax(&b[5], z + 1);
    }
}

__global__ void k_boxes_init(int32_t *boxes, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        boxes[6 * i + 0] = boxes[6 * i + 1] = boxes[6 * i + 2] = 0x7fffffff;
        boxes[6 * i + 3] = boxes[6 * i + 4] = boxes[6 * i + 5] = 0;
    }
}

}  // namespace

size_t assign_scratch_bytes() { return sizeof(AssignState) + kBins * sizeof(uint32_t); }

void launch_assign(const uint32_t *bits, const uint32_t *prefix, int64_t n_words, int gx, int gy, uint32_t S, int n,
                   uint32_t *vox, uint16_t *field, int32_t *boxes, void *scratch, int n_sm, cudaStream_t s)
{
    AssignState *st = reinterpret_cast<AssignState *>(scratch);
    uint32_t *hist = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(scratch) + sizeof(AssignState));
    cudaMemsetAsync(scratch, 0, assign_scratch_bytes(), s);
    cudaMemsetAsync(field, 0xff, (size_t)S * sizeof(uint16_t), s);
    k_occupied_list<<<n_sm * 8, 256, 0, s>>>(bits, prefix, n_words, vox);
    const uint32_t per = S / (uint32_t)n;
    const int grid = n_sm * 4;
    // per network: 4 digit passes (histogram, then the select in the block
    // that finishes last) and the take (then the next anchor, likewise)
    if (n > 1) k_anchor<<<1, 1024, 0, s>>>(field, S, vox, gx, gy, st, per - 1u);
    for (int k = 0; k + 1 < n; ++k) {
        // one block per SM: fewer blocks flushing their shared histograms
        // (the first digits fall in a few bins, whose global atomics collide)
        for (int pass = 0; pass < 4; ++pass)
            k_hist_select<<<n_sm, 512, 0, s>>>(field, S, vox, gx, gy, st, pass, hist);
        k_take_anchor<<<grid, 1024, 0, s>>>(field, S, vox, gx, gy, st, (uint16_t)k, per - 1u);
    }
    k_take_rest<<<grid, 256, 0, s>>>(field, S, (uint16_t)(n - 1));
    if (boxes) {
        k_boxes_init<<<(n + 255) / 256, 256, 0, s>>>(boxes, n);
        k_boxes<<<grid, 256, 0, s>>>(field, S, vox, gx, gy, boxes);
    }
}

uint32_t assign_status(const void *scratch)
{
    AssignState st{};
    cudaMemcpy(&st, scratch, sizeof(st), cudaMemcpyDeviceToHost);
    return st.status;
}

}  // namespace roam
