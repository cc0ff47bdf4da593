// Adaptive assignment of the occupied voxels to n networks (Alg. 1 stage
// II, Sec. "Adaptive Radiance Fields Slimming and Fine-tuning"): network k
// takes the smallest unassigned voxel (lexicographic (z, y, x), i.e. the
// smallest linear index) as its anchor plus the s - 1 unassigned voxels
// nearest to it (squared distance in voxel units, ties to the smaller linear
// index), s = S / n; the last network takes what remains.
//
// The networks are built one after the other (each depends on the voxels
// the earlier ones took); within a network everything is data parallel:
//   k_anchor    one block: the first unassigned voxel from a cursor
//   k_hist      per digit of the 47-bit key (squared distance << 27 |
//               rank), a histogram of the candidates matching the digits
//               fixed so far (shared-memory bins, then global atomics)
//   k_select    one block: the bin holding the wanted rank; the key prefix
//               grows by one digit (4 digits of 12 bits)
//   k_take      every unassigned voxel whose key is <= the selected key
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

__global__ void __launch_bounds__(1024) k_anchor(const uint16_t *field, uint32_t S, const uint32_t *vox, int gx,
                                                 int gy, AssignState *st, uint32_t s_minus_1)
{
    __shared__ uint32_t found;
    if (threadIdx.x == 0) found = 0xffffffffu;
    __syncthreads();
    for (uint32_t base = st->cursor; base < S; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        if (i < S && field[i] == kFree) atomicMin(&found, i);
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

__device__ __forceinline__ unsigned long long key_of(const AssignState &st, uint32_t v, uint32_t rank, int gx, int gy)
{
    const int x = (int)(v % (uint32_t)gx), y = (int)((v / (uint32_t)gx) % (uint32_t)gy),
              z = (int)(v / ((uint32_t)gx * (uint32_t)gy));
    const long long dx = x - (int)st.ax, dy = y - (int)st.ay, dz = z - (int)st.az;
    const unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
    return (d2 << kRankBits) | rank;
}

// histogram of digit `pass` (0 = most significant) of the keys matching the prefix
__global__ void __launch_bounds__(512) k_hist(const uint16_t *field, uint32_t S, const uint32_t *vox, int gx, int gy,
                                              const AssignState *st_p, int pass, uint32_t *hist)
{
    __shared__ uint32_t sh[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const AssignState st = *st_p;
    const int shift = (3 - pass) * kDigitBits;
    for (uint32_t i = st.cursor + blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        if (field[i] != kFree) continue;
        const unsigned long long k = key_of(st, vox[i], i, gx, gy);
        if (pass > 0 && (k >> (shift + kDigitBits)) != st.prefix) continue;
        atomicAdd(&sh[(k >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

// one block of kBins / 4 threads: the bin holding rank_left; clears the histogram
__global__ void __launch_bounds__(1024) k_select(uint32_t *hist, AssignState *st)
{
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;               // 4 bins per thread
    const uint32_t want = st->rank_left;     // read by every thread before any write below
    uint32_t c[4], sum = 0;
    for (int q = 0; q < 4; ++q) { c[q] = hist[4 * t + q]; sum += c[q]; }
    part[t] = sum;
    __syncthreads();
    // inclusive scan over the 1024 partial sums
    for (int o = 1; o < 1024; o <<= 1) {
        const uint32_t v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const uint32_t before = t > 0 ? part[t - 1] : 0u;
    if (want >= before && want < part[t]) {
        uint32_t acc = before;
        for (int q = 0; q < 4; ++q) {
            if (want < acc + c[q]) {
                st->prefix = (st->prefix << kDigitBits) | (unsigned long long)(4 * t + q);
                st->rank_left = want - acc;
                break;
            }
            acc += c[q];
        }
    }
    if (t == 1023 && want >= part[1023]) st->status = 1u;   // fewer candidates than asked for
    for (int q = 0; q < 4; ++q) hist[4 * t + q] = 0u;
}

__global__ void k_take(uint16_t *field, uint32_t S, const uint32_t *vox, int gx, int gy, const AssignState *st_p,
                       uint16_t net)
{
    const AssignState st = *st_p;
    const unsigned long long thr = st.prefix;   // the (s-1)-th smallest key
    for (uint32_t i = st.cursor + blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        if (field[i] != kFree) continue;
        if (key_of(st, vox[i], i, gx, gy) <= thr) field[i] = net;
    }
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
    for (int k = 0; k + 1 < n; ++k) {
        k_anchor<<<1, 1024, 0, s>>>(field, S, vox, gx, gy, st, per - 1u);
        for (int pass = 0; pass < 4; ++pass) {
            k_hist<<<grid, 512, 0, s>>>(field, S, vox, gx, gy, st, pass, hist);
            k_select<<<1, 1024, 0, s>>>(hist, st);
        }
        k_take<<<grid, 256, 0, s>>>(field, S, vox, gx, gy, st, (uint16_t)k);
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
