// Adjoint of the per-field tiny MLPs on the 5th-generation tensor cores
// (BF16 operands, FP32 accumulation), for the fine-tuning step (L2 loss on
// rendered pixels) and the distillation step (Eq. 7).  One CTA per SM walks
// a contiguous run of 128-sample tiles of the bucketed samples; per tile it
//   1. recomputes the forward chain with tcgen05.mma (A = the layer input in
//      shared memory, B = the field's weight image), keeping every layer's
//      input X_l [128 samples x K] in shared memory,
//   2. walks the layers backwards: per layer
//        dgrad   dX = dZ W          D[128 x W]  += dZ (K-major) * image (MN-major)
//        wgrad   dW^T += X^T dZ     D[K x N]    += X (MN-major) * dZ (MN-major)
//      where the wgrad accumulators of all layers stay in TMEM across the
//      tiles of one field and are added to the global FP32 gradient (one
//      atomic per parameter) when the field changes.  The MMAs of one
//      backward group write independent accumulators, so up to three warps
//      issue them side by side.
// Two chains of 8 warps carry alternate tiles (t0 + chain, + 2, ...): while
// one recomputes its tile's forward, the other runs the previous tile's
// backward, so the commit round trips of one chain overlap the other's
// epilogues.  Each chain has its own accumulator D, barrier and two MMA
// mbarriers: in a backward group the dgrad MMAs land on one, the wgrad MMAs
// on the other, so the dX epilogue (TMEM load, ReLU mask, packing) runs
// while the wgrad MMAs still read dZ, and dZ is rewritten once both have
// landed.  Within a chain the two warps of one TMEM lane quarter take half
// of the row's columns each.  The chains share the weight image (their
// tiles are of one field: a field change drains them), the wgrad
// accumulators, a pool of H + 4 activation chunks, dZ and the tail chunk;
// a progress word per chain orders every reuse (see prog_word), so wgrad
// accumulation stays in tile order.
//
// Every activation tile exists once, in the 128-byte-swizzled layout with
// samples as rows and 64 features per 128-byte row ("natural" layout).  Read
// with K = features it is the K-major A operand of the forward and dgrad
// MMAs; read with K = samples it is the MN-major operand of the wgrad MMAs
// (64-feature blocks LBO apart, 8-sample groups 1024 bytes apart).  The
// weight image of the forward kernel, read MN-major, is the B operand of
// the dgrad MMAs (B[k_in][n_out] = W[n_out][k_in]).  Biases ride in the
// MMAs as in the forward kernel (a constant-1 feature column), so their
// gradients come out of the wgrad accumulators as one more feature row.
//
// Shared memory (W = 64): the image; H + 4 chunks of 64 columns for the
// two chains' X_0 (encoding), X_1..X_H (hidden inputs), X_{H+1} (colour
// input) and X_g (colour output); dZ (one chunk); and the tail chunk T whose
// columns 0..31 hold [1 | F(d) | 0] of the tile in its colour layer (the
// second K chunk of the hidden, head and colour layers), columns 32..47 the
// head's dZ columns 64..79 or the output layer's dZ, columns 48..63 the
// colour layer's partial sums.  At W = 32 the tail [1 | F(d) | 0] sits inside
// each chunk (columns 32..63) and T only pads the M = 128 wgrad operand
// besides holding the output layer's dZ and the partial sums.
#include "tc_common.cuh"
#include <cuda_bf16.h>

namespace roam {

namespace {
constexpr int kChunk = 16384;       // one 64-column chunk of 128 rows
constexpr int kChains = 2;          // independent tile chains per CTA
constexpr int kChainThreads = 256;  // 8 warps: 2 column groups x 4 TMEM lane quarters
constexpr int kBwThreads = kChains * kChainThreads;

template <int W, int H>
struct BwShape {
    using S = TcShape<W, H, false>;
    static_assert(S::kFold, "the tensor-core adjoint folds every bias into the MMAs (BF16, W <= 64)");
    static constexpr int kNBuf = H + 4;               // activation chunks shared by the two chains
    static constexpr int kOffX = S::kImageAlloc;
    static constexpr int kOffDZ = kOffX + kNBuf * kChunk;
    static constexpr int kOffT = kOffDZ + kChunk;     // after dZ: the head's dZ columns past 64 live in T
    static constexpr int kSmem = kOffT + kChunk;
    // TMEM: each chain's D (forward / dgrad accumulator), then one wgrad
    // accumulator per layer l = 0 .. H+2 (H+2 = the 3-output layer)
    static constexpr int kDCols = S::N_HEAD;
    __host__ __device__ static constexpr int wN(int l) { return l == H ? S::N_HEAD : (l == H + 2 ? 16 : W); }
    __host__ __device__ static constexpr int wcol(int l)
    {
        int c = kChains * kDCols;
        for (int i = 0; i < l; ++i) c += wN(i);
        return c;
    }
    static constexpr int kCols = wcol(H + 3);
    static_assert(kCols <= 512, "TMEM holds both chains' D and every layer's wgrad accumulator");
    // physical chunk of X_j for a tile of chain parity p: even tiles use
    // 0 .. H+2, odd tiles H+3 for X_0 and H+3-j for j >= 1, so X_j of one
    // chain reuses the chunk of the other chain's X_{H+3-j}
    __host__ __device__ static constexpr int buf(int p, int j) { return p == 0 ? j : (j == 0 ? H + 3 : H + 3 - j); }
};

// Progress of a chain through its current tile, in one word:
// (tile index within the CTA's run + 1) << 4 | n, where n = 0 when the
// tile has started (its field's image is in place), n = 2 when its colour
// and output wgrads have landed (X_{H+2}, X_{H+1} and the tail's F(d)
// columns are free), n = H + 3 - l once X_l is free (its mask read by the
// epilogue of layer l), and n = H + 3 when the tile is done (X_0, dZ and
// every wgrad MMA).  Words only grow.
__host__ __device__ constexpr uint32_t prog_word(uint32_t u_rel, uint32_t n) { return ((u_rel + 1u) << 4) | n; }

// Waits until the other chain's progress word reaches `need`; false on an
// abort (flagged by any thread) or after the wait limit.
__device__ __forceinline__ bool wait_prog(const volatile uint32_t *p, uint32_t need, volatile int *abort_flag,
                                          uint32_t *status)
{
    if (*p >= need) {
        __threadfence_block();
        return true;
    }
    const unsigned long long t0 = now_ns();
    for (;;) {
        __nanosleep(32);
        if (*p >= need) {
            __threadfence_block();
            return true;
        }
        if (*abort_flag) return false;
        if (now_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}

// byte offset of 16-byte unit u (8 BF16 elements) of row r within a chunk
__device__ __forceinline__ uint32_t sw_off(int r, int u)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((u ^ (r & 7)) << 4));
}

// writes units [u0, u0 + n) of row r from packed BF16 pairs p[4 (u - u0) ..]
template <int N>
__device__ __forceinline__ void st_units(uint8_t *chunk, int r, int u0, const uint32_t (&p)[4 * N])
{
#pragma unroll
    for (int u = 0; u < N; ++u)
        *reinterpret_cast<uint4 *>(chunk + sw_off(r, u0 + u)) = make_uint4(p[4 * u], p[4 * u + 1], p[4 * u + 2],
                                                                           p[4 * u + 3]);
}

// the 16 TMEM columns [c, c + 16) of this thread's lane as floats
__device__ __forceinline__ void ld16f(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    tmem_ld16_nowait(taddr, r);
    tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// 0xffff in each 16-bit half of x (two BF16 activations) that is > 0, else
// 0: the ReLU derivative as a mask for a packed BF16 pair
__device__ __forceinline__ uint32_t relu_mask(uint32_t x)
{
    return __hgt2_mask(*reinterpret_cast<const __nv_bfloat162 *>(&x), __float2bfloat162_rn(0.f));
}

// one TMEM column of this thread's lane (complete after tcgen05.wait::ld)
__device__ __forceinline__ uint32_t tmem_ld1_nowait(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return r;
}

// one arrival without a transaction (no tcgen05 work to track)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// N (8 or 16) consecutive TMEM columns of this thread's lane as floats
template <int N>
__device__ __forceinline__ void ldcf(uint32_t taddr, float (&v)[N])
{
    static_assert(N == 8 || N == 16, "one x8 or x16 load");
    if constexpr (N == 16) {
        ld16f(taddr, v);
    } else {
        uint32_t r[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr));
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
    }
}

constexpr int kFreqX = (kPeX - 3) / 6;     // frequencies of F(x)

// frequency k of F(x) fills columns [3 + 6k, 9 + 6k) of X_0
__host__ __device__ constexpr bool freq_meets(int k, int lo, int hi) { return 3 + 6 * k < hi && 9 + 6 * k > lo; }
__host__ __device__ constexpr int freq_last(int lo, int hi)
{
    int r = -1;
    for (int k = 0; k < kFreqX; ++k)
        if (freq_meets(k, lo, hi)) r = k;
    return r;
}
__host__ __device__ constexpr int freq_first(int lo, int hi)
{
    for (int k = 0; k < kFreqX; ++k)
        if (freq_meets(k, lo, hi)) return k;
    return kFreqX;
}

// Columns [16 G, 16 G + 16) of X_0 = [x | sin, cos (2^k pi x), k < 10 | 1]
// as 8 packed BF16 pairs.  The same arithmetic as the forward kernel's
// encoding (direct evaluation at k = 0 and k = 5, angle doubling in
// between), so the recomputed chain sees the forward's operands bit for bit;
// only the frequencies this block's columns (or their doubling chain) need
// are evaluated.
template <int G>
__device__ __forceinline__ void enc_x0(const float (&xl)[3], uint32_t (&p)[8])
{
    constexpr int lo = 16 * G, hi = lo + 16;
    constexpr int k_hi = freq_last(lo, hi);
    constexpr int k_start = freq_first(lo, hi) >= 5 ? 5 : 0;
    float e[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) e[q] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a >= lo && a < hi) e[a - lo] = xl[a];
    if (63 >= lo && 63 < hi) e[63 - lo] = 1.0f;
    // (x, y) as packed pairs (each half rounded as the scalar operation), z alone
    float2 s01 = make_float2(0.f, 0.f), c01 = make_float2(1.f, 1.f);
    float s2 = 0.f, c2 = 1.f;
#pragma unroll
    for (int k = k_start; k <= k_hi; ++k) {
        if (k == 0 || k == 5) {
            sincospi_fast(xl[0] * (float)(1 << k), s01.x, c01.x);
            sincospi_fast(xl[1] * (float)(1 << k), s01.y, c01.y);
            sincospi_fast(xl[2] * (float)(1 << k), s2, c2);
        } else {
            const float2 t01 = __fmul2_rn(make_float2(2.0f, 2.0f), s01);
            const float2 sn01 = __fmul2_rn(t01, c01);
            c01 = __ffma2_rn(make_float2(-t01.x, -t01.y), s01, make_float2(1.0f, 1.0f));
            s01 = sn01;
            const float t2 = 2.0f * s2;
            const float sn2 = t2 * c2;
            c2 = fmaf(-t2, s2, 1.0f);
            s2 = sn2;
        }
        const float sn[3] = {s01.x, s01.y, s2}, cs[3] = {c01.x, c01.y, c2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int cs_col = 3 + 6 * k + a, cc_col = 6 + 6 * k + a;
            if (cs_col >= lo && cs_col < hi) e[cs_col - lo] = sn[a];
            if (cc_col >= lo && cc_col < hi) e[cc_col - lo] = cs[a];
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = pack_bf16(e[2 * q], e[2 * q + 1]);
}

// The MMA groups of the adjoint, fully unrolled: each operand descriptor is
// built once and stepped by compile-time offsets (16-byte units), so that an
// N <= 64 MMA issues in its ~25 ns slot instead of ~80 ns with a descriptor
// rebuilt per instruction.
//   forward layer: D[s][n] = sum_k X[s][k] W[n][k]; K-major A (X, then the
//   tail chunk T past column 64) and B (the image), K / 16 MMAs
template <int K, int N>
__device__ __forceinline__ void mma_fwd(uint32_t tD, uint32_t xa, uint32_t st, uint32_t ba)
{
    constexpr uint32_t idesc = idesc_bf16_t(N, 0, 0);
    const uint64_t dx = sdesc(xa), dt = sdesc(st), db = sdesc(ba);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
        const int ch = ks >> 2, kin = ks & 3;
        umma_ss(tD, (ch == 0 ? dx : dt) + (uint64_t)(kin * 2), db + (uint64_t)((ch * N * 128 + kin * 32) >> 4), idesc,
                ks > 0 ? 1u : 0u);
    }
}
//   wgrad: D_w[k][n] (+)= sum_s X[s][k] dZ[s][n]; both operands MN-major,
//   8 MMAs of 16 samples (two 8-row groups, 2048 bytes) each
template <int N>
__device__ __forceinline__ void mma_wgrad(uint32_t td, uint32_t xa, uint32_t lbo_x, uint32_t dza, uint32_t dz_lbo,
                                          uint32_t acc0)
{
    constexpr uint32_t idesc = idesc_bf16_t(N, 1, 1);
    const uint64_t da = sdesc_mn(xa, lbo_x), db = sdesc_mn(dza, dz_lbo);
#pragma unroll
    for (int j = 0; j < 8; ++j)
        umma_ss(td, da + (uint64_t)(j * 128), db + (uint64_t)(j * 128), idesc, (j > 0 || acc0) ? 1u : 0u);
}
//   dgrad: D[s][k] = sum_n dZ[s][n] W[n][k], k < W; A = dZ K-major (its
//   columns 64..79, the head's, at sdz_hi), B = the image read MN-major,
//   Kn / 16 MMAs
template <int W, int Kn>
__device__ __forceinline__ void mma_dgrad(uint32_t tD, uint32_t sdz, uint32_t sdz_hi, uint32_t ba)
{
    static_assert(Kn <= 80, "dZ columns 64..79 at most past the first chunk");
    constexpr uint32_t idesc = idesc_bf16_t(W, 0, 1);
    const uint64_t da = sdesc(sdz), dh = sdesc(sdz_hi), db = sdesc_mn(ba, 1024u);
#pragma unroll
    for (int ks = 0; ks < Kn / 16; ++ks)
        umma_ss(tD, (ks < 4 ? da + (uint64_t)(ks * 2) : dh), db + (uint64_t)(ks * 128), idesc, ks > 0 ? 1u : 0u);
}

// Where feature row k of wgrad accumulator l lands in the API layout (per
// layer row-major [out][in] then bias[out]): column n (n < n_rows) goes to
// base + n * stride; the head's column W (its density logit, API row 0) to
// base0.  base < 0: the row holds no parameter.
struct RowMap {
    int64_t base, stride, base0;
    int n_rows;
};

template <int W, int H>
__device__ __forceinline__ RowMap row_map(int l, int k)
{
    const int64_t o_hid = (int64_t)W * kPeX + W;
    const int64_t o_head = o_hid + (int64_t)(H - 1) * (W * W + W);
    const int64_t o_col = o_head + (int64_t)(1 + W) * W + (1 + W);
    const int64_t o_out = o_col + (int64_t)W * (W + kPeD) + W;
    RowMap m{-1, 0, -1, 0};
    if (l == 0) {
        m.n_rows = W;
        if (k < kPeX) { m.base = k; m.stride = kPeX; }
        else if (k == kPeX) { m.base = (int64_t)W * kPeX; m.stride = 1; }
    } else if (l < H) {
        m.n_rows = W;
        const int64_t ob = o_hid + (int64_t)(l - 1) * (W * W + W);
        if (k < W) { m.base = ob + k; m.stride = W; }
        else if (k == W) { m.base = ob + (int64_t)W * W; m.stride = 1; }
    } else if (l == H) {
        // MMA columns: W features (API rows 1..W), then the density logit (API row 0)
        m.n_rows = W;
        if (k < W) { m.base = o_head + W + k; m.stride = W; m.base0 = o_head + k; }
        else if (k == W) { m.base = o_head + (int64_t)(1 + W) * W + 1; m.stride = 1; m.base0 = o_head + (int64_t)(1 + W) * W; }
    } else if (l == H + 1) {
        m.n_rows = W;
        const int kc = W + kPeD;
        if (k < W) { m.base = o_col + k; m.stride = kc; }
        else if (k == W) { m.base = o_col + (int64_t)W * kc; m.stride = 1; }
        else if (k <= W + kPeD) { m.base = o_col + (k - 1); m.stride = kc; }
    } else {
        m.n_rows = 3;
        if (k < W) { m.base = o_out + k; m.stride = W; }
        else if (k == W) { m.base = o_out + 3 * (int64_t)W; m.stride = 1; }
    }
    return m;
}


template <int W, int H>
__global__ void __launch_bounds__(kBwThreads, 1)
    k_mlp_bwd_tc(const void *wimg, int64_t img_bytes, const float *affine, float sig_scale, int act, int64_t P,
                 SampleSrc src, BucketBufs b, Counters *ctr, const float4 *gsr, float *grad)
{
    using S = TcShape<W, H, false>;
    using B = BwShape<W, H>;
    constexpr int kLayers = S::kLayers;              // tensor-core layers of the forward chain
    constexpr int kStageRec = kLayers >= 5 ? 2 : 1;  // the layer that gathers the chain's next records
    constexpr int CW = W / 2;                        // columns of one thread's share of a row
    constexpr int NSB = CW / 16;                     // ... in 16-column sub-blocks
    constexpr uint32_t kFull = (uint32_t)(H + 3);
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_d[kChains], bar_g[kChains], bar_w;
    __shared__ uint32_t tmem_slot, img_field, n_img;
    __shared__ volatile uint32_t prog[kChains];
    __shared__ int abort_flag;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t *sm = smem_raw + (base - smem_u32(smem_raw));
    uint8_t *IMG = sm;
    uint8_t *DZ = sm + B::kOffDZ;
    uint8_t *T = sm + B::kOffT;
    const uint32_t sIMG = base, sX = base + B::kOffX, sDZ = base + B::kOffDZ, sT = base + B::kOffT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chain = warp >> 3;                      // tiles t0 + chain, t0 + chain + 2, ...
    const int cw = warp & 7;                          // warp within the chain
    const int quarter = warp & 3;                     // TMEM lane quarter this warp may access
    const int g = cw >> 2;                            // column group within the chain
    const int row = quarter * 32 + lane;              // TMEM lane == tile row == sample
    const int c0 = g * CW;                            // first column of this thread's share
    const int ctid = tid & (kChainThreads - 1);
    const bool lead = lane == 0 && cw < 4;            // commits each MMA group (issuers: chain warps 0..2)
    volatile int *abortp = &abort_flag;
    uint32_t *status = &ctr->status;

    if (tid == 0) {
        mbar_init(&bar_d[0], 4);
        mbar_init(&bar_d[1], 4);
        mbar_init(&bar_g[0], 2);
        mbar_init(&bar_g[1], 2);
        mbar_init(&bar_w, 1);
        abort_flag = 0;
        img_field = 0xffffffffu;
        n_img = 0;
        prog[0] = 0u;
        prog[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // T: zero, with the constant-1 column 0 that the hidden, head and colour
    // layers' bias rows read (W = 64; at W = 32 T only pads the wgrad operands)
    for (int q = tid; q < kChunk / 16; q += kBwThreads) reinterpret_cast<uint4 *>(T)[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (W == 64 && tid < 128) *reinterpret_cast<uint32_t *>(T + sw_off(tid, 0)) = pack_bf16(1.0f, 0.f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = (uint32_t)(quarter * 32) << 16;
    const uint32_t tD = tmem + (uint32_t)(chain * B::kDCols);
    const uint32_t tDc = tD + tlane + (uint32_t)c0;   // this thread's share of its chain's D
    // every wgrad accumulator starts at zero (the MMAs always accumulate)
    {
        uint32_t z[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) z[q] = 0u;
        for (int l = 0; l < H + 3; ++l)
            for (int c = 16 * (warp >> 2); c < B::wN(l); c += 64) tmem_st16(tmem + tlane + (uint32_t)(B::wcol(l) + c), z);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t n_tiles = ctr->n_tiles;
    const uint32_t t0 = (uint32_t)((uint64_t)n_tiles * blockIdx.x / gridDim.x);
    const uint32_t t1 = (uint32_t)((uint64_t)n_tiles * (blockIdx.x + 1) / gridDim.x);
    const volatile uint32_t *other = &prog[chain ^ 1];

    uint32_t d_ph = 0, g_ph = 0;
    int d_open = -1, g_open = -1;        // a lead's committed phase not yet waited for
    bool w_pending = false;              // an image load in flight (the issuing thread's view)
    bool aborted = false;


    // the chain's barrier: its threads' generic shared-memory stores become
    // visible to the MMAs, and it agrees on `good` (every thread's last wait)
    auto publish = [&](bool good) -> bool {
        fence_async_smem();
        tc_fence_before();
        const bool bad = named_sync_or(1 + chain, kChainThreads, !good || *abortp);
        tc_fence_after();
        return !bad;
    };
    auto commit = [&]() {
        if (lead) {
            umma_commit(&bar_d[chain]);
            d_open = (int)d_ph;
        }
    };
    // a backward group: the wgrad issuers (chain warps 0 and 1) commit to
    // bar_g and only arrive on bar_d, so that bar_d lands with the dgrad
    // (warp 2) and the dX epilogue overlaps the wgrad MMAs
    auto commit_split = [&]() {
        if (lead) {
            if (cw < 2) {
                umma_commit(&bar_g[chain]);
                g_open = (int)g_ph;
                mbar_arrive(&bar_d[chain]);
            } else {
                umma_commit(&bar_d[chain]);
                d_open = (int)d_ph;
            }
        }
    };
    // wait for the chain's committed group: true when it landed
    auto land = [&]() -> bool {
        const bool got = mbar_wait(&bar_d[chain], d_ph, abortp, status);
        if (got) d_open = -1;
        d_ph ^= 1u;
        tc_fence_after();
        return got;
    };
    // ... and for its wgrad MMAs (before dZ, the tail or an X they read is rewritten)
    auto land_g = [&]() -> bool {
        const bool got = mbar_wait(&bar_g[chain], g_ph, abortp, status);
        if (got) g_open = -1;
        g_ph ^= 1u;
        tc_fence_after();
        return got;
    };
    // the chain's progress word (by its first thread, after whatever the
    // word promises has happened for every thread of the chain)
    auto progress = [&](uint32_t u_rel, uint32_t n) {
        if (ctid == 0) {
            __threadfence_block();
            prog[chain] = prog_word(u_rel, n);
        }
    };
    // add the wgrad accumulators of field f to the global gradient and clear
    // them; the 16-column pieces of each layer go round `ng` column groups
    auto flush = [&](uint32_t f, int gid, int ng) {
        float *gf = grad + (int64_t)f * P;
        uint32_t z[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) z[q] = 0u;
#pragma unroll 1
        for (int l = 0; l < H + 3; ++l) {
            const RowMap m = row_map<W, H>(l, row);
#pragma unroll 1
            for (int c = 16 * gid; c < B::wN(l); c += 16 * ng) {
                const uint32_t ta = tmem + tlane + (uint32_t)(B::wcol(l) + c);
                float v[16];
                ld16f(ta, v);
                tmem_st16(ta, z);
                if (m.base < 0) continue;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c + q;
                    if (v[q] == 0.f) continue;
                    if (n < m.n_rows) atomicAdd(gf + m.base + (int64_t)n * m.stride, v[q]);
                    else if (n == W && m.base0 >= 0) atomicAdd(gf + m.base0, v[q]);
                }
            }
        }
        tmem_wait_st();
        tc_fence_before();
    };
    // 16-byte unit u of row `row` in chunk X_j of a tile of parity p
    auto xchunk = [&](int p, int j) -> uint8_t * { return sm + B::kOffX + B::buf(p, j) * kChunk; };
    auto xaddr = [&](int p, int j) -> uint32_t { return sX + (uint32_t)(B::buf(p, j) * kChunk); };


    // the chain's tiles t0 + chain, t0 + chain + 2, ...: the current one, the
    // next (its sample gathered in stages during this one) and the one after
    Tile tl_cur{0u, 0u, 0u, 0u}, tl_nx{0u, 0u, 0u, 0u};
    SampleIn nxt{0u, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    Pending pend{};
    float aff_n[6] = {1.f, 1.f, 1.f, 0.f, 0.f, 0.f};  // the next tile's affine map
    auto load_aff = [&](const Tile &tt) {
        if (tt.count == 0) return;
        const float *af = affine + 6 * (int64_t)tt.field;
#pragma unroll
        for (int q = 0; q < 6; ++q) aff_n[q] = __ldg(af + q);
    };
    if (t0 + chain < t1) {
        tl_cur = b.tiles[t0 + chain];
        nxt = fetch_sample(src, b, tl_cur, row);
        load_aff(tl_cur);
        if (t0 + chain + kChains < t1) tl_nx = b.tiles[t0 + chain + kChains];
    }
    uint32_t w_pend_ph = 0;
    bool good = true;                    // this thread's last wait
#pragma unroll 1
    for (uint32_t t = t0 + chain; t < t1 && !aborted; t += kChains) {
        const uint32_t u_rel = t - t0;
        const Tile tl = tl_cur;
        const bool more = t + kChains < t1;
        const Tile tl_next = tl_nx;
        tl_nx = t + 2 * kChains < t1 ? b.tiles[t + 2 * kChains] : Tile{0u, 0u, 0u, 0u};
        tl_cur = tl_next;
        const SampleIn smp = nxt;
        float aff[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) aff[q] = aff_n[q];
        if (tl.count == 0) {
            // keeps the run's order: done once the tile before it is
            bool ok = good && (u_rel == 0 || wait_prog(other, prog_word(u_rel - 1, kFull), abortp, status));
            if (!publish(ok)) {
                aborted = true;
                break;
            }
            progress(u_rel, kFull);
            if (more) {
                nxt = fetch_sample(src, b, tl_next, row);
                load_aff(tl_next);
            }
            continue;
        }
        // the tile before has settled the image (its field is img_field)
        bool ok = good && (u_rel == 0 || wait_prog(other, prog_word(u_rel - 1, 0), abortp, status));
        if (!publish(ok)) {
            aborted = true;
            break;
        }
        if (tl.field != img_field) {
            // a new field: every tile of the old one done, its gradient
            // flushed, then this field's image
            ok = u_rel == 0 || wait_prog(other, prog_word(u_rel - 1, kFull), abortp, status);
            if (!publish(ok)) {
                aborted = true;
                break;
            }
            if (img_field != 0xffffffffu) flush(img_field, g, 2);
            // generic reads of the old image come before the bulk copy that
            // overwrites it (the other chain fenced its own before its last word)
            if (!publish(true)) {
                aborted = true;
                break;
            }
            const uint32_t wph = n_img & 1u;
            if (ctid == 0) {
                mbar_expect_tx(&bar_w, (uint32_t)S::kImageBytes);
                const uint8_t *gsrc = reinterpret_cast<const uint8_t *>(wimg) + (int64_t)tl.field * img_bytes;
                for (int off = 0; off < S::kImageBytes; off += 16384) {
                    const int nb = S::kImageBytes - off < 16384 ? S::kImageBytes - off : 16384;
                    bulk_g2s(IMG + off, gsrc + off, (uint32_t)nb, &bar_w);
                }
                w_pending = true;
                w_pend_ph = wph;
            }
            ok = mbar_wait(&bar_w, wph, abortp, status);
            if (ctid == 0 && ok) w_pending = false;
            if (!publish(ok)) {
                aborted = true;
                break;
            }
            if (ctid == 0) {
                img_field = tl.field;
                n_img = n_img + 1u;
            }
        }
        progress(u_rel, 0);

        // ---- the sample ----
        const bool valid = (uint32_t)row < tl.count;
        const float4 dl = valid ? gsr[smp.idx] : make_float4(0.f, 0.f, 0.f, 0.f);
        // ---- this thread's 32 columns of X_0 = [F(x_loc) | 1] (its own
        // chunk: no wait); at W = 32 group 0 also packs the tail
        // [1 | F(d) | 0] that every X_i carries ----
        uint32_t tailp[16];
        {
            const float xl[3] = {fmaf(aff[0], smp.px, aff[3]), fmaf(aff[1], smp.py, aff[4]),
                                 fmaf(aff[2], smp.pz, aff[5])};
            uint8_t *x0 = xchunk(chain, 0);
            uint32_t p[8];
            if (g == 0) {
                enc_x0<0>(xl, p);
                st_units<2>(x0, row, 0, p);
                enc_x0<1>(xl, p);
                st_units<2>(x0, row, 2, p);
                if constexpr (W == 32) {
                    const float dv[3] = {smp.dx, smp.dy, smp.dz};
                    encode_packed<false, 4, 1, false, 32>(dv, tailp);
                }
            } else {
                enc_x0<2>(xl, p);
                st_units<2>(x0, row, 4, p);
                enc_x0<3>(xl, p);
                st_units<2>(x0, row, 6, p);
            }
        }
        // the tail of X_i at W = 32 (columns 32..63), by group 0
        auto store_tail = [&](int i) {
            if constexpr (W == 32)
                if (g == 0) st_units<4>(xchunk(chain, i), row, 4, tailp);
        };


        // ---- forward chain ----
        float s_logit = 0.f;
        float dsig = 0.f;
#pragma unroll 1
        for (int l = 0; l < kLayers; ++l) {
            ok = publish(ok);
            if (!ok) break;
            if (ctid == 0) {
                const uint32_t xa = xaddr(chain, l);
                const uint32_t ba = sIMG + (uint32_t)S::offset(l);
                if (l == 0) mma_fwd<S::K(0), W>(tD, xa, sT, ba);
                else if (l < H) mma_fwd<S::K_HID, W>(tD, xa, sT, ba);
                else if (l == H) mma_fwd<S::K_HID, S::N_HEAD>(tD, xa, sT, ba);
                else mma_fwd<S::K_COL, W>(tD, xa, sT, ba);
            }
            commit();
            if (l == 0) stage_index(pend, b, tl_next, row, more);
            if (l == kStageRec) stage_record(pend, src);
            if (l == kLayers - 1) {
                stage_ray(pend, src);
                if (more) load_aff(tl_next);
            }
            ok = land();
            // the chunk this epilogue writes held the other chain's X_{H+3-j}
            // (the colour layer also writes dZ and the tail's columns 64..127)
            const int j = l + 1;
            const uint32_t need = l == kLayers - 1 ? kFull : (uint32_t)(j > 2 ? j : 2);
            if (ok && u_rel > 0) ok = wait_prog(other, prog_word(u_rel - 1, need), abortp, status);
            if (l < H) {
                // next hidden input: ReLU
                uint8_t *xc = xchunk(chain, l + 1);
#pragma unroll
                for (int sb = 0; sb < NSB; ++sb) {
                    float va[16];
                    ldcf<16>(tDc + (uint32_t)(16 * sb), va);
                    uint32_t p[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) p[q] = pack_bf16_relu(va[2 * q], va[2 * q + 1]);
                    st_units<2>(xc, row, (c0 + 16 * sb) / 8, p);
                }
                store_tail(l + 1);
            } else if (l == H) {
                // head: features (linear) -> colour input, column W = density logit
                uint8_t *xc = xchunk(chain, H + 1);
                // (group 0 loads the logit with its last sub-block: one wait)
                uint32_t s_raw = 0u;
#pragma unroll
                for (int sb = 0; sb < NSB; ++sb) {
                    uint32_t r[16];
                    tmem_ld16_nowait(tDc + (uint32_t)(16 * sb), r);
                    if (g == 0 && sb == NSB - 1) s_raw = tmem_ld1_nowait(tD + tlane + (uint32_t)W);
                    tmem_wait_ld();
                    uint32_t p[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) p[q] = pack_bf16(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
                    st_units<2>(xc, row, (c0 + 16 * sb) / 8, p);
                }
                if (g == 0) s_logit = __uint_as_float(s_raw);
                store_tail(H + 1);
            }
            // this tile's F(d) in the shared tail, once the other chain's
            // colour wgrad no longer reads it (with X_2)
            if (W == 64 && l == 1 && g == 0) {
                const float dv[3] = {smp.dx, smp.dy, smp.dz};
                encode_packed<false, 4, 1, false, 32>(dv, tailp);
                st_units<4>(T, row, 0, tailp);
            }
            if (l == kLayers - 1) {
                // colour: z -> g = relu(z) (X_g), rgb = sigmoid(Wo g + bo) in FP32, then
                // the output layer's adjoint and dZ of the colour layer
                // the FP32 table's rows c over k: each float4 load is one
                // colour's weights for four k (the even and odd k summed apart
                // by packed FMAs, then together)
                const float *wo = reinterpret_cast<const float *>(IMG + S::kMatBytes);
                float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
#pragma unroll
                for (int sb = 0; sb < NSB; ++sb) {
                    float va[16];
                    ldcf<16>(tDc + (uint32_t)(16 * sb), va);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = c0 + 16 * sb + 4 * q;
                        const float2 g01 = make_float2(fmaxf(va[4 * q], 0.f), fmaxf(va[4 * q + 1], 0.f));
                        const float2 g23 = make_float2(fmaxf(va[4 * q + 2], 0.f), fmaxf(va[4 * q + 3], 0.f));
                        const float4 wx = *reinterpret_cast<const float4 *>(wo + k);
                        ax = __ffma2_rn(make_float2(wx.x, wx.y), g01, ax);
                        ax = __ffma2_rn(make_float2(wx.z, wx.w), g23, ax);
                        const float4 wy = *reinterpret_cast<const float4 *>(wo + W + k);
                        ay = __ffma2_rn(make_float2(wy.x, wy.y), g01, ay);
                        ay = __ffma2_rn(make_float2(wy.z, wy.w), g23, ay);
                        const float4 wz = *reinterpret_cast<const float4 *>(wo + 2 * W + k);
                        az = __ffma2_rn(make_float2(wz.x, wz.y), g01, az);
                        az = __ffma2_rn(make_float2(wz.z, wz.w), g23, az);
                    }
                }
                // the two column groups' partial sums of the row meet in
                // units 6 and 7 of the tail (no MMA reads those as anything
                // but ignored feature rows); both add them in group order
                *reinterpret_cast<float4 *>(T + sw_off(row, 6 + g)) =
                    make_float4(ax.x + ax.y, ay.x + ay.y, az.x + az.y, 0.f);
                asm volatile("bar.sync %0, %1;" ::"r"(3 + 4 * chain + quarter), "r"(64) : "memory");
                float4 acc = *reinterpret_cast<const float4 *>(wo + 4 * W);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float4 pp = *reinterpret_cast<const float4 *>(T + sw_off(row, 6 + q));
                    acc.x += pp.x;
                    acc.y += pp.y;
                    acc.z += pp.z;
                }
                const float r0 = sigmoid_f(acc.x), r1 = sigmoid_f(acc.y), r2 = sigmoid_f(acc.z);
                const float dz0 = dl.y * r0 * (1.f - r0), dz1 = dl.z * r1 * (1.f - r1), dz2 = dl.w * r2 * (1.f - r2);
                const float2 dz0p = make_float2(dz0, dz0), dz1p = make_float2(dz1, dz1), dz2p = make_float2(dz2, dz2);
                uint8_t *xg = xchunk(chain, H + 2);
#pragma unroll
                for (int sb = 0; sb < NSB; ++sb) {
                    float va[16];
                    ldcf<16>(tDc + (uint32_t)(16 * sb), va);     // re-read: cheaper than holding them
                    uint32_t pg[8], pd[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = c0 + 16 * sb + 4 * q;
                        const float4 wx = *reinterpret_cast<const float4 *>(wo + k);
                        const float4 wy = *reinterpret_cast<const float4 *>(wo + W + k);
                        const float4 wz = *reinterpret_cast<const float4 *>(wo + 2 * W + k);
                        // dL/dg_k = sum_c Wo[c][k] dz_c, for k and k + 1 at once
                        float2 d01 = __fmul2_rn(make_float2(wz.x, wz.y), dz2p);
                        d01 = __ffma2_rn(make_float2(wy.x, wy.y), dz1p, d01);
                        d01 = __ffma2_rn(make_float2(wx.x, wx.y), dz0p, d01);
                        float2 d23 = __fmul2_rn(make_float2(wz.z, wz.w), dz2p);
                        d23 = __ffma2_rn(make_float2(wy.z, wy.w), dz1p, d23);
                        d23 = __ffma2_rn(make_float2(wx.z, wx.w), dz0p, d23);
                        const float z0 = va[4 * q], z1 = va[4 * q + 1], z2 = va[4 * q + 2], z3 = va[4 * q + 3];
                        pg[2 * q] = pack_bf16_relu(z0, z1);
                        pg[2 * q + 1] = pack_bf16_relu(z2, z3);
                        pd[2 * q] = pack_bf16(z0 > 0.f ? d01.x : 0.f, z1 > 0.f ? d01.y : 0.f);
                        pd[2 * q + 1] = pack_bf16(z2 > 0.f ? d23.x : 0.f, z3 > 0.f ? d23.y : 0.f);
                    }
                    st_units<2>(xg, row, (c0 + 16 * sb) / 8, pg);
                    st_units<2>(DZ, row, (c0 + 16 * sb) / 8, pd);     // dZ of the colour layer
                }
                store_tail(H + 2);
                if (g == 0) {
                    dsig = dl.x * sig_scale * (act == ROAM_RELU ? (s_logit > 0.f ? 1.f : 0.f) : sigmoid_f(s_logit));
                    if constexpr (W == 32) {
                        uint32_t z4[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) z4[q] = 0u;
                        st_units<4>(DZ, row, 4, z4);
                    }
                    // dZ of the 3-output layer: units 4..5 of the tail
                    uint32_t po[8];
                    po[0] = pack_bf16(dz0, dz1);
                    po[1] = pack_bf16(dz2, 0.f);
#pragma unroll
                    for (int q = 2; q < 8; ++q) po[q] = 0u;
                    st_units<2>(T, row, 4, po);
                }
            }
        }


        // ---- backward chain ----
        // wgrad of layer l into its accumulator (N = its outputs); the dZ
        // operand's second 64-column block (the head's columns 64..79) sits
        // at byte 64 of the tail's rows
        auto issue_wgrad = [&](int l, uint32_t dza) {
            const uint32_t xa = xaddr(chain, l);
            const uint32_t td = tmem + (uint32_t)B::wcol(l);
            if (l == H + 2) mma_wgrad<16>(td, xa, sT - xa, dza, 1024u, 1u);
            else if (l == H) mma_wgrad<S::N_HEAD>(td, xa, sT - xa, dza, sT + 64u - dza, 1u);
            else mma_wgrad<W>(td, xa, sT - xa, dza, 1024u, 1u);
        };
        // dZ of the layer below from this thread's share of dX (its chain's
        // D), masked by that layer's ReLU (X_i > 0) when i > 0: packed into
        // registers while the group's wgrad MMAs still read dZ ...
        auto dz_of = [&](int i, bool relu, uint32_t (&p)[NSB][8]) {
            const uint8_t *xc = xchunk(chain, i);
#pragma unroll
            for (int sb = 0; sb < NSB; ++sb) {
                const int u0 = (c0 + 16 * sb) / 8;
                float va[16];
                ldcf<16>(tDc + (uint32_t)(16 * sb), va);
#pragma unroll
                for (int q = 0; q < 8; ++q) p[sb][q] = pack_bf16(va[2 * q], va[2 * q + 1]);
                if (relu) {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const uint4 m = *reinterpret_cast<const uint4 *>(xc + sw_off(row, u0 + u));
                        p[sb][4 * u] &= relu_mask(m.x);
                        p[sb][4 * u + 1] &= relu_mask(m.y);
                        p[sb][4 * u + 2] &= relu_mask(m.z);
                        p[sb][4 * u + 3] &= relu_mask(m.w);
                    }
                }
            }
        };
        // ... and stored once they have landed; at the head also the
        // density column (group 0)
        auto dz_store = [&](const uint32_t (&p)[NSB][8], bool head) {
#pragma unroll
            for (int sb = 0; sb < NSB; ++sb) st_units<2>(DZ, row, (c0 + 16 * sb) / 8, p[sb]);
            if (g == 0) {
                if constexpr (W == 64) {
                    if (head) {
                        uint32_t po[8];
                        po[0] = pack_bf16(dsig, 0.f);
#pragma unroll
                        for (int q = 1; q < 8; ++q) po[q] = 0u;
                        st_units<2>(T, row, 4, po);
                    }
                } else {
                    uint32_t z4[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) z4[q] = 0u;
                    if (head) z4[0] = pack_bf16(dsig, 0.f);
                    st_units<4>(DZ, row, 4, z4);
                }
            }
        };

        // output and colour layers (the barrier also agrees on the forward's last wait)
        bool ok2 = publish(ok);
        if (ok2) {
            // independent accumulators, so three warps issue them side by side
            if (ctid == 0) issue_wgrad(H + 2, sT + 64u);
            if (ctid == 32) issue_wgrad(H + 1, sDZ);
            if (ctid == 64) mma_dgrad<W, W>(tD, sDZ, sT + 64u, sIMG + (uint32_t)S::offset(H + 1));
            commit_split();
            ok2 = land();
            uint32_t p[NSB][8];
            dz_of(H + 1, false, p);               // dZ of the head: [d feat | d logit | 0]
            const bool gw = land_g();
            ok2 = ok2 && gw;
            if (ok2) progress(u_rel, 2);          // X_{H+2}, X_{H+1} and F(d) no longer read
            dz_store(p, true);
            ok2 = publish(ok2);
        }
        if (ok2) {
            // head
            if (ctid == 0) issue_wgrad(H, sDZ);
            if (ctid == 64) mma_dgrad<W, S::N_HEAD>(tD, sDZ, sT + 64u, sIMG + (uint32_t)S::offset(H));
            commit_split();
            ok2 = land();
            uint32_t p[NSB][8];
            dz_of(H, true, p);
            const bool gw = land_g();
            ok2 = ok2 && gw;
            dz_store(p, false);
            // hidden layers H-1 .. 1
#pragma unroll 1
            for (int l = H - 1; l >= 1; --l) {
                ok2 = publish(ok2);
                if (!ok2) break;
                progress(u_rel, (uint32_t)(H + 2 - l));   // X_{l+1}: its mask was read above
                if (ctid == 0) issue_wgrad(l, sDZ);
                if (ctid == 64) mma_dgrad<W, W>(tD, sDZ, sT + 64u, sIMG + (uint32_t)S::offset(l));
                commit_split();
                ok2 = land();
                dz_of(l, true, p);
                const bool gl = land_g();
                ok2 = ok2 && gl;
                dz_store(p, false);
            }
            ok2 = publish(ok2);
        }
        // every ok2 here is a barrier's verdict, the same for the whole chain
        if (!ok2) {
            aborted = true;
            break;
        }
        // first layer: wgrad only
        progress(u_rel, (uint32_t)(H + 2));               // X_1 free
        if (ctid == 0) issue_wgrad(0, sDZ);
        commit();
        good = land();                                    // agreed at the next tile's first barrier
        if (good) progress(u_rel, kFull);                 // X_0, dZ, the tail and every wgrad
        if (more) nxt = stage_finish(pend, src);
    }
    // both chains done: the last field's gradient, by every thread
    const bool any_abort = __syncthreads_or(aborted || *abortp) != 0;
    tc_fence_after();
    if (!any_abort && img_field != 0xffffffffu) flush(img_field, warp >> 2, 4);
    // drain before TMEM is freed: a commit whose wait gave up, an image load nobody waited for
    if (lead && d_open >= 0) mbar_wait(&bar_d[chain], (uint32_t)d_open, abortp, status, true);
    if (lead && g_open >= 0) mbar_wait(&bar_g[chain], (uint32_t)g_open, abortp, status, true);
    if (ctid == 0 && w_pending) mbar_wait(&bar_w, w_pend_ph, abortp, status, true);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int W, int H>
void launch_bt(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, const float4 *gsr,
               float *grad, int n_sm, cudaStream_t s)
{
    const int smem = 1024 + BwShape<W, H>::kSmem;
    static int smem_set[kMaxDevices] = {};
    raise_smem_limit((const void *)k_mlp_bwd_tc<W, H>, smem, smem_set);
    k_mlp_bwd_tc<W, H><<<n_sm, kBwThreads, smem, s>>>(w.wimg, w.img_bytes, w.affine, w.sigma_scale, w.act, w.P, src, b, ctr,
                                                gsr, grad);
}

#define ROAM_BWTC_CASES \
    ROAM_CASE(32, 1) ROAM_CASE(32, 2) ROAM_CASE(32, 3) ROAM_CASE(32, 4) ROAM_CASE(64, 1) ROAM_CASE(64, 2) ROAM_CASE(64, 3)

}  // namespace

bool mlp_bwd_tc_supported(int W, int H)
{
#define ROAM_CASE(WW, HH) \
    if (W == WW && H == HH) return 1024 + BwShape<WW, HH>::kSmem <= 227 * 1024;
    ROAM_BWTC_CASES
#undef ROAM_CASE
    return false;
}

void launch_mlp_bwd_tc(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr,
                       const float4 *gsr, float *grad, int n_sm, cudaStream_t s)
{
#define ROAM_CASE(WW, HH)                                              \
    if (w.W == WW && w.H == HH) {                                      \
        launch_bt<WW, HH>(w, src, b, ctr, gsr, grad, n_sm, s);         \
        return;                                                        \
    }
    ROAM_BWTC_CASES
#undef ROAM_CASE
}

}  // namespace roam
