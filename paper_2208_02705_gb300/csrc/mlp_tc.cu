// tcgen05 evaluation of the per-field tiny MLPs (the concurrent MLP queries
// of Sec. "Real-time Rendering Speedup" as a grouped GEMM chain on the
// 5th-generation tensor cores), with BF16 or FP8 E4M3 operands and FP32
// accumulation.  One tile = 128 samples of one field = one M=128 MMA row
// block; every layer of the chain is
//   D[128 x N] (TMEM, FP32) = A[128 x K] (TMEM) * B[K x N] (SMEM)
// with tcgen05.mma kind::f16 (BF16) or kind::f8f6f4 (E4M3).  The activations
// A never touch shared memory: the epilogue reads D with tcgen05.ld (one row
// per thread), converts and writes the next layer's A with tcgen05.st, so
// the MMA streams only the weights from shared memory.  The field's weight
// image (all layers' B operands in the 128-byte-swizzled K-major layout,
// then FP32 tables) is copied to shared memory by the bulk-copy (TMA) engine
// when the field changes.
//
// A columns (row = sample):
//   L1 input        [F(x_loc) (63) | 1]                          K = 64
//   after L1        [h (W) | 1 | F(d) (27) | 0 0 0 0]             (the tail stays)
//   hidden / head   [h (W) | 1 | ...]                            K = W + 16 or W
//   colour          [feat (W) | 1 | F(d) (27) | 0 0 0 0]          K = W + 32
//
// Biases.  BF16 at W <= 64 folds every bias into the MMA: the constant-1
// column of A meets the bias row of B.  BF16 at W = 128 folds only the L1
// and colour biases (their K has the spare column anyway): a folded bias in
// the hidden and head layers would cost a third 64-column K-chunk per layer
// and the image would not fit in shared memory.  E4M3 folds none (a bias
// rounded to 3 mantissa bits loses too much).  Unfolded biases are added in
// FP32 by the epilogue from a per-layer table at the end of the image.
//
// E4M3 weights carry one FP32 scale per output channel (row n of layer l):
// s = max_k |W[n][k]| / 448, B[k][n] = e4m3(W[n][k] / s), and the epilogue
// forms y = s * D + b.  Activations are rounded to E4M3 unscaled (the
// ReLU/PE values of these networks sit well inside the format's range).
#include "tc_common.cuh"

namespace roam {

namespace {

__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return r;
}

// 32 (BF16: 16 words, two x8 stores; E4M3: 8 words, one x8 store) ... of A
template <bool F8>
__device__ __forceinline__ void st_words32(uint32_t tArow, int c, const uint32_t *w)
{
    if constexpr (F8) {
        uint32_t o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = w[q];
        tmem_st8(tArow + 8 * c, o);
    } else {
        uint32_t o[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) o[q] = w[q];
        tmem_st16(tArow + 16 * c, o);
    }
}

// Persistent kernel, one CTA per SM, kSlots tiles in flight.  Slot s is
// warpgroup s: its 128 threads encode and run the epilogues of their tile
// (one row each), and its first thread issues the tile's MMAs itself --
// tcgen05.mma and tcgen05.commit occupy the issuing thread for tens to
// hundreds of cycles each, so one issuer per slot lets the slots' chains
// overlap.  Tiles come in field-uniform groups of kSlots (bucket padding);
// at a field change all slots meet at a CTA barrier, thread 0 reloads the
// shared weight image, and each issuer waits for it before its next MMA.
template <int W, int H, bool F8>
__global__ void __launch_bounds__(TcShape<W, H, F8>::kSlots * 128, 1)
    k_mlp_tc(const void *wimg, int64_t img_bytes, int field_base, int cls, const float *affine, float sig_scale,
             int act, SampleSrc src, BucketBufs b, Counters *ctr, float4 *out, unsigned long long wait_ns,
             int withhold_image)
{
    using S = TcShape<W, H, F8>;
    constexpr int kSlots = S::kSlots;
    constexpr int kLayers = S::kLayers;
    constexpr int kStageRec = kLayers >= 4 ? 1 : 0;  // the layer after which the next tile's records are gathered
    constexpr int kCols = S::kSlotCols;
    constexpr int kTmemAlloc = kSlots * kCols <= 32 ? 32 : (kSlots * kCols <= 64 ? 64 :
                               (kSlots * kCols <= 128 ? 128 : (kSlots * kCols <= 256 ? 256 : 512)));
    static_assert(kSlots * kCols <= 512, "TMEM holds every slot's accumulator and activations");
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_d[kSlots];
    __shared__ uint64_t bar_w;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t *IMG = smem_raw + (base - smem_u32(smem_raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = warp >> 2, wq = warp & 3;
    const int row = wq * 32 + lane;                           // TMEM lane == tile row
    // the slot's issuing thread sits in the slot's warp with index = slot mod 4,
    // so the slots' issuers run on different SM sub-partitions
    const bool issuer = wq == (slot & 3) && lane == 0;
    volatile int *abortp = &abort_flag;
    uint32_t *status = &ctr->status;

    if (threadIdx.x == 0) {
        for (int q = 0; q < kSlots; ++q) mbar_init(&bar_d[q], 1);
        mbar_init(&bar_w, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemAlloc)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tslot = tmem + (uint32_t)(slot * kCols);        // accumulator D
    const uint32_t tA = tslot + (uint32_t)S::kDCols;                  // activations A
    const uint32_t trow = tslot + ((uint32_t)(wq * 32) << 16);
    const uint32_t tArow = tA + ((uint32_t)(wq * 32) << 16);
    const uint32_t imga = smem_u32(IMG);
    const float *tab = reinterpret_cast<const float *>(IMG + S::kMatBytes + S::kOutBytes);

    // this width class's tiles (a multiple of kSlots apart: bucket padding)
    const Tile *tiles = b.tiles + ctr->class_tiles[cls];
    const uint32_t n_groups = (ctr->class_tiles[cls + 1] - ctr->class_tiles[cls]) / kSlots;
    const uint32_t g0 = (uint32_t)((uint64_t)n_groups * blockIdx.x / gridDim.x);
    const uint32_t g1 = (uint32_t)((uint64_t)n_groups * (blockIdx.x + 1) / gridDim.x);

    uint32_t d_ph = 0, n_changes = 0, n_commits = 0, n_waits = 0;
    uint32_t cur_field = 0xffffffffu;
    bool w_ready = false, w_waited_last = true;
    bool img_seen = false;     // this thread has waited for the current image (before generic loads of it)
    bool aborted = false;
    Tile tl{0u, 0u, 0u, 0u};
    SampleIn nxt{0u, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    Pending pend{};
    uint32_t g = g0;
    if (g < g1) {
        tl = tiles[g * kSlots + slot];
        nxt = fetch_sample(src, b, tl, row);
    }
    for (; g < g1; ++g) {
        const uint32_t f = tl.field;           // identical for every slot (field-uniform groups)
        if (f != cur_field) {
            // A load whose groups held only empty tiles was never waited for:
            // thread 0 retires it BEFORE the barrier.  After the barrier any
            // thread may wait for the next phase of bar_w by its parity, and
            // a parity wait passes at once while the phase before it is still
            // pending -- a slot would then read the image while it lands.
            if (threadIdx.x == 0 && !w_waited_last) {
                w_waited_last = mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status, true, wait_ns);
                if (!w_waited_last) *abortp = 1;   // the old load never landed: give up (status flagged)
            }
            // generic reads of the old image (the FP32 tables) come before the
            // bulk copy that overwrites it
            fence_async_smem();
            // every slot has waited on its last layer, so no MMA reads the old
            // image; meet (and agree on any abort), reload, issuers wait below
            if (named_sync_or(15, kSlots * 128, aborted || *abortp)) break;
            if (threadIdx.x == 0 && !withhold_image) {
                // each phase of bar_w carries exactly one arrival and one image
                mbar_expect_tx(&bar_w, (uint32_t)S::kImageBytes);
                const uint8_t *gsrc = reinterpret_cast<const uint8_t *>(wimg) + (int64_t)(f - field_base) * img_bytes;
                for (int off = 0; off < S::kImageBytes; off += 16384) {
                    const int nb = S::kImageBytes - off < 16384 ? S::kImageBytes - off : 16384;
                    bulk_g2s(IMG + off, gsrc + off, (uint32_t)nb, &bar_w);
                }
                w_waited_last = false;
            }
            // (withheld, in the self-test: no copy and no arrival, so every
            // wait on this phase runs out; nothing is in flight to drain)
            ++n_changes;
            cur_field = f;
            w_ready = false;
            img_seen = false;
        }
        const Tile cur = tl;
        const SampleIn sm = nxt;
        if (g + 1 < g1) tl = tiles[(g + 1) * kSlots + slot];
        if (cur.count == 0 || aborted) {
            if (g + 1 < g1) nxt = fetch_sample(src, b, tl, row);
            continue;
        }
        const bool valid = (uint32_t)row < cur.count;
        const float *aff = affine + 6 * (int64_t)cur.field;
        // ---- L1 input: [F(x_loc) | 1] ----
        {
            const float xl[3] = {fmaf(__ldg(aff + 0), sm.px, __ldg(aff + 3)), fmaf(__ldg(aff + 1), sm.py, __ldg(aff + 4)),
                                 fmaf(__ldg(aff + 2), sm.pz, __ldg(aff + 5))};
            // rows past the tile's count compute garbage that is never stored
            uint32_t w[F8 ? 16 : 32];
            encode_packed<F8, 10, 0, true, 64>(xl, w);
            st_words32<F8>(tArow, 0, w);
            st_words32<F8>(tArow, 1, w + (F8 ? 8 : 16));
        }
        // the next tile's gathers overlap this tile's layers
        stage_index(pend, b, tl, row, g + 1 < g1);
        float sigma = 0.f;
#pragma unroll 1
        for (int l = 0; l < kLayers; ++l) {
            // A for layer l is complete once all 128 threads of the slot arrive
            tmem_wait_st();
            tc_fence_before();
            if (named_sync_or(1 + slot, 128, aborted || *abortp)) {
                aborted = true;
                break;
            }
            if (issuer) {
                bool ok = true;
                if (!w_ready) {
                    ok = mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status, false, wait_ns);
                    w_ready = ok;
                    if (threadIdx.x == 0) w_waited_last = ok;
                }
                if (ok) {
                    tc_fence_after();
                    const uint32_t ba = imga + S::offset(l);
                    // one MMA per 32 bytes of K: 4 per 128-byte chunk, 8 TMEM columns of A each
                    if (l == 0) umma_chain_ta<F8, S::K(0), W>(tslot, tA, ba);
                    else if (l < H) umma_chain_ta<F8, S::K_HID, W>(tslot, tA, ba);
                    else if (l == H) umma_chain_ta<F8, S::K_HID, S::N_HEAD>(tslot, tA, ba);
                    else umma_chain_ta<F8, S::K_COL, W>(tslot, tA, ba);
                }
                umma_commit(&bar_d[slot]);
                ++n_commits;
            }
            // the tail of A from here on, [1 | F(d) | 0 0 0 0] at elements
            // W .. W+31: at W >= 64 in L1's shadow (L1, K = 64, does not read
            // those elements), at W = 32 (they are L1's input) after L1 landed
            auto store_tail = [&]() {
                const float dv[3] = {sm.dx, sm.dy, sm.dz};
                uint32_t w[F8 ? 8 : 16];
                encode_packed<F8, 4, 1, false, 32>(dv, w);
                st_words32<F8>(tArow, W / 32, w);
            };
            if (W >= 64 && l == 0) store_tail();
            const bool got = mbar_wait(&bar_d[slot], d_ph, abortp, status, false, wait_ns);
            if (issuer && got) ++n_waits;
            d_ph ^= 1u;
            // tcgen05.ld is warp-collective: the warp decides together; the
            // slot decides together at the next barrier
            if (!__all_sync(0xffffffffu, got)) {
                aborted = true;
                continue;
            }
            tc_fence_after();
            // the FP32 per-layer table, where this layer's epilogue uses it
            const bool use_tab = S::kTab && (F8 || (l >= 1 && l <= H));
            const float *tsc = tab + l * 2 * S::kTabStride, *tbi = tsc + S::kTabStride;
            if ((use_tab || l == H + 1) && !img_seen) {
                mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status, false, wait_ns);
                img_seen = true;
            }
            if (l < H + 1) {
                if constexpr (W == 64 && !S::kTab) {
                    // both 32-column halves in flight before one wait
                    uint32_t ra[32], rb[32];
                    tmem_ld32_nowait(trow, ra);
                    tmem_ld32_nowait(trow + 32, rb);
                    tmem_wait_ld();
                    float v[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(ra[q]);
                    if (l == H) st_act32<F8, false>(tArow, 0, v);
                    else st_act32<F8, true>(tArow, 0, v);
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(rb[q]);
                    if (l == H) st_act32<F8, false>(tArow, 1, v);
                    else st_act32<F8, true>(tArow, 1, v);
                } else {
                // next activations, 32 columns at a time (few live registers):
                // head features stay linear, every other layer ReLU
#pragma unroll
                for (int c = 0; c < W / 32; ++c) {
                    uint32_t r32[32];
                    tmem_ld32_nowait(trow + 32 * c, r32);
                    tmem_wait_ld();
                    float v[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r32[q]);
                    if constexpr (S::kTab) {
                        if (use_tab) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 bb = reinterpret_cast<const float4 *>(tbi + 32 * c)[q];
                                if constexpr (F8) {
                                    // y = s D + b as packed pairs (each half rounded as fmaf)
                                    const float4 ss = reinterpret_cast<const float4 *>(tsc + 32 * c)[q];
                                    const float2 v01 = __ffma2_rn(make_float2(v[4 * q], v[4 * q + 1]),
                                                                  make_float2(ss.x, ss.y), make_float2(bb.x, bb.y));
                                    const float2 v23 = __ffma2_rn(make_float2(v[4 * q + 2], v[4 * q + 3]),
                                                                  make_float2(ss.z, ss.w), make_float2(bb.z, bb.w));
                                    v[4 * q] = v01.x; v[4 * q + 1] = v01.y; v[4 * q + 2] = v23.x; v[4 * q + 3] = v23.y;
                                } else {
                                    v[4 * q] += bb.x; v[4 * q + 1] += bb.y; v[4 * q + 2] += bb.z; v[4 * q + 3] += bb.w;
                                }
                            }
                        }
                    }
                    if (l == H) st_act32<F8, false>(tArow, c, v);
                    else st_act32<F8, true>(tArow, c, v);
                }
                }
                if (W < 64 && l == 0) store_tail();
                if (l == H) {
                    // density from column W of the head
                    float sl = __uint_as_float(tmem_ld1(trow + W));
                    tmem_wait_ld();
                    if (use_tab) sl = F8 ? fmaf(sl, tsc[W], tbi[W]) : sl + tbi[W];
                    sigma = sig_scale * (act == ROAM_RELU ? fmaxf(sl, 0.f) : softplus_f(sl));
                }
            } else {
                // colour layer: g = relu(z) in FP32, then rgb = sigmoid(Wo g + bo) with
                // the FP32 output table at the end of the shared image (this thread
                // has waited for the image itself before reading it with generic loads)
                // table rows c over k: each float4 load gives one colour's weights
                // for four k, two pairs for the packed FMAs (the even and odd k
                // summed apart, then together with the bias)
                const float *wo = reinterpret_cast<const float *>(IMG + S::kMatBytes);
                float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
                // chunk c + 1's TMEM load in flight during chunk c's FMAs
                uint32_t ra[16], rb[16];
                tmem_ld16_nowait(trow, ra);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < W / 16; ++c) {
                    uint32_t(&r)[16] = (c & 1) ? rb : ra;
                    uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
                    if (c + 1 < W / 16) tmem_ld16_nowait(trow + 16 * (c + 1), nxt);
                    float gk[16];
                    if constexpr (F8) {
                        // y = s z + b per channel, packed pairs (each half rounded as fmaf)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 ss = reinterpret_cast<const float4 *>(tsc + 16 * c)[q];
                            const float4 bb = reinterpret_cast<const float4 *>(tbi + 16 * c)[q];
                            const float2 y01 = __ffma2_rn(make_float2(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1])),
                                                          make_float2(ss.x, ss.y), make_float2(bb.x, bb.y));
                            const float2 y23 = __ffma2_rn(make_float2(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3])),
                                                          make_float2(ss.z, ss.w), make_float2(bb.z, bb.w));
                            gk[4 * q] = fmaxf(y01.x, 0.f); gk[4 * q + 1] = fmaxf(y01.y, 0.f);
                            gk[4 * q + 2] = fmaxf(y23.x, 0.f); gk[4 * q + 3] = fmaxf(y23.y, 0.f);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) gk[q] = fmaxf(__uint_as_float(r[q]), 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = 16 * c + 4 * q;
                        const float2 g01 = make_float2(gk[4 * q], gk[4 * q + 1]);
                        const float2 g23 = make_float2(gk[4 * q + 2], gk[4 * q + 3]);
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
                    if (c + 1 < W / 16) tmem_wait_ld();
                }
                const float4 bo = *reinterpret_cast<const float4 *>(wo + 4 * W);
                const float4 acc = make_float4(bo.x + (ax.x + ax.y), bo.y + (ay.x + ay.y), bo.z + (az.x + az.y), 0.f);
                if (valid) out[sm.idx] = make_float4(sigma, sigmoid_f(acc.x), sigmoid_f(acc.y), sigmoid_f(acc.z));
            }
            tc_fence_before();
            // each gather stage a layer or more after the load it depends on
            if (l == kStageRec) stage_record(pend, src);
            if (l == kLayers - 2) stage_ray(pend, src);
        }
        if (!aborted) nxt = stage_finish(pend, src);
    }
    // drain before TMEM is freed and the CTA exits: a commit whose wait gave
    // up, and an image load nobody waited for
    if (issuer && n_commits > n_waits) mbar_wait(&bar_d[slot], (n_commits - 1) & 1u, abortp, status, true, wait_ns);
    if (threadIdx.x == 0 && !w_waited_last) mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status, true, wait_ns);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemAlloc)
                     : "memory");
    }
}

// ---- packing: API layout -> tensor-core image ----

// offsets of one field's layers in the API layout (row-major [out][in], then bias[out])
struct ApiLayout {
    int64_t l1, hid, head, col, out;
    __host__ __device__ ApiLayout(int W, int H)
    {
        l1 = 0;
        hid = (int64_t)W * kPeX + W;
        head = hid + (int64_t)(H - 1) * (W * W + W);
        col = head + (int64_t)(1 + W) * W + (1 + W);
        out = col + (int64_t)W * (W + kPeD) + W;
    }
};

// Weight at (n, k) of the B operand of layer l, as the MMA sees it (folded
// bias entries included where the layout folds them).
template <int W, int H, bool F8>
__device__ float operand_value(const float *wf, const ApiLayout &o, int l, int n, int k)
{
    using S = TcShape<W, H, F8>;
    if (k >= S::K(l)) return 0.f;
    if (l == 0) {
        if (n >= W) return 0.f;
        if (k < kPeX) return wf[o.l1 + (int64_t)n * kPeX + k];
        return (k == kPeX && !F8) ? wf[o.l1 + (int64_t)W * kPeX + n] : 0.f;
    }
    if (l < H) {
        const int64_t ob = o.hid + (int64_t)(l - 1) * (W * W + W);
        if (k < W) return wf[ob + (int64_t)n * W + k];
        return (k == W && S::kFold) ? wf[ob + (int64_t)W * W + n] : 0.f;
    }
    if (l == H) {
        // rows: W features (API rows 1..W), then the density logit (API row 0)
        const int ar = n < W ? 1 + n : (n == W ? 0 : -1);
        if (ar < 0) return 0.f;
        if (k < W) return wf[o.head + (int64_t)ar * W + k];
        return (k == W && S::kFold) ? wf[o.head + (int64_t)(1 + W) * W + ar] : 0.f;
    }
    const int kc = W + kPeD;
    if (k < W) return wf[o.col + (int64_t)n * kc + k];
    if (k == W) return F8 ? 0.f : wf[o.col + (int64_t)W * kc + n];
    if (k <= W + kPeD) return wf[o.col + (int64_t)n * kc + (k - 1)];
    return 0.f;
}

// bias of output n of layer l (the head's n = W is the density logit)
template <int W, int H>
__device__ float layer_bias(const float *wf, const ApiLayout &o, int l, int n)
{
    if (l == 0) return n < W ? wf[o.l1 + (int64_t)W * kPeX + n] : 0.f;
    if (l < H) return n < W ? wf[o.hid + (int64_t)(l - 1) * (W * W + W) + (int64_t)W * W + n] : 0.f;
    if (l == H)
        return n < W ? wf[o.head + (int64_t)(1 + W) * W + 1 + n] : (n == W ? wf[o.head + (int64_t)(1 + W) * W] : 0.f);
    return n < W ? wf[o.col + (int64_t)W * (W + kPeD) + n] : 0.f;
}

// per-layer FP32 table: E4M3 channel scales (max |row| / 448, 1 for an
// all-zero row; 1 for BF16) and the biases
template <int W, int H, bool F8>
__global__ void k_pack_tab(const float *__restrict__ w32, int n_fields, int64_t P, uint8_t *__restrict__ img,
                           int64_t img_bytes)
{
    using S = TcShape<W, H, F8>;
    const ApiLayout o(W, H);
    const int64_t per = (int64_t)S::kLayers * S::kTabStride;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)n_fields * per;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = g / per;
        const int l = (int)((g % per) / S::kTabStride), n = (int)(g % S::kTabStride);
        const float *wf = w32 + f * P;
        float s = 1.f;
        if (F8 && n < S::N(l)) {
            float amax = 0.f;
            for (int k = 0; k < S::K(l); ++k) amax = fmaxf(amax, fabsf(operand_value<W, H, F8>(wf, o, l, n, k)));
            if (amax > 0.f) s = amax / 448.0f;
        }
        float *t = reinterpret_cast<float *>(img + f * img_bytes + S::kMatBytes + S::kOutBytes) + l * 2 * S::kTabStride;
        t[n] = s;
        t[S::kTabStride + n] = layer_bias<W, H>(wf, o, l, n);
    }
}

template <int W, int H, bool F8>
__global__ void k_pack_tc(const float *__restrict__ w32, int n_fields, int64_t P, uint8_t *__restrict__ img,
                          int64_t img_bytes)
{
    using S = TcShape<W, H, F8>;
    const ApiLayout o(W, H);
    const int64_t per = S::kMatBytes / S::kEB;        // operand elements per field
    const int64_t n = (int64_t)n_fields * per;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = g / per;
        const int byte = (int)((g % per) * S::kEB);
        // find the layer and (n, k) of this element
        int l = 0;
        while (l + 1 < S::kLayers && byte >= S::offset(l + 1)) ++l;
        const int lb = byte - S::offset(l);
        const int N = S::N(l);
        const int chunk = lb / (N * 128);
        const int in_chunk = lb % (N * 128);
        const int nrow = (in_chunk / 1024) * 8 + (in_chunk % 1024) / 128;
        const int sw16 = (in_chunk % 128) / 16;
        const int u = (sw16 ^ (nrow & 7)) & 7;               // 16-byte unit before the swizzle
        const int k = chunk * S::kCE + u * (16 / S::kEB) + (in_chunk % 16) / S::kEB;
        const float *wf = w32 + f * P;
        const float v = operand_value<W, H, F8>(wf, o, l, nrow, k);
        uint8_t *dst = img + f * img_bytes;
        if constexpr (F8) {
            const float s =
                reinterpret_cast<const float *>(dst + S::kMatBytes + S::kOutBytes)[l * 2 * S::kTabStride + nrow];
            uint16_t q;
            asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(q) : "f"(v / s), "f"(0.f));
            dst[g % per] = (uint8_t)(q & 0xffu);
        } else {
            const uint32_t bits = __float_as_uint(v);
            const uint32_t r = bits + 0x7fffu + ((bits >> 16) & 1u);     // round to nearest even
            reinterpret_cast<uint16_t *>(dst)[g % per] = (uint16_t)(r >> 16);
        }
    }
    // FP32 output layer after the operands: [4][W] (weights of the 3 colours over k, a zero row), then bias[4]
    const int nout = 4 * W + 4;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < (int64_t)n_fields * nout;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = gi / nout;
        const int q = (int)(gi % nout);
        const float *wf = w32 + f * P;
        float v = 0.f;
        if (q < 4 * W) {
            const int c = q / W, k = q % W;
            if (c < 3) v = wf[o.out + (int64_t)c * W + k];
        } else if (q - 4 * W < 3) {
            v = wf[o.out + 3 * W + (q - 4 * W)];
        }
        reinterpret_cast<float *>(img + f * img_bytes + S::kMatBytes)[q] = v;
    }
}

// Where parameter q of a field (API layout) sits in its BF16 image: the byte
// offset of its element, or -1 - r for entry r of the FP32 3-output table.
template <int W, int H>
__device__ __forceinline__ int image_slot(const ApiLayout &o, int64_t q)
{
    using S = TcShape<W, H, false>;
    int l, nr, k;
    if (q < o.hid) {
        const int r = (int)(q - o.l1);
        l = 0;
        if (r < W * kPeX) { nr = r / kPeX; k = r % kPeX; }
        else { nr = r - W * kPeX; k = kPeX; }
    } else if (q < o.head) {
        const int64_t r0 = q - o.hid;
        l = 1 + (int)(r0 / (W * W + W));
        const int r = (int)(r0 % (W * W + W));
        if (r < W * W) { nr = r / W; k = r % W; }
        else { nr = r - W * W; k = W; }
    } else if (q < o.col) {
        const int r = (int)(q - o.head);
        int ar;
        l = H;
        if (r < (1 + W) * W) { ar = r / W; k = r % W; }
        else { ar = r - (1 + W) * W; k = W; }
        nr = ar == 0 ? W : ar - 1;          // image rows: W features, then the density logit
    } else if (q < o.out) {
        const int r = (int)(q - o.col), kc = W + kPeD;
        l = H + 1;
        if (r < W * kc) { nr = r / kc; const int ka = r % kc; k = ka < W ? ka : ka + 1; }
        else { nr = r - W * kc; k = W; }
    } else {
        // the FP32 3-output layer: [4][W] (its API rows c, then a zero row) then bias[4]
        const int r = (int)(q - o.out);
        return -1 - (r < 3 * W ? r : 4 * W + (r - 3 * W));
    }
    const int N = S::N(l);
    return S::offset(l) + (k / S::kCE) * N * 128 + (nr >> 3) * 1024 + (nr & 7) * 128 +
           ((((k % S::kCE) >> 3) ^ (nr & 7)) << 4) + (k & 7) * 2;
}

// Adam on the FP32 masters fused with the refresh of the BF16 image (every
// bias folded into the MMA: W <= 64): one thread per four parameters (vector
// loads and stores of the masters, moments and gradient), each written into
// its image element (or its FP32 output-table entry).  The step is
// w -= (lr / bc1) m / (sqrt(v / bc2) + eps) with one correctly rounded
// reciprocal (within a few units of 2^-24 of the two divisions).
template <int W, int H>
__global__ void k_adam_tc(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                          const float *__restrict__ g, int n_fields, int64_t P, uint8_t *__restrict__ img,
                          int64_t img_bytes, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    using S = TcShape<W, H, false>;
    static_assert(S::kFold, "fused refresh needs every bias in the image's MMA operands");
    const ApiLayout o(W, H);
    const int64_t f = blockIdx.y;                      // one grid row per field: no 64-bit division
    if (f >= n_fields) return;
    const float lr_t = lr / bc1, inv_bc2 = 1.f / bc2;
    uint8_t *dst = img + f * img_bytes;
    auto update = [&](int64_t q, float gi, float &mi, float &vi, float &wi) {
        mi = fmaf(b1, mi, (1.f - b1) * gi);
        vi = fmaf(b2, vi, (1.f - b2) * gi * gi);
        wi = wi - lr_t * mi * __frcp_rn(sqrtf(vi * inv_bc2) + eps);
        const int at = image_slot<W, H>(o, q);
        if (at < 0) {
            reinterpret_cast<float *>(dst + S::kMatBytes)[-1 - at] = wi;
        } else {
            const uint32_t bits = __float_as_uint(wi);
            *reinterpret_cast<uint16_t *>(dst + at) = (uint16_t)((bits + 0x7fffu + ((bits >> 16) & 1u)) >> 16);
        }
    };
    const int64_t q0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (q0 >= P) return;
    const int64_t i0 = f * P + q0;
    if (q0 + 4 <= P && (i0 & 3) == 0) {
        float4 g4 = *reinterpret_cast<const float4 *>(g + i0);
        float4 m4 = *reinterpret_cast<const float4 *>(m + i0);
        float4 v4 = *reinterpret_cast<const float4 *>(v + i0);
        float4 w4 = *reinterpret_cast<const float4 *>(w + i0);
        update(q0, g4.x, m4.x, v4.x, w4.x);
        update(q0 + 1, g4.y, m4.y, v4.y, w4.y);
        update(q0 + 2, g4.z, m4.z, v4.z, w4.z);
        update(q0 + 3, g4.w, m4.w, v4.w, w4.w);
        *reinterpret_cast<float4 *>(m + i0) = m4;
        *reinterpret_cast<float4 *>(v + i0) = v4;
        *reinterpret_cast<float4 *>(w + i0) = w4;
    } else {
        for (int64_t q = q0; q < q0 + 4 && q < P; ++q) {
            const int64_t i = f * P + q;
            float mi = m[i], vi = v[i], wi = w[i];
            update(q, g[i], mi, vi, wi);
            m[i] = mi;
            v[i] = vi;
            w[i] = wi;
        }
    }
}

template <int W, int H, bool F8>
int tc_smem_bytes() { return 1024 + TcShape<W, H, F8>::kImageAlloc; }

template <int W, int H, bool F8>
void launch_t(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, float4 *out, int n_sm,
              cudaStream_t s)
{
    constexpr int kSlots = TcShape<W, H, F8>::kSlots;
    const int smem = tc_smem_bytes<W, H, F8>();
    static int smem_set[kMaxDevices] = {};
    raise_smem_limit((const void *)k_mlp_tc<W, H, F8>, smem, smem_set);
    const void *img = F8 ? w.wimg8 : w.wimg;
    const int64_t ib = F8 ? w.img8_bytes : w.img_bytes;
    k_mlp_tc<W, H, F8><<<n_sm, kSlots * 128, smem, s>>>(img, ib, w.field_base, w.cls, w.affine, w.sigma_scale, w.act,
                                                        src, b, ctr, out, w.wait_ns ? w.wait_ns : kWaitNs,
                                                        w.withhold_image);
}

#define ROAM_TC_CASES                                                                                   \
    ROAM_CASE(32, 1) ROAM_CASE(32, 2) ROAM_CASE(32, 3) ROAM_CASE(32, 4) ROAM_CASE(64, 1) ROAM_CASE(64, 2) \
    ROAM_CASE(64, 3) ROAM_CASE(64, 4) ROAM_CASE(128, 1) ROAM_CASE(128, 2) ROAM_CASE(128, 3) ROAM_CASE(128, 4)

}  // namespace

bool tc_supported(int W, int H, bool f8)
{
    if (H < 1 || H > 4) return false;
#define ROAM_CASE(WW, HH) \
    if (W == WW && H == HH) return (f8 ? tc_smem_bytes<WW, HH, true>() : tc_smem_bytes<WW, HH, false>()) <= 227 * 1024;
    ROAM_TC_CASES
#undef ROAM_CASE
    return false;
}

int64_t tc_image_bytes(int W, int H, bool f8)
{
#define ROAM_CASE(WW, HH) \
    if (W == WW && H == HH) return f8 ? TcShape<WW, HH, true>::kImageBytes : TcShape<WW, HH, false>::kImageBytes;
    ROAM_TC_CASES
#undef ROAM_CASE
    return 0;
}

int tc_tile_samples() { return 128; }

int tc_tile_group(int W, bool f8)
{
    if (W <= 32) return f8 ? TcShape<32, 1, true>::kSlots : TcShape<32, 1, false>::kSlots;
    if (W <= 64) return f8 ? TcShape<64, 1, true>::kSlots : TcShape<64, 1, false>::kSlots;
    return f8 ? TcShape<128, 1, true>::kSlots : TcShape<128, 1, false>::kSlots;
}

void launch_pack_tc(const float *w32, int n_fields, int W, int H, int64_t P, void *wimg, int64_t img_bytes, bool f8,
                    cudaStream_t s)
{
#define ROAM_CASE(WW, HH)                                                                                      \
    if (W == WW && H == HH) {                                                                                  \
        if (f8) {                                                                                              \
            k_pack_tab<WW, HH, true><<<1024, 256, 0, s>>>(w32, n_fields, P, (uint8_t *)wimg, img_bytes);      \
            k_pack_tc<WW, HH, true><<<2048, 256, 0, s>>>(w32, n_fields, P, (uint8_t *)wimg, img_bytes);       \
        } else {                                                                                               \
            if (TcShape<WW, HH, false>::kTab)                                                                  \
                k_pack_tab<WW, HH, false><<<1024, 256, 0, s>>>(w32, n_fields, P, (uint8_t *)wimg, img_bytes); \
            k_pack_tc<WW, HH, false><<<2048, 256, 0, s>>>(w32, n_fields, P, (uint8_t *)wimg, img_bytes);      \
        }                                                                                                      \
        return;                                                                                                \
    }
    ROAM_TC_CASES
#undef ROAM_CASE
}

bool launch_adam_tc(float *w32, float *m, float *v, const float *g, int n_fields, int W, int H, int64_t P, void *wimg,
                    int64_t img_bytes, float lr, float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s)
{
    if (n_fields > 65535) return false;           // one grid row per field
#define ROAM_ADAM_CASE(WW, HH)                                                                                   \
    if (W == WW && H == HH) {                                                                                  \
        const dim3 grid((unsigned)((P + 1023) / 1024), (unsigned)n_fields);                                     \
        k_adam_tc<WW, HH><<<grid, 256, 0, s>>>(w32, m, v, g, n_fields, P, (uint8_t *)wimg, img_bytes, lr, b1, b2, \
                                               eps, bc1, bc2);                                                 \
        return true;                                                                                           \
    }
    ROAM_ADAM_CASE(32, 1) ROAM_ADAM_CASE(32, 2) ROAM_ADAM_CASE(32, 3) ROAM_ADAM_CASE(32, 4)
    ROAM_ADAM_CASE(64, 1) ROAM_ADAM_CASE(64, 2) ROAM_ADAM_CASE(64, 3) ROAM_ADAM_CASE(64, 4)
#undef ROAM_ADAM_CASE
    return false;
}

void launch_mlp_tc(const MlpWeights &w, bool f8, const SampleSrc &src, const BucketBufs &b, Counters *ctr,
                   float4 *out, int n_sm, cudaStream_t s)
{
#define ROAM_CASE(WW, HH)                                             \
    if (w.W == WW && w.H == HH) {                                     \
        if (f8) launch_t<WW, HH, true>(w, src, b, ctr, out, n_sm, s); \
        else launch_t<WW, HH, false>(w, src, b, ctr, out, n_sm, s);   \
        return;                                                       \
    }
    ROAM_TC_CASES
#undef ROAM_CASE
}

}  // namespace roam
