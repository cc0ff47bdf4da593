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
//      issue them side by side; every warp's lane 0 commits to the group's
//      barrier.
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
// Shared memory (W = 64): the image, X_0 (encoding), X_1..X_H (hidden
// inputs), X_{H+1} (colour input), X_g (colour output), each one 64-column
// chunk; a tail chunk T = [1 | F(d) | 0] that continues every row past
// column 64 (the second K chunk of the hidden, head and colour layers); and
// dZ (two chunks).  At W = 32 the tail sits inside each chunk (columns
// 32..63) and T only pads the M = 128 wgrad operand.
#include "tc_common.cuh"

namespace roam {

namespace {

constexpr int kChunk = 16384;       // one 64-column chunk of 128 rows

template <int W, int H>
struct BwShape {
    using S = TcShape<W, H, false>;
    static_assert(S::kFold, "the tensor-core adjoint folds every bias into the MMAs (BF16, W <= 64)");
    static constexpr int kNX = H + 3;                 // X_0 .. X_{H+1}, X_g
    static constexpr int kOffX = S::kImageAlloc;
    static constexpr int kOffT = kOffX + kNX * kChunk;
    static constexpr int kOffDZ = kOffT + kChunk;
    static constexpr int kSmem = kOffDZ + 2 * kChunk;
    // TMEM: D (forward / dgrad accumulator) at column 0, then one wgrad
    // accumulator per layer l = 0 .. H+2 (H+2 = the 3-output layer)
    static constexpr int kDCols = S::N_HEAD;
    __host__ __device__ static constexpr int wN(int l) { return l == H ? S::N_HEAD : (l == H + 2 ? 16 : W); }
    __host__ __device__ static constexpr int wcol(int l)
    {
        int c = kDCols;
        for (int i = 0; i < l; ++i) c += wN(i);
        return c;
    }
    static constexpr int kCols = wcol(H + 3);
    static_assert(kCols <= 512, "TMEM holds D and every layer's wgrad accumulator");
};

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

// N consecutive TMEM columns of this thread's lane as floats, one wait for all
template <int N>
__device__ __forceinline__ void ldNf(uint32_t taddr, float (&v)[N])
{
    uint32_t r[N / 16][16];
#pragma unroll
    for (int c = 0; c < N / 16; ++c) tmem_ld16_nowait(taddr + (uint32_t)(16 * c), r[c]);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < N / 16; ++c)
#pragma unroll
        for (int q = 0; q < 16; ++q) v[16 * c + q] = __uint_as_float(r[c][q]);
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
__global__ void __launch_bounds__(128, 1)
    k_mlp_bwd_tc(const void *wimg, int64_t img_bytes, const float *affine, float sig_scale, int act, int64_t P,
                 SampleSrc src, BucketBufs b, Counters *ctr, const float4 *gsr, float *grad)
{
    using S = TcShape<W, H, false>;
    using B = BwShape<W, H>;
    constexpr int kLayers = S::kLayers;              // tensor-core layers of the forward chain
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_d, bar_w;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t *sm = smem_raw + (base - smem_u32(smem_raw));
    uint8_t *IMG = sm;
    uint8_t *T = sm + B::kOffT;
    uint8_t *DZ = sm + B::kOffDZ;
    const uint32_t sIMG = base, sX = base + B::kOffX, sT = base + B::kOffT, sDZ = base + B::kOffDZ;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid;                               // TMEM lane == tile row == sample
    const bool issuer = tid == 0;                     // forward chain
    const bool lead = (tid & 31) == 0;                // every warp's lane 0 commits each MMA group
    volatile int *abortp = &abort_flag;
    uint32_t *status = &ctr->status;

    if (tid == 0) {
        mbar_init(&bar_d, 4);                         // one commit per warp leader
        mbar_init(&bar_w, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the tail chunk only pads the wgrad operands at W = 32: keep it finite
    if (W < 64)
        for (int q = tid; q < kChunk / 16; q += 128) reinterpret_cast<uint4 *>(T)[q] = make_uint4(0u, 0u, 0u, 0u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = (uint32_t)(warp * 32) << 16;
    const uint32_t tD = tmem;

    const uint32_t n_tiles = ctr->n_tiles;
    const uint32_t t0 = (uint32_t)((uint64_t)n_tiles * blockIdx.x / gridDim.x);
    const uint32_t t1 = (uint32_t)((uint64_t)n_tiles * (blockIdx.x + 1) / gridDim.x);

    uint32_t d_ph = 0, w_ph = 0, n_commits = 0, n_waits = 0;
    bool w_pending = false;              // an image load in flight (thread 0's view)
    uint32_t cur = 0xffffffffu;
    bool wnew = true;                    // the wgrad accumulators hold nothing yet
    bool aborted = false;

    // issue, commit and wait: true when the MMAs landed
    auto mma_wait = [&]() -> bool {
        if (lead) {
            umma_commit(&bar_d);
            ++n_commits;
        }
        const bool got = mbar_wait(&bar_d, d_ph, abortp, status);
        if (lead && got) ++n_waits;
        d_ph ^= 1u;
        const bool all = __syncthreads_and(got) != 0;
        tc_fence_after();
        return all;
    };
    // every thread's generic shared-memory stores become visible to the MMAs
    auto publish = [&]() {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    };
    // flush the wgrad accumulators of field f to the global gradient
    auto flush = [&](uint32_t f) {
        float *gf = grad + (int64_t)f * P;
#pragma unroll 1
        for (int l = 0; l < H + 3; ++l) {
            const RowMap m = row_map<W, H>(l, row);
#pragma unroll 1
            for (int c = 0; c < B::wN(l); c += 16) {
                float v[16];
                ld16f(tmem + tlane + (uint32_t)(B::wcol(l) + c), v);
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
        tc_fence_before();
    };

    // the next tile's sample is gathered in stages during this tile's forward
    // layers (index, then record and ray, then position), so no stage waits
    // on its own load
    Tile tl_cur{0u, 0u, 0u, 0u};
    SampleIn nxt{0u, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    Pending pend{};
    if (t0 < t1) {
        tl_cur = b.tiles[t0];
        nxt = fetch_sample(src, b, tl_cur, row);
    }
    for (uint32_t t = t0; t < t1 && !aborted; ++t) {
        const Tile tl = tl_cur;
        const bool more = t + 1 < t1;
        const Tile tl_nx = more ? b.tiles[t + 1] : Tile{0u, 0u, 0u, 0u};
        const SampleIn smp = nxt;
        tl_cur = tl_nx;
        if (tl.count == 0) {
            if (more) nxt = fetch_sample(src, b, tl_nx, row);
            continue;
        }
        if (tl.field != cur) {
            if (cur != 0xffffffffu && !wnew) flush(cur);
            // generic reads of the old image (the epilogue tables) come before
            // the bulk copy that overwrites it
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                mbar_expect_tx(&bar_w, (uint32_t)S::kImageBytes);
                const uint8_t *gsrc = reinterpret_cast<const uint8_t *>(wimg) + (int64_t)tl.field * img_bytes;
                for (int off = 0; off < S::kImageBytes; off += 16384) {
                    const int nb = S::kImageBytes - off < 16384 ? S::kImageBytes - off : 16384;
                    bulk_g2s(IMG + off, gsrc + off, (uint32_t)nb, &bar_w);
                }
                w_pending = true;
            }
            // everyone waits for the image: the epilogues read its FP32 output table
            const bool ok = mbar_wait(&bar_w, w_ph, abortp, status);
            if (tid == 0 && ok) w_pending = false;
            w_ph ^= 1u;
            if (!__syncthreads_and(ok)) {
                aborted = true;
                break;
            }
            cur = tl.field;
            wnew = true;
        }

        // ---- the sample ----
        const bool valid = (uint32_t)row < tl.count;
        const float4 dl = valid ? gsr[smp.idx] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float *aff = affine + 6 * (int64_t)tl.field;

        // ---- X_0 = [F(x_loc) | 1] and the tail [1 | F(d) | 0] ----
        uint32_t tailp[16];
        {
            const float xl[3] = {fmaf(__ldg(aff + 0), smp.px, __ldg(aff + 3)),
                                 fmaf(__ldg(aff + 1), smp.py, __ldg(aff + 4)),
                                 fmaf(__ldg(aff + 2), smp.pz, __ldg(aff + 5))};
            float e[64];
            e[0] = xl[0]; e[1] = xl[1]; e[2] = xl[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float sn[10], cs[10];
                encode1<10>(xl[a], sn, cs);
#pragma unroll
                for (int k = 0; k < 10; ++k) {
                    e[3 + 6 * k + a] = sn[k];
                    e[6 + 6 * k + a] = cs[k];
                }
            }
            e[63] = 1.0f;
            uint32_t p[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) p[q] = pack_bf16(e[2 * q], e[2 * q + 1]);
            st_units<8>(sm + B::kOffX, row, 0, p);

            float ft[32];
            ft[0] = 1.0f;
            const float dv[3] = {smp.dx, smp.dy, smp.dz};
            ft[1] = dv[0]; ft[2] = dv[1]; ft[3] = dv[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float sn[4], cs[4];
                encode1<4>(dv[a], sn, cs);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    ft[4 + 6 * k + a] = sn[k];
                    ft[7 + 6 * k + a] = cs[k];
                }
            }
            ft[28] = ft[29] = ft[30] = ft[31] = 0.f;
#pragma unroll
            for (int q = 0; q < 16; ++q) tailp[q] = pack_bf16(ft[2 * q], ft[2 * q + 1]);
            if (W == 64) {
                uint32_t z[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) z[q] = 0u;
                st_units<4>(T, row, 0, tailp);
                st_units<4>(T, row, 4, z);
            }
        }
        // row `row` of X_i: the tail at W = 32 (columns 32..63); the
        // activations go in 16-column pieces (units 2c/16, 2c/16 + 1)
        auto store_tail = [&](int i) {
            if constexpr (W == 32) st_units<4>(sm + B::kOffX + i * kChunk, row, 4, tailp);
        };
        // ---- forward chain ----
        float s_logit = 0.f;
        float dsig = 0.f;
        bool ok = true;
#pragma unroll 1
        for (int l = 0; l < kLayers && ok; ++l) {
            publish();
            if (issuer) {
                const int K = S::K(l), N = S::N(l);
                const uint32_t idesc = idesc_bf16_t(N, 0, 0);
                const uint32_t xa = sX + (uint32_t)(l * kChunk);
                const uint32_t ba = sIMG + (uint32_t)S::offset(l);
#pragma unroll 1
                for (int ks = 0; ks < K / 16; ++ks) {
                    const int ch = ks >> 2, kin = ks & 3;
                    const uint32_t a = (ch == 0 ? xa : sT) + (uint32_t)(kin * 32);
                    umma_ss(tD, sdesc(a), sdesc(ba + (uint32_t)(ch * N * 128 + kin * 32)), idesc, ks > 0 ? 1u : 0u);
                }
            }
            if (l == 0) stage_index(pend, b, tl_nx, row, more);
            if (l == 1) stage_record(pend, src);
            if (l == 2) stage_ray(pend, src);
            ok = mma_wait();
            if (!ok) break;
            if (l < H) {
                // next hidden input: ReLU
                uint8_t *xc = sm + B::kOffX + (l + 1) * kChunk;
#pragma unroll
                for (int cb = 0; cb < W; cb += 32) {
                    float va[32];
                    ldNf<32>(tD + tlane + (uint32_t)cb, va);
#pragma unroll
                    for (int c = 0; c < 32; c += 16) {
                        uint32_t p[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) p[q] = pack_bf16_relu(va[c + 2 * q], va[c + 2 * q + 1]);
                        st_units<2>(xc, row, (cb + c) / 8, p);
                    }
                }
                store_tail(l + 1);
            } else if (l == H) {
                // head: features (linear) -> colour input, column W = density logit
                uint8_t *xc = sm + B::kOffX + (H + 1) * kChunk;
#pragma unroll
                for (int cb = 0; cb < W; cb += 32) {
                    float va[32];
                    ldNf<32>(tD + tlane + (uint32_t)cb, va);
#pragma unroll
                    for (int c = 0; c < 32; c += 16) {
                        uint32_t p[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) p[q] = pack_bf16(va[c + 2 * q], va[c + 2 * q + 1]);
                        st_units<2>(xc, row, (cb + c) / 8, p);
                    }
                }
                {
                    float v[16];
                    ld16f(tD + tlane + (uint32_t)W, v);
                    s_logit = v[0];
                }
                store_tail(H + 1);
            } else {
                // colour: z -> g = relu(z) (X_g), rgb = sigmoid(Wo g + bo) in FP32, then
                // the output layer's adjoint and dZ of the colour layer
                const float4 *wo = reinterpret_cast<const float4 *>(IMG + S::kMatBytes);
                float4 acc = wo[W];
#pragma unroll
                for (int cb = 0; cb < W; cb += 32) {
                    float va[32];
                    ldNf<32>(tD + tlane + (uint32_t)cb, va);
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const float gk = fmaxf(va[k], 0.f);
                        const float4 wk = wo[cb + k];
                        acc.x = fmaf(wk.x, gk, acc.x);
                        acc.y = fmaf(wk.y, gk, acc.y);
                        acc.z = fmaf(wk.z, gk, acc.z);
                    }
                }
                const float r0 = sigmoid_f(acc.x), r1 = sigmoid_f(acc.y), r2 = sigmoid_f(acc.z);
                const float dz0 = dl.y * r0 * (1.f - r0), dz1 = dl.z * r1 * (1.f - r1), dz2 = dl.w * r2 * (1.f - r2);
                dsig = dl.x * sig_scale *
                       (act == ROAM_RELU ? (s_logit > 0.f ? 1.f : 0.f) : sigmoid_f(s_logit));
                uint8_t *xg = sm + B::kOffX + (H + 2) * kChunk;
#pragma unroll
                for (int c = 0; c < W; c += 16) {
                    float va[16];
                    ld16f(tD + tlane + (uint32_t)c, va);     // re-read: cheaper than holding all W in registers
                    uint32_t pg[8], pd[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float gg[2], dd[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float zk = va[2 * q + h];
                            const float4 wk = wo[c + 2 * q + h];
                            gg[h] = fmaxf(zk, 0.f);
                            dd[h] = zk > 0.f ? fmaf(wk.x, dz0, fmaf(wk.y, dz1, wk.z * dz2)) : 0.f;
                        }
                        pg[q] = pack_bf16(gg[0], gg[1]);
                        pd[q] = pack_bf16(dd[0], dd[1]);
                    }
                    st_units<2>(xg, row, c / 8, pg);
                    // dZ: colour rows in chunk 0 (columns 0..W-1), the 3-output layer's in chunk 1
                    st_units<2>(DZ, row, c / 8, pd);
                }
                store_tail(H + 2);
                if constexpr (W == 32) {
                    uint32_t z4[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) z4[q] = 0u;
                    st_units<4>(DZ, row, 4, z4);
                }
                uint32_t po[8];
                po[0] = pack_bf16(dz0, dz1);
                po[1] = pack_bf16(dz2, 0.f);
#pragma unroll
                for (int q = 2; q < 8; ++q) po[q] = 0u;
                st_units<2>(DZ + kChunk, row, 0, po);
            }
        }
        if (!ok) {
            aborted = true;
            break;
        }

        // ---- backward chain ----
        const uint32_t wacc0 = wnew ? 0u : 1u;
        // wgrad of layer l: D_w(l)[k][n] += sum_s X[s][k] dZ[s][n]
        auto issue_wgrad = [&](int l, uint32_t xa, uint32_t dza, uint32_t dz_lbo) {
            const int N = B::wN(l);
            const uint32_t idesc = idesc_bf16_t(N, 1, 1);
            const uint32_t lbo_x = sT - xa;
            const uint32_t td = tmem + (uint32_t)B::wcol(l);
#pragma unroll 1
            for (int j = 0; j < 8; ++j)
                umma_ss(td, sdesc_mn(xa + (uint32_t)(j * 2048), lbo_x),
                        sdesc_mn(dza + (uint32_t)(j * 2048), dz_lbo), idesc, (j > 0 || wacc0) ? 1u : 0u);
        };
        // dgrad of layer l: D[s][k] = sum_n dZ[s][n] W_l[n][k], k < W, over Kn outputs
        auto issue_dgrad = [&](int l, int Kn) {
            const uint32_t idesc = idesc_bf16_t(W, 0, 1);
            const uint32_t ba = sIMG + (uint32_t)S::offset(l);
#pragma unroll 1
            for (int ks = 0; ks < Kn / 16; ++ks) {
                const int ch = ks >> 2, kin = ks & 3;
                umma_ss(tD, sdesc(sDZ + (uint32_t)(ch * kChunk + kin * 32)), sdesc_mn(ba + (uint32_t)(ks * 2048), 1024u),
                        idesc, ks > 0 ? 1u : 0u);
            }
        };
        // reads dX (W columns of D) and writes dZ of the layer below: masked by
        // that layer's ReLU (X_i > 0) when i > 0, and at the head also the density column
        auto next_dz = [&](int i, bool relu, bool head) {
            const uint8_t *xc = sm + B::kOffX + i * kChunk;
#pragma unroll
            for (int cb = 0; cb < W; cb += 32) {
                float va[32];
                ldNf<32>(tD + tlane + (uint32_t)cb, va);
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    const int c = cb + c0;
                    uint4 m0 = make_uint4(0u, 0u, 0u, 0u), m1 = m0;
                    if (relu) {
                        m0 = *reinterpret_cast<const uint4 *>(xc + sw_off(row, c / 8));
                        m1 = *reinterpret_cast<const uint4 *>(xc + sw_off(row, c / 8 + 1));
                    }
                    const uint32_t mk[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
                    uint32_t p[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float a = va[c0 + 2 * q], bb = va[c0 + 2 * q + 1];
                        if (relu) {
                            if ((mk[q] & 0xffffu) == 0u) a = 0.f;
                            if ((mk[q] >> 16) == 0u) bb = 0.f;
                        }
                        p[q] = pack_bf16(a, bb);
                    }
                    st_units<2>(DZ, row, c / 8, p);
                }
            }
            if constexpr (W == 64) {
                if (head) {
                    uint32_t po[8];
                    po[0] = pack_bf16(dsig, 0.f);
#pragma unroll
                    for (int q = 1; q < 8; ++q) po[q] = 0u;
                    st_units<2>(DZ + kChunk, row, 0, po);
                }
            } else {
                uint32_t z4[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) z4[q] = 0u;
                if (head) z4[0] = pack_bf16(dsig, 0.f);
                st_units<4>(DZ, row, 4, z4);
            }
        };

        // output and colour layers
        publish();
        // independent accumulators, so three warps issue them side by side
        if (tid == 0) issue_wgrad(H + 2, sX + (uint32_t)((H + 2) * kChunk), sDZ + kChunk, 1024u);
        if (tid == 32) issue_wgrad(H + 1, sX + (uint32_t)((H + 1) * kChunk), sDZ, 1024u);
        if (tid == 64) issue_dgrad(H + 1, W);
        if (!mma_wait()) { aborted = true; break; }
        next_dz(H + 1, false, true);          // dZ of the head: [d feat | d logit | 0]
        // head
        publish();
        if (tid == 0) issue_wgrad(H, sX + (uint32_t)(H * kChunk), sDZ, (uint32_t)kChunk);
        if (tid == 32) issue_dgrad(H, S::N_HEAD);
        if (!mma_wait()) { aborted = true; break; }
        next_dz(H, true, false);
        // hidden layers H-1 .. 1
        bool ok2 = true;
#pragma unroll 1
        for (int l = H - 1; l >= 1; --l) {
            publish();
            if (tid == 0) issue_wgrad(l, sX + (uint32_t)(l * kChunk), sDZ, 1024u);
            if (tid == 32) issue_dgrad(l, W);
            if (!mma_wait()) { ok2 = false; break; }
            next_dz(l, true, false);
        }
        if (!ok2) { aborted = true; break; }
        // first layer: wgrad only
        publish();
        if (issuer) issue_wgrad(0, sX, sDZ, 1024u);
        if (!mma_wait()) { aborted = true; break; }
        wnew = false;
        if (more) nxt = stage_finish(pend, src);
    }
    if (!aborted && cur != 0xffffffffu && !wnew) flush(cur);
    // drain before TMEM is freed: a commit whose wait gave up, an image load nobody waited for
    if (lead && n_commits > n_waits) mbar_wait(&bar_d, (n_commits - 1) & 1u, abortp, status, true);
    if (tid == 0 && w_pending) mbar_wait(&bar_w, w_ph ^ 1u, abortp, status, true);
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
    k_mlp_bwd_tc<W, H><<<n_sm, 128, smem, s>>>(w.wimg, w.img_bytes, w.affine, w.sigma_scale, w.act, w.P, src, b, ctr,
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
