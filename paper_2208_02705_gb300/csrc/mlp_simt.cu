// FP32 SIMT evaluation of the per-field tiny MLPs (the plain FP32 form of
// querying many MLPs at once), tiles of 128 samples of one field, each layer
// a register-tiled FP32 product: a thread owns 4 consecutive samples (a
// sample group) and TN = W / OG of the layer's outputs, so every weight it
// loads feeds 4 FMAs and every activation TN.  The layer's input sits in
// shared memory, feature-major ([k][128 samples]); the weights are a
// transposed FP32 copy ([in][out], output rows padded to 16 bytes), in
// shared memory (W <= 64) or read through the L1 cache (W = 128), each
// warp's loads of them uniform.  Positional encoding (Eq. 1's F(.)) is
// recomputed in the kernel.  The density (the head's extra output) rides in
// the head layer's loop; the 3-output colour layer is formed from the colour
// features still in registers, the output groups' shares summed through
// shared memory.
#include "internal.cuh"

namespace roam {

namespace {

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// Thread layout of one tile: OG warps, one per output group, each over the
// tile's 32 sample groups of 4 samples; lane l of warp og owns samples
// 4l .. 4l + 3 and outputs n = 4 (q OG + og) + i (q < TN / 4, i < 4).  A
// warp's weight loads are uniform (one broadcast per float4) and its
// activation loads one contiguous 512-byte row segment, so each row k costs
// the shared memory 4 + TN / 4 wavefronts per warp.
template <int W>
struct SimtShape {
    static constexpr int OG = W >= 128 ? 8 : 4;
    static constexpr int TN = W / OG;
    static constexpr int kThreads = 32 * OG;
    static constexpr int kMinBlocks = 2;          // blocks per SM of the read-only-path form (W = 128)
    static constexpr int kRows = (W + kPeD) > kPeX ? (W + kPeD) : kPeX;   // activation rows in shared memory
    static constexpr size_t kSmem = (size_t)kRows * 128 * sizeof(float) + 128 * sizeof(uint32_t);
    static_assert(TN % 4 == 0, "whole float4 runs per thread");
    static_assert(3 * OG + 1 <= kRows, "the colour sums fit in the activation buffer");
};

// Parameter offsets of the transposed copy: per layer WT[in][n_pad] then
// bias[n_pad]; the head's row holds the W features, then the density logit
// (column W), then zeros.
struct TLayout {
    int64_t l1, hid, head, col, out, total;
    __host__ __device__ TLayout(int W, int H)
    {
        int64_t o = 0;
        l1 = o;   o += (int64_t)kPeX * W + W;
        hid = o;  o += (int64_t)(H - 1) * ((int64_t)W * W + W);
        head = o; o += (int64_t)W * round4(1 + W) + round4(1 + W);
        col = o;  o += (int64_t)(W + kPeD) * W + W;
        out = o;  o += (int64_t)W * 4 + 4;
        total = o;
    }
};

// Weight loads: from the block's shared copy, or through the read-only path.
template <bool kShared>
__device__ __forceinline__ float4 ldw4(const float4 *p)
{
    if constexpr (kShared) return *p;
    else return __ldg(p);
}
template <bool kShared>
__device__ __forceinline__ float ldw1(const float *p)
{
    if constexpr (kShared) return *p;
    else return __ldg(p);
}

// Accumulators: this thread's output j of sample s is component j % 2 of
// acc[s][j / 2], so that each packed FMA (__ffma2_rn: two independent
// single-precision FMAs, each rounded as fmaf) updates two outputs.
template <int TN>
__device__ __forceinline__ float acc_get(const float2 (&acc)[4][TN / 2], int s, int j)
{
    return (j & 1) ? acc[s][j >> 1].y : acc[s][j >> 1].x;
}

// acc[s][4q + i] = b[n] + sum_k x[k][4 sg + s] WT[k][n] over rows [0, K) of
// the shared activations, n = 4 (q OG + og) + i; with kDens also
// dens[s] = b[W] + sum_k x[k][4 sg + s] WT[k][W] (every thread of the
// sample group forms the same value).
template <int K, int N, int OG, int TN, bool kDens, bool kShared>
__device__ __forceinline__ void dense_tile(const float *__restrict__ sx, const float *__restrict__ wt, int og,
                                           int sg, float2 (&acc)[4][TN / 2], float (&dens)[4])
{
    const float4 *b4 = reinterpret_cast<const float4 *>(wt + (int64_t)K * N) + og;
#pragma unroll
    for (int q = 0; q < TN / 4; ++q) {
        const float4 b = ldw4<kShared>(b4 + q * OG);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            acc[s][2 * q] = make_float2(b.x, b.y);
            acc[s][2 * q + 1] = make_float2(b.z, b.w);
        }
    }
    if constexpr (kDens) {
        const float bd = ldw1<kShared>(wt + (int64_t)K * N + (N - 4));
#pragma unroll
        for (int s = 0; s < 4; ++s) dens[s] = bd;
    }
    // software-pipelined: row k + 1's weights and activations are in flight
    // while row k's 8 TN packed FMAs issue (two register sets used in turn, so no
    // copies between rows)
    const float4 *xs = reinterpret_cast<const float4 *>(sx) + sg;   // row k at xs[32 k]
    const float4 *wr = reinterpret_cast<const float4 *>(wt) + og;    // row k at wr[k N / 4]
    float4 wa[TN / 4], wb[TN / 4], xa, xb;
    float da = 0.f, db = 0.f;
    auto load = [&](int k, float4(&wv)[TN / 4], float4 &xv, float &dv) {
        const float4 *wk = wr + (int64_t)k * (N / 4);
#pragma unroll
        for (int q = 0; q < TN / 4; ++q) wv[q] = ldw4<kShared>(wk + q * OG);
        xv = xs[32 * k];
        if constexpr (kDens) dv = ldw1<kShared>(wt + (int64_t)k * N + (N - 4));
    };
    auto fma_row = [&](const float4(&wv)[TN / 4], const float4 &xv, float dv) {
        const float x4[4] = {xv.x, xv.y, xv.z, xv.w};
        float2 xx[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) xx[s] = make_float2(x4[s], x4[s]);
#pragma unroll
        for (int q = 0; q < TN / 4; ++q) {
            const float2 w01 = make_float2(wv[q].x, wv[q].y), w23 = make_float2(wv[q].z, wv[q].w);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                acc[s][2 * q] = __ffma2_rn(w01, xx[s], acc[s][2 * q]);
                acc[s][2 * q + 1] = __ffma2_rn(w23, xx[s], acc[s][2 * q + 1]);
            }
        }
        if constexpr (kDens) {
#pragma unroll
            for (int s = 0; s < 4; ++s) dens[s] = fmaf(dv, x4[s], dens[s]);
        }
    };
    if constexpr (kShared) {
        load(0, wa, xa, da);
#pragma unroll 1
        for (int k = 0; k < K; k += 2) {
            if (k + 1 < K) load(k + 1, wb, xb, db);
            fma_row(wa, xa, da);
            if (k + 1 < K) {
                if (k + 2 < K) load(k + 2, wa, xa, da);
                fma_row(wb, xb, db);
            }
        }
    } else {
        // (the read-only-path form runs at 128 registers: no second set; the
        // compiler schedules two rows at a time)
#pragma unroll 2
        for (int k = 0; k < K; ++k) {
            load(k, wb, xb, db);
            fma_row(wb, xb, db);
        }
    }
}

// Writes this thread's outputs (through a ReLU when kRelu) as rows n of the
// shared activations, its 4 samples at once.
template <int OG, int TN, bool kRelu>
__device__ __forceinline__ void store_tile(float *sx, const float2 (&acc)[4][TN / 2], int og, int sg)
{
    float4 *xs = reinterpret_cast<float4 *>(sx) + sg;
#pragma unroll
    for (int q = 0; q < TN / 4; ++q) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = 4 * (q * OG + og) + i;
            const int j = 4 * q + i;
            float4 v = make_float4(acc_get<TN>(acc, 0, j), acc_get<TN>(acc, 1, j), acc_get<TN>(acc, 2, j),
                                   acc_get<TN>(acc, 3, j));
            if (kRelu) {
                v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
            }
            xs[32 * n] = v;
        }
    }
}

// F(x) = [x, sin(2^k pi x), cos(2^k pi x)]_k, three sines then three cosines
// per frequency, as rows base.. of column tid; 2^k x is exact in FP32,
// sincospif reduces it exactly.
template <int L>
__device__ __forceinline__ void encode(float x0, float x1, float x2, float *sx, int base, int tid)
{
    sx[(base + 0) * 128 + tid] = x0;
    sx[(base + 1) * 128 + tid] = x1;
    sx[(base + 2) * 128 + tid] = x2;
    const float xs[3] = {x0, x1, x2};
#pragma unroll
    for (int k = 0; k < L; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s, c;
            sincospif(ldexpf(xs[a], k), &s, &c);
            sx[(base + 3 + 6 * k + a) * 128 + tid] = s;
            sx[(base + 6 + 6 * k + a) * 128 + tid] = c;
        }
    }
}

// Field-local coordinate scale * (o + t d) + offset of sample j, with
// t = (j + 1/2) delta and d = dh + dl carried as unevaluated FP32 pairs
// (error-free products and sums, explicitly rounded operations so that no
// step is contracted): accurate to about one FP32 ulp of the result.
__device__ __forceinline__ float local_coord(float th0, float delta, float o, float dh, float dl, float scale,
                                             float offset)
{
    const float t_hi = __fmul_rn(th0, delta);
    const float t_lo = __fmaf_rn(th0, delta, -t_hi);
    const float ph = __fmul_rn(t_hi, dh);
    const float pl = __fadd_rn(__fmaf_rn(t_hi, dh, -ph), __fadd_rn(__fmul_rn(t_hi, dl), __fmul_rn(t_lo, dh)));
    const float sh = __fadd_rn(o, ph);
    const float bv = __fsub_rn(sh, o);
    const float se = __fadd_rn(__fsub_rn(o, __fsub_rn(sh, bv)), __fsub_rn(ph, bv));
    const float sl = __fadd_rn(se, pl);
    const float qh = __fmul_rn(scale, sh);
    const float ql = __fadd_rn(__fmaf_rn(scale, sh, -qh), __fmul_rn(scale, sl));
    return __fadd_rn(__fadd_rn(qh, offset), ql);
}

__device__ __forceinline__ float softplus_f(float s) { return s > 20.f ? s : log1pf(expf(s)); }
__device__ __forceinline__ float sigmoid_f(float s) { return 1.f / (1.f + expf(-s)); }

__device__ __forceinline__ void group_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// One tile of 128 samples through the whole network by one thread group of
// SimtShape<W>::kThreads threads (barrier `bar`): sx / s_idx are the group's
// activations and sample indices, wf the field's transposed weights (in
// shared memory when kShared).
template <int W, int H, bool kShared>
__device__ __forceinline__ void run_tile(const Tile &tl, const MlpWeights &w, const SampleSrc &src,
                                         const BucketBufs &b, const float *wf, float *sx, uint32_t *s_idx,
                                         int tid, int bar, float4 *out)
{
    using S = SimtShape<W>;
    constexpr int OG = S::OG, TN = S::TN, NT = S::kThreads;
    constexpr int NH = round4(1 + W);
    const int og = tid >> 5, sg = tid & 31;
    const TLayout L(W, H);
    float2 acc[4][TN / 2];
    float dens[4];
    // ---- gather and encode: thread tid < 128 takes sample tid of the tile ----
    float dx = 0.f, dy = 0.f, dz = 1.f;
    group_sync(bar, NT);                                 // the previous tile's reads of sx and s_idx are done
    if (tid < 128) {
        const bool valid = (uint32_t)tid < tl.count;
        const uint32_t idx = valid ? b.sorted[tl.start + tid] : 0u;
        const float *aff = w.affine + 6 * (int64_t)tl.field;
        float xl0 = 0.f, xl1 = 0.f, xl2 = 0.f;
        if (valid) {
            if (src.mode == 0) {
                const uint32_t col = idx >> 5;
                const uint32_t i = (col / (uint32_t)src.R) * 32u + (idx & 31u);
                const uint32_t ray = src.live ? src.live[i] : i;
                const uint32_t j = src.recs[idx] & 0xffffu;
                const float4 o = src.st.orig[ray], d = src.st.dir[ray];
                dx = d.x; dy = d.y; dz = d.z;
                if (src.accurate) {
                    const float4 dl = src.st.dir_lo[ray];
                    const float th0 = (float)j + 0.5f;
                    xl0 = local_coord(th0, src.delta, o.x, d.x, dl.x, aff[0], aff[3]);
                    xl1 = local_coord(th0, src.delta, o.y, d.y, dl.y, aff[1], aff[4]);
                    xl2 = local_coord(th0, src.delta, o.z, d.z, dl.z, aff[2], aff[5]);
                } else {
                    const float tt = ((float)j + 0.5f) * src.delta;
                    xl0 = fmaf(aff[0], fmaf(tt, d.x, o.x), aff[3]);
                    xl1 = fmaf(aff[1], fmaf(tt, d.y, o.y), aff[4]);
                    xl2 = fmaf(aff[2], fmaf(tt, d.z, o.z), aff[5]);
                }
            } else {
                const float px = src.p[3 * (int64_t)idx], py = src.p[3 * (int64_t)idx + 1],
                            pz = src.p[3 * (int64_t)idx + 2];
                dx = src.d[3 * (int64_t)idx]; dy = src.d[3 * (int64_t)idx + 1]; dz = src.d[3 * (int64_t)idx + 2];
                xl0 = fmaf(aff[0], px, aff[3]);
                xl1 = fmaf(aff[1], py, aff[4]);
                xl2 = fmaf(aff[2], pz, aff[5]);
            }
        }
        s_idx[tid] = valid ? idx : 0xffffffffu;
        encode<10>(xl0, xl1, xl2, sx, 0, tid);
    }
    group_sync(bar, NT);

    // ---- L1, then F(d) beside the hidden features (rows W ..), which
    // only the colour layer reads ----
    dense_tile<kPeX, W, OG, TN, false, kShared>(sx, wf + L.l1, og, sg, acc, dens);
    group_sync(bar, NT);
    store_tile<OG, TN, true>(sx, acc, og, sg);
    if (tid < 128) encode<4>(dx, dy, dz, sx, W, tid);
    group_sync(bar, NT);
#pragma unroll 1
    for (int k = 0; k < H - 1; ++k) {
        dense_tile<W, W, OG, TN, false, kShared>(sx, wf + L.hid + (int64_t)k * (W * W + W), og, sg, acc, dens);
        group_sync(bar, NT);
        store_tile<OG, TN, true>(sx, acc, og, sg);
        group_sync(bar, NT);
    }
    // ---- head: features (linear) and the density logit ----
    dense_tile<W, NH, OG, TN, true, kShared>(sx, wf + L.head, og, sg, acc, dens);
    group_sync(bar, NT);
    store_tile<OG, TN, false>(sx, acc, og, sg);
    group_sync(bar, NT);
    // ---- colour features g = relu(Wc [feat; F(d)] + bc), in registers ----
    dense_tile<W + kPeD, W, OG, TN, false, kShared>(sx, wf + L.col, og, sg, acc, dens);
    // ---- rgb = sigmoid(Wo g + bo): each warp's share of the sums over its
    // outputs, then thread t < 128 adds the OG shares of sample t ----
    const float4 *wo = reinterpret_cast<const float4 *>(wf + L.out);   // [W][4], then bias[4]
    float z[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s) z[s][0] = z[s][1] = z[s][2] = 0.f;
#pragma unroll
    for (int q = 0; q < TN / 4; ++q) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 wk = ldw4<kShared>(wo + 4 * (q * OG + og) + i);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float g = fmaxf(acc_get<TN>(acc, s, 4 * q + i), 0.f);
                z[s][0] = fmaf(wk.x, g, z[s][0]);
                z[s][1] = fmaf(wk.y, g, z[s][1]);
                z[s][2] = fmaf(wk.z, g, z[s][2]);
            }
        }
    }
    // shares and the density (every warp formed it) through the activation
    // buffer, rows (3 og + c) and 3 OG
    group_sync(bar, NT);                                 // every warp is done reading the colour input
    float4 *red = reinterpret_cast<float4 *>(sx) + sg;
#pragma unroll
    for (int c = 0; c < 3; ++c) red[32 * (3 * og + c)] = make_float4(z[0][c], z[1][c], z[2][c], z[3][c]);
    if (og == 0) red[32 * 3 * OG] = make_float4(dens[0], dens[1], dens[2], dens[3]);
    group_sync(bar, NT);
    if (tid < 128) {
        const uint32_t idx = s_idx[tid];
        if (idx != 0xffffffffu) {
            const float4 bo = ldw4<kShared>(wo + W);
            float zc[3] = {bo.x, bo.y, bo.z};
#pragma unroll
            for (int g = 0; g < OG; ++g) {
#pragma unroll
                for (int c = 0; c < 3; ++c) zc[c] += sx[(3 * g + c) * 128 + tid];
            }
            const float sl = sx[3 * OG * 128 + tid];
            const float sigma = w.sigma_scale * (w.act == ROAM_RELU ? fmaxf(sl, 0.f) : softplus_f(sl));
            out[idx] = make_float4(sigma, sigmoid_f(zc[0]), sigmoid_f(zc[1]), sigmoid_f(zc[2]));
        }
    }
}

// Tiles of one width class split evenly over the blocks, in order.
__device__ __forceinline__ void tile_range(const Counters *ctr, int cls, uint32_t &t0, uint32_t &t1)
{
    const uint32_t c0 = ctr->class_tiles[cls], n_tiles = ctr->class_tiles[cls + 1] - c0;
    t0 = c0 + (uint32_t)((uint64_t)n_tiles * blockIdx.x / gridDim.x);
    t1 = c0 + (uint32_t)((uint64_t)n_tiles * (blockIdx.x + 1) / gridDim.x);
}

// Weights through the read-only path (W = 128: a field's 378 KB do not fit
// in shared memory): one thread group per block, several blocks per SM.
template <int W, int H>
__global__ void __launch_bounds__(SimtShape<W>::kThreads, SimtShape<W>::kMinBlocks)
    k_mlp_simt(MlpWeights w, SampleSrc src, BucketBufs b, Counters *ctr, float4 *out)
{
    using S = SimtShape<W>;
    extern __shared__ float sx[];                       // [kRows][128 samples], then 128 sample indices
    uint32_t *s_idx = reinterpret_cast<uint32_t *>(sx + S::kRows * 128);
    uint32_t t0, t1;
    tile_range(ctr, w.cls, t0, t1);
    for (uint32_t t = t0; t < t1; ++t) {
        const Tile tl = b.tiles[t];
        const float *wf = w.wt + (int64_t)((int)tl.field - w.field_base) * w.Pt;
        run_tile<W, H, false>(tl, w, src, b, wf, sx, s_idx, threadIdx.x, 1, out);
    }
}

// Weights in shared memory (W <= 64): one block per SM holds the current
// field's transposed copy and kGroups thread groups that take the field's
// tiles in turn, each with its own activations and barrier.  Tiles come
// sorted by field, so a block reloads the copy only where its run of tiles
// crosses into the next field.
template <int W>
struct SimtSharedShape {
    static constexpr int kGroups = 2;
    static constexpr size_t kGroupFloats = (size_t)SimtShape<W>::kRows * 128 + 128;
    static size_t smem(int64_t Pt) { return ((size_t)Pt + kGroups * kGroupFloats) * sizeof(float); }
};

template <int W, int H>
__global__ void __launch_bounds__(SimtSharedShape<W>::kGroups * SimtShape<W>::kThreads, 1)
    k_mlp_simt_sw(MlpWeights w, SampleSrc src, BucketBufs b, Counters *ctr, float4 *out)
{
    using S = SimtShape<W>;
    using SS = SimtSharedShape<W>;
    extern __shared__ float4 smem4[];
    __shared__ uint32_t s_end;
    float *wsm = reinterpret_cast<float *>(smem4);                      // Pt floats (a multiple of 4)
    const int grp = threadIdx.x / S::kThreads, tid = threadIdx.x % S::kThreads;
    float *sx = wsm + w.Pt + grp * SS::kGroupFloats;
    uint32_t *s_idx = reinterpret_cast<uint32_t *>(sx + S::kRows * 128);
    uint32_t t0, t1;
    tile_range(ctr, w.cls, t0, t1);
    uint32_t t = t0;
    while (t < t1) {
        // the run of tiles of field f starting at t: its end is the first
        // tile of another field (tiles are sorted by field)
        const uint32_t f = b.tiles[t].field;
        __syncthreads();                                 // every group is done with the previous copy
        if (threadIdx.x == 0) s_end = t1;
        __syncthreads();
        for (uint32_t base = t + 1; base < t1; base += blockDim.x) {
            const uint32_t c = base + threadIdx.x;
            if (c < t1 && b.tiles[c].field != f) atomicMin(&s_end, c);
            __syncthreads();
            const bool found = s_end < t1;
            __syncthreads();
            if (found) break;
        }
        const uint32_t e = s_end;
        // the field's transposed copy into shared memory
        const float4 *src4 = reinterpret_cast<const float4 *>(w.wt + (int64_t)((int)f - w.field_base) * w.Pt);
        for (int64_t i = threadIdx.x; i < w.Pt / 4; i += blockDim.x) smem4[i] = __ldg(src4 + i);
        __syncthreads();
        for (uint32_t u = t + (uint32_t)grp; u < e; u += SS::kGroups) {
            const Tile tl = b.tiles[u];
            run_tile<W, H, true>(tl, w, src, b, wsm, sx, s_idx, tid, 1 + grp, out);
        }
        t = e;
    }
}

// API layout -> transposed copy: one thread per source parameter.
__global__ void k_pack_simt(const float *__restrict__ w32, int n_fields, int W, int H, int64_t P,
                            float *__restrict__ wt, int64_t Pt)
{
    const TLayout L(W, H);
    const int64_t n = (int64_t)n_fields * P;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = g / P;
        int64_t q = g % P;
        // walk the layers of the API layout: (n_out, n_in, dst offset, padded n_out)
        int64_t dst = -1;
        const int nl = H + 3;
        for (int l = 0; l < nl && dst < 0; ++l) {
            int n_out, n_in, n_pad;
            int64_t base;
            if (l == 0) { n_out = W; n_in = kPeX; base = L.l1; n_pad = W; }
            else if (l < H) { n_out = W; n_in = W; base = L.hid + (int64_t)(l - 1) * (W * W + W); n_pad = W; }
            else if (l == H) { n_out = 1 + W; n_in = W; base = L.head; n_pad = round4(1 + W); }
            else if (l == H + 1) { n_out = W; n_in = W + kPeD; base = L.col; n_pad = W; }
            else { n_out = 3; n_in = W; base = L.out; n_pad = 4; }
            const int64_t nw = (int64_t)n_out * n_in;
            // the head's output 0 (density) goes to column W, its features to 0 .. W-1
            auto column = [&](int64_t o) { return l == H ? (o == 0 ? (int64_t)W : o - 1) : o; };
            if (q < nw) {
                const int64_t o = q / n_in, i = q % n_in;
                dst = base + i * n_pad + column(o);
            } else if (q < nw + n_out) {
                dst = base + (int64_t)n_in * n_pad + column(q - nw);
            } else {
                q -= nw + n_out;
            }
        }
        if (dst >= 0) wt[f * Pt + dst] = w32[g];
    }
}

}  // namespace

int64_t simt_transposed_size(int W, int H) { return TLayout(W, H).total; }

void launch_pack_simt(const float *w32, int n_fields, int W, int H, int64_t P, float *wt, int64_t Pt,
                      cudaStream_t s)
{
    cudaMemsetAsync(wt, 0, (size_t)n_fields * Pt * sizeof(float), s);
    k_pack_simt<<<1024, 256, 0, s>>>(w32, n_fields, W, H, P, wt, Pt);
}

template <int W, int H>
static void launch_t(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, float4 *out,
                     int n_sm, cudaStream_t s)
{
    using S = SimtShape<W>;
    if constexpr (W <= 64) {
        // one block per SM, the field's weights in shared memory
        const size_t sh = SimtSharedShape<W>::smem(w.Pt);
        static int smem_set[kMaxDevices] = {};
        raise_smem_limit((const void *)k_mlp_simt_sw<W, H>, (int)sh, smem_set);
        k_mlp_simt_sw<W, H><<<n_sm, SimtSharedShape<W>::kGroups * S::kThreads, sh, s>>>(w, src, b, ctr, out);
    } else {
        // one wave of resident blocks; each takes a contiguous run of tiles
        static int smem_set[kMaxDevices] = {};
        raise_smem_limit((const void *)k_mlp_simt<W, H>, (int)S::kSmem, smem_set);
        static int per_sm_dev[kMaxDevices] = {};
        int dev = -1;
        cudaGetDevice(&dev);
        int per_sm = dev >= 0 && dev < kMaxDevices ? per_sm_dev[dev] : 0;
        if (per_sm == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_simt<W, H>, S::kThreads, S::kSmem) !=
                    cudaSuccess || per_sm < 1)
                per_sm = 1;
            if (dev >= 0 && dev < kMaxDevices) per_sm_dev[dev] = per_sm;
        }
        k_mlp_simt<W, H><<<n_sm * per_sm, S::kThreads, S::kSmem, s>>>(w, src, b, ctr, out);
    }
}

void launch_mlp_simt(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, float4 *out,
                     int n_sm, cudaStream_t s)
{
#define ROAM_CASE(WW, HH) \
    if (w.W == WW && w.H == HH) { launch_t<WW, HH>(w, src, b, ctr, out, n_sm, s); return; }
    ROAM_CASE(32, 1) ROAM_CASE(32, 2) ROAM_CASE(32, 3) ROAM_CASE(32, 4)
    ROAM_CASE(64, 1) ROAM_CASE(64, 2) ROAM_CASE(64, 3) ROAM_CASE(64, 4)
    ROAM_CASE(128, 1) ROAM_CASE(128, 2) ROAM_CASE(128, 3) ROAM_CASE(128, 4)
#undef ROAM_CASE
}

}  // namespace roam
