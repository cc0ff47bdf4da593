// tcgen05 BF16 evaluation of the per-field tiny MLPs (the concurrent MLP
// queries of Sec. "Real-time Rendering Speedup" as a grouped GEMM chain on
// the 5th-generation tensor cores).  One tile = 128 samples of one field =
// one M=128 MMA row block; every layer of the chain is
//   D[128 x N] (TMEM, FP32) = A[128 x K] (TMEM, BF16) * B[K x N] (SMEM, BF16)
// with tcgen05.mma kind::f16.  The activations A never touch shared memory:
// the epilogue reads D with tcgen05.ld (one row per thread), converts
// (cvt.rn.relu.bf16x2 fuses the ReLU) and writes the next layer's A with
// tcgen05.st, so the MMA streams only the weights from shared memory.  Every
// bias rides in the MMA: A carries a constant-1 column and B the bias in the
// matching row.  The field's weight image (all layers' B operands in the
// 128-byte-swizzled K-major layout, then an FP32 table of the 3-output
// layer) is copied to shared memory by the bulk-copy (TMA) engine when the
// field changes.
//
// A columns (row = sample):
//   L1 input        [F(x_loc) (63) | 1]                          K = 64
//   after L1        [h (W) | 1 | F(d) (27) | 0 0 0 0]             (the tail stays)
//   hidden / head   [h (W) | 1 | ...]     B zero past the bias    K = W + 16
//   colour          [feat (W) | 1 | F(d) (27) | 0 0 0 0]          K = W + 32
// At W = 128 the folded hidden/head biases would cost a third 64-column
// K-chunk per layer and the image would not fit in shared memory, so there
// the hidden and head layers run at K = W and their biases are added in
// FP32 by the epilogue from a table at the end of the image; the image then
// fits (about 200 KB at H = 4) and two slots fill the 512 TMEM columns.
#include "internal.cuh"

namespace roam {

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }

// ---- shapes of the weight image ----
template <int W, int H>
struct TcShape {
    static constexpr bool kFold = W <= 64;     // hidden/head biases ride in the MMA
    static constexpr int N_HEAD = W + 16;
    static constexpr int K_COL = W + 32;
    static constexpr int K_HID = kFold ? W + 16 : W;
    static constexpr int N_OUT = 16;
    static constexpr int kSlots = W <= 64 ? 4 : 2;
    static constexpr int kLayers = H + 2;      // L1, hidden, head, colour (the 3-output layer runs on CUDA cores)
    __host__ __device__ static constexpr int K(int l) { return l == 0 ? 64 : (l == H + 1 ? K_COL : K_HID); }
    __host__ __device__ static constexpr int N(int l) { return l == H ? N_HEAD : W; }
    __host__ __device__ static constexpr int chunks(int l) { return cdiv(K(l), 64); }
    __host__ __device__ static constexpr int bytes(int l) { return chunks(l) * N(l) * 128; }
    __host__ __device__ static constexpr int offset(int l)
    {
        int o = 0;
        for (int i = 0; i < l; ++i) o += bytes(i);
        return o;
    }
    static constexpr int kMatBytes = offset(H + 2);
    // after the MMA operands: FP32 output layer, [W][4] (3 outputs + pad) then bias[4]
    static constexpr int kOutBytes = (4 * W + 4) * 4;
    // unfolded widths: FP32 biases of the hidden layers ((H-1) x W), then the
    // head's W features and its density logit, padded to 16 bytes
    static constexpr int kNTab = kFold ? 0 : (((H - 1) * W + W + 1 + 3) & ~3);
    static constexpr int kTabBytes = kNTab * 4;
    static constexpr int kImageBytes = kMatBytes + kOutBytes + kTabBytes;
    static constexpr int kImageAlloc = (kImageBytes + 1023) & ~1023;
    static constexpr int kXChunks = cdiv(K_COL, 64) > 1 ? cdiv(K_COL, 64) : 1;
    static constexpr int kXBytes = kXChunks * 128 * 128;
    static constexpr int kNBias = ((H - 1) * W + W + 1 + 3 + 3) & ~3;
    static constexpr int kTmemCols = N_HEAD <= 32 ? 32 : (N_HEAD <= 64 ? 64 : (N_HEAD <= 128 ? 128 : 256));
    // TMEM of one slot: accumulator D (N_HEAD columns), then the activations A
    // of the next MMA (K_COL BF16 per row, two per 32-bit column)
    static constexpr int kDCols = N_HEAD;
    static constexpr int kACols = K_COL / 2;
    static constexpr int kSlotCols = kDCols + kACols;
    static constexpr int kSmem = 1024 + kXBytes + kImageBytes + 64;
};

// byte offset of element (n, k) in a K-major, 128B-swizzled operand whose
// K-chunks of 64 elements are stored as consecutive [rows][128 B] regions
__host__ __device__ inline int swz_offset(int n, int k, int rows)
{
    const int chunk = k >> 6, kk = k & 63;
    return chunk * rows * 128 + (n >> 3) * 1024 + (n & 7) * 128 + ((((kk >> 3) ^ (n & 7)) & 7) << 4) + (kk & 7) * 2;
}

// ---- PTX wrappers ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// try_wait with a suspend-time hint: the warp sleeps in hardware until the
// phase completes (or ~20 us pass) instead of spinning on issue slots that
// the other slots' warps need
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `parity` to complete; gives up after kWaitNs or as
// soon as another thread has flagged an abort.  Returns false on give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint32_t *status, bool drain = false)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        {
            if (*abort_flag && !drain) return false;
            if (now_ns() - t0 > kWaitNs) {
                *abort_flag = 1;
                atomicOr(status, kStatusTimeout);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

// 8 consecutive BF16 columns [c8*8, c8*8+8) of row `row` of a swizzled X
__device__ __forceinline__ void st_x8(uint8_t *X, int row, int c8, uint4 v)
{
    const int chunk = c8 >> 3, cc = c8 & 7;
    uint8_t *p = X + chunk * 16384 + (row >> 3) * 1024 + (row & 7) * 128 + (((cc ^ (row & 7)) & 7) << 4);
    *reinterpret_cast<uint4 *>(p) = v;
}

__device__ __forceinline__ void st_x16(uint8_t *X, int row, int col, const float (&v)[16])
{
    uint4 a, b;
    a.x = pack_bf16(v[0], v[1]); a.y = pack_bf16(v[2], v[3]); a.z = pack_bf16(v[4], v[5]); a.w = pack_bf16(v[6], v[7]);
    b.x = pack_bf16(v[8], v[9]); b.y = pack_bf16(v[10], v[11]); b.z = pack_bf16(v[12], v[13]);
    b.w = pack_bf16(v[14], v[15]);
    st_x8(X, row, col >> 3, a);
    st_x8(X, row, (col >> 3) + 1, b);
}

// sin(pi y), cos(pi y) for |y| up to 2^9: exact reduction of y to
// r in [-1, 1] (y - 2 rint(y/2) is exact in FP32), then the hardware
// approximations on [-pi, pi] (absolute error < 1e-6).
__device__ __forceinline__ void sincospi_fast(float y, float &s, float &c)
{
    const float r = y - 2.0f * rintf(0.5f * y);
    __sincosf(3.14159265358979f * r, &s, &c);
}

// F(v) for one coordinate, frequencies 2^0 .. 2^(L-1): direct evaluation at
// k = 0 and k = 5, angle doubling (sin 2a = 2 sin a cos a,
// cos 2a = 1 - 2 sin^2 a) in between, so the doubling error stays below
// 2^4 times the direct error.
template <int L>
__device__ __forceinline__ void encode1(float v, float (&s)[L], float (&c)[L])
{
#pragma unroll
    for (int k = 0; k < L; ++k) {
        if (k == 0 || k == 5) {
            sincospi_fast(ldexpf(v, k), s[k], c[k]);
        } else {
            const float sp = s[k - 1], cp = c[k - 1];
            s[k] = 2.0f * sp * cp;
            c[k] = fmaf(-2.0f * sp, sp, 1.0f);
        }
    }
}

__device__ __forceinline__ float softplus_f(float s) { return s > 20.f ? s : log1pf(__expf(s)); }
__device__ __forceinline__ float sigmoid_f(float s) { return 1.f / (1.f + __expf(-s)); }

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D (TMEM) [+]= A (TMEM, 128 lanes x K/2 columns of BF16 pairs) * B (SMEM descriptor)
__device__ __forceinline__ void umma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// 32 floats -> 16 BF16 pairs (element 2c in the low half of column c)
__device__ __forceinline__ void pack16(const float *v, uint32_t (&o)[16])
{
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q] = pack_bf16(v[2 * q], v[2 * q + 1]);
}

__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b)
{
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

// Named barrier over n threads that also ORs a flag across them: every
// participant gets the same answer, so an abort leaves all of them together.
__device__ __forceinline__ bool named_sync_or(int id, int n, bool flag)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %3, 0;\n\t"
        "bar.red.or.pred q, %1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(id), "r"(n), "r"((uint32_t)flag)
        : "memory");
    return r != 0;
}

// 16 accumulator columns -> 16 BF16 X columns (two 16-byte chunks)
template <bool kRelu>
__device__ __forceinline__ void st_x16_bits(uint8_t *X, int row, int col, const uint32_t (&r)[16])
{
    uint4 a, b;
    if (kRelu) {
        a.x = pack_bf16_relu(__uint_as_float(r[0]), __uint_as_float(r[1]));
        a.y = pack_bf16_relu(__uint_as_float(r[2]), __uint_as_float(r[3]));
        a.z = pack_bf16_relu(__uint_as_float(r[4]), __uint_as_float(r[5]));
        a.w = pack_bf16_relu(__uint_as_float(r[6]), __uint_as_float(r[7]));
        b.x = pack_bf16_relu(__uint_as_float(r[8]), __uint_as_float(r[9]));
        b.y = pack_bf16_relu(__uint_as_float(r[10]), __uint_as_float(r[11]));
        b.z = pack_bf16_relu(__uint_as_float(r[12]), __uint_as_float(r[13]));
        b.w = pack_bf16_relu(__uint_as_float(r[14]), __uint_as_float(r[15]));
    } else {
        a.x = pack_bf16(__uint_as_float(r[0]), __uint_as_float(r[1]));
        a.y = pack_bf16(__uint_as_float(r[2]), __uint_as_float(r[3]));
        a.z = pack_bf16(__uint_as_float(r[4]), __uint_as_float(r[5]));
        a.w = pack_bf16(__uint_as_float(r[6]), __uint_as_float(r[7]));
        b.x = pack_bf16(__uint_as_float(r[8]), __uint_as_float(r[9]));
        b.y = pack_bf16(__uint_as_float(r[10]), __uint_as_float(r[11]));
        b.z = pack_bf16(__uint_as_float(r[12]), __uint_as_float(r[13]));
        b.w = pack_bf16(__uint_as_float(r[14]), __uint_as_float(r[15]));
    }
    st_x8(X, row, col >> 3, a);
    st_x8(X, row, (col >> 3) + 1, b);
}

// Everything the encoding of one sample needs, fetched a tile ahead.
struct SampleIn {
    uint32_t idx;
    float px, py, pz, dx, dy, dz;
};

__device__ __forceinline__ SampleIn fetch_sample(const SampleSrc &src, const BucketBufs &b, const Tile &tl, int row)
{
    SampleIn r{0u, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    if ((uint32_t)row >= tl.count) return r;
    r.idx = b.sorted[tl.start + row];
    if (src.mode == 0) {
        const uint32_t col = r.idx >> 5;
        const uint32_t i = (col / (uint32_t)src.R) * 32u + (r.idx & 31u);
        const uint32_t ray = src.live ? src.live[i] : i;
        const uint32_t j = src.recs[r.idx] & 0xffffu;
        const float tt = ((float)j + 0.5f) * src.delta;
        const float4 o = src.st.orig[ray], d = src.st.dir[ray];
        r.px = fmaf(tt, d.x, o.x); r.py = fmaf(tt, d.y, o.y); r.pz = fmaf(tt, d.z, o.z);
        r.dx = d.x; r.dy = d.y; r.dz = d.z;
    } else {
        r.px = src.p[3 * (int64_t)r.idx]; r.py = src.p[3 * (int64_t)r.idx + 1]; r.pz = src.p[3 * (int64_t)r.idx + 2];
        r.dx = src.d[3 * (int64_t)r.idx]; r.dy = src.d[3 * (int64_t)r.idx + 1]; r.dz = src.d[3 * (int64_t)r.idx + 2];
    }
    return r;
}

// Persistent kernel, one CTA per SM, kSlots tiles in flight.  Slot s is
// warpgroup s: its 128 threads encode and run the epilogues of their tile
// (one row each), and its first thread issues the tile's MMAs itself --
// tcgen05.mma and tcgen05.commit occupy the issuing thread for tens to
// hundreds of cycles each, so one issuer per slot lets the slots' chains
// overlap.  Tiles come in field-uniform groups of kSlots (bucket padding);
// at a field change all slots meet at a CTA barrier, thread 0 reloads the
// shared weight image, and each issuer waits for it before its next MMA.
template <int W, int H, int kSlots>
__global__ void __launch_bounds__(kSlots * 128, 1)
    k_mlp_tc(MlpWeights w, SampleSrc src, BucketBufs b, Counters *ctr, float4 *out)
{
    using S = TcShape<W, H>;
    constexpr int kLayers = S::kLayers;
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
    const bool issuer = (threadIdx.x & 127) == 0;
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

    const uint32_t n_groups = ctr->n_tiles / kSlots;
    const uint32_t g0 = (uint32_t)((uint64_t)n_groups * blockIdx.x / gridDim.x);
    const uint32_t g1 = (uint32_t)((uint64_t)n_groups * (blockIdx.x + 1) / gridDim.x);

    uint32_t d_ph = 0, n_changes = 0, n_commits = 0, n_waits = 0;
    uint32_t cur_field = 0xffffffffu;
    bool w_ready = false, w_waited_last = true;
    bool img_seen = false;     // this thread has waited for the current image (before generic loads of it)
    bool aborted = false;
    const float sig_scale = w.sigma_scale;
    Tile tl{0u, 0u, 0u, 0u};
    SampleIn nxt{0u, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    uint32_t g = g0;
    if (g < g1) {
        tl = b.tiles[g * kSlots + slot];
        nxt = fetch_sample(src, b, tl, row);
    }
    for (; g < g1; ++g) {
        const uint32_t f = tl.field;           // identical for every slot (field-uniform groups)
        if (f != cur_field) {
            // every slot has waited on its last layer, so no MMA reads the old
            // image; meet (and agree on any abort), reload, issuers wait below
            if (named_sync_or(15, kSlots * 128, aborted || *abortp)) break;
            if (threadIdx.x == 0) {
                mbar_expect_tx(&bar_w, (uint32_t)S::kImageBytes);
                const uint8_t *gsrc = reinterpret_cast<const uint8_t *>(w.wimg) + (int64_t)f * w.img_bytes;
                for (int off = 0; off < S::kImageBytes; off += 16384) {
                    const int nb = S::kImageBytes - off < 16384 ? S::kImageBytes - off : 16384;
                    bulk_g2s(IMG + off, gsrc + off, (uint32_t)nb, &bar_w);
                }
                w_waited_last = false;
            }
            ++n_changes;
            cur_field = f;
            w_ready = false;
            img_seen = false;
        }
        const Tile cur = tl;
        const SampleIn sm = nxt;
        if (g + 1 < g1) tl = b.tiles[(g + 1) * kSlots + slot];
        if (cur.count == 0 || aborted) {
            if (g + 1 < g1) nxt = fetch_sample(src, b, tl, row);
            continue;
        }
        const bool valid = (uint32_t)row < cur.count;
        const float *aff = w.affine + 6 * (int64_t)cur.field;
        // ---- L1 input: [F(x_loc) | 1] ----
        {
            const float xl[3] = {fmaf(__ldg(aff + 0), sm.px, __ldg(aff + 3)), fmaf(__ldg(aff + 1), sm.py, __ldg(aff + 4)),
                                 fmaf(__ldg(aff + 2), sm.pz, __ldg(aff + 5))};
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
            if (!valid) {
#pragma unroll
                for (int q = 0; q < 64; ++q) e[q] = 0.f;
            }
            uint32_t pk[16];
            pack16(e, pk);
            tmem_st16(tArow, pk);
            pack16(e + 32, pk);
            tmem_st16(tArow + 16, pk);
        }
        // the next tile's gathers overlap this tile's layers
        if (g + 1 < g1) nxt = fetch_sample(src, b, tl, row);
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
                    ok = mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status);
                    w_ready = ok;
                    if (threadIdx.x == 0) w_waited_last = ok;
                }
                if (ok) {
                    tc_fence_after();
                    const int K = S::K(l), N = S::N(l);
                    const uint32_t idesc = idesc_bf16(N);
                    const uint32_t ba = imga + S::offset(l);
#pragma unroll 1
                    for (int ks = 0; ks < K / 16; ++ks) {
                        const int ch = ks >> 2, kin = ks & 3;
                        umma_ta(tslot, tA + (uint32_t)(ks * 8), sdesc(ba + ch * N * 128 + kin * 32), idesc,
                                ks > 0 ? 1u : 0u);
                    }
                }
                umma_commit(&bar_d[slot]);
                ++n_commits;
            }
            const bool got = mbar_wait(&bar_d[slot], d_ph, abortp, status);
            if (issuer && got) ++n_waits;
            d_ph ^= 1u;
            // tcgen05.ld is warp-collective: the warp decides together; the
            // slot decides together at the next barrier
            if (!__all_sync(0xffffffffu, got)) {
                aborted = true;
                continue;
            }
            tc_fence_after();
            uint32_t r[W / 16][16];
#pragma unroll
            for (int c = 0; c < W / 16; ++c) tmem_ld16_nowait(trow + 16 * c, r[c]);
            uint32_t rs[16];
            if (l == H) tmem_ld16_nowait(trow + W, rs);
            tmem_wait_ld();
            tc_fence_before();
            const float *btab = reinterpret_cast<const float *>(IMG + S::kMatBytes + S::kOutBytes) + (l >= 1 ? l - 1 : 0) * W;
            if constexpr (!S::kFold) {
                if (l >= 1 && !img_seen) {
                    mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status);
                    img_seen = true;
                }
            }
            if (l < H + 1) {
                // next activations: head features stay linear, every other layer ReLU
#pragma unroll
                for (int c = 0; c < W / 32; ++c) {
                    float bv[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) bv[q] = 0.f;
                    if constexpr (!S::kFold) {
                        if (l >= 1) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 t = reinterpret_cast<const float4 *>(btab + 32 * c)[q];
                                bv[4 * q] = t.x; bv[4 * q + 1] = t.y; bv[4 * q + 2] = t.z; bv[4 * q + 3] = t.w;
                            }
                        }
                    }
                    uint32_t v16[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int e0 = 32 * c + 2 * q;
                        const float a0 = __uint_as_float(r[e0 >> 4][e0 & 15]) + bv[2 * q];
                        const float a1 = __uint_as_float(r[(e0 + 1) >> 4][(e0 + 1) & 15]) + bv[2 * q + 1];
                        v16[q] = l == H ? pack_bf16(a0, a1) : pack_bf16_relu(a0, a1);
                    }
                    tmem_st16(tArow + 16 * c, v16);
                }
                if (l == H) {
                    // density from column W of the head
                    float sl = __uint_as_float(rs[0]);
                    if constexpr (!S::kFold) sl += btab[W];
                    sigma = sig_scale * (w.act == ROAM_RELU ? fmaxf(sl, 0.f) : softplus_f(sl));
                }
                if (l == 0) {
                    // tail of X from here on: [1 | F(d) | 0 0 0 0] at columns W .. W+31
                    float e[32];
                    e[0] = valid ? 1.0f : 0.0f;
                    const float dv[3] = {sm.dx, sm.dy, sm.dz};
                    e[1] = dv[0]; e[2] = dv[1]; e[3] = dv[2];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float sn[4], cs[4];
                        encode1<4>(dv[a], sn, cs);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            e[4 + 6 * k + a] = sn[k];
                            e[7 + 6 * k + a] = cs[k];
                        }
                    }
                    e[28] = e[29] = e[30] = e[31] = 0.f;
                    uint32_t pt[16];
                    pack16(e, pt);
                    tmem_st16(tArow + W / 2, pt);
                }
            } else {
                // colour layer: g = relu(z) in FP32, then rgb = sigmoid(Wo g + bo) with
                // the FP32 output table at the end of the shared image (this thread
                // waits for the image itself before reading it with generic loads)
                if (!img_seen) {
                    mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status);
                    img_seen = true;
                }
                const float4 *wo = reinterpret_cast<const float4 *>(IMG + S::kMatBytes);
                float4 acc = wo[W];
#pragma unroll
                for (int c = 0; c < W / 16; ++c) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float gk = fmaxf(__uint_as_float(r[c][q]), 0.f);
                        const float4 wk = wo[16 * c + q];
                        acc.x = fmaf(wk.x, gk, acc.x);
                        acc.y = fmaf(wk.y, gk, acc.y);
                        acc.z = fmaf(wk.z, gk, acc.z);
                    }
                }
                if (valid) out[sm.idx] = make_float4(sigma, sigmoid_f(acc.x), sigmoid_f(acc.y), sigmoid_f(acc.z));
            }
        }
    }
    // drain before TMEM is freed and the CTA exits: a commit whose wait gave
    // up, and an image load nobody waited for
    if (issuer && n_commits > n_waits) mbar_wait(&bar_d[slot], (n_commits - 1) & 1u, abortp, status, true);
    if (threadIdx.x == 0 && !w_waited_last) mbar_wait(&bar_w, (n_changes - 1) & 1u, abortp, status, true);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemAlloc)
                     : "memory");
    }
}

// API layout -> BF16 image of every layer + FP32 bias table.
template <int W, int H>
__global__ void k_pack_tc(const float *__restrict__ w32, int n_fields, int64_t P, uint8_t *__restrict__ img,
                          int64_t img_bytes, float *__restrict__ bias, int nb)
{
    using S = TcShape<W, H>;
    // offsets of the API layout
    const int64_t o_l1 = 0, o_hid = (int64_t)W * kPeX + W;
    const int64_t o_head = o_hid + (int64_t)(H - 1) * (W * W + W);
    const int64_t o_col = o_head + (int64_t)(1 + W) * W + (1 + W);
    const int64_t o_out = o_col + (int64_t)W * (W + kPeD) + W;
    const int64_t per = S::kMatBytes / 2;        // BF16 elements of the MMA operands per field
    const int64_t n = (int64_t)n_fields * per;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = g / per;
        const int byte = (int)((g % per) * 2);
        // find the layer and (n, k) of this byte
        int l = 0;
        while (l + 1 < S::kLayers && byte >= S::offset(l + 1)) ++l;
        const int lb = byte - S::offset(l);
        const int N = S::N(l), K = S::K(l);
        const int chunk = lb / (N * 128);
        const int in_chunk = lb % (N * 128);
        const int nrow = (in_chunk / 1024) * 8 + (in_chunk % 1024) / 128;
        const int sw16 = (in_chunk % 128) / 16;
        const int k8 = (sw16 ^ (nrow & 7)) & 7;
        const int k = chunk * 64 + k8 * 8 + (in_chunk % 16) / 2;
        const float *wf = w32 + f * P;
        float v = 0.f;
        if (k < K) {
            if (l == 0) {
                if (k < kPeX) v = wf[o_l1 + (int64_t)nrow * kPeX + k];
                else if (k == kPeX) v = wf[o_l1 + (int64_t)W * kPeX + nrow];
            } else if (l < H) {
                const int64_t ob = o_hid + (int64_t)(l - 1) * (W * W + W);
                if (k < W) v = wf[ob + (int64_t)nrow * W + k];
                else if (k == W) v = wf[ob + (int64_t)W * W + nrow];
            } else if (l == H) {
                // rows: W features (API rows 1..W), then the density logit (API row 0)
                const int ar = nrow < W ? 1 + nrow : (nrow == W ? 0 : -1);
                if (ar >= 0) {
                    if (k < W) v = wf[o_head + (int64_t)ar * W + k];
                    else if (k == W) v = wf[o_head + (int64_t)(1 + W) * W + ar];
                }
            } else if (l == H + 1) {
                const int kc = W + kPeD;
                if (k < W) v = wf[o_col + (int64_t)nrow * kc + k];
                else if (k == W) v = wf[o_col + (int64_t)W * kc + nrow];
                else if (k <= W + kPeD) v = wf[o_col + (int64_t)nrow * kc + (k - 1)];
            }
        }
        const uint32_t bits = __float_as_uint(v);
        // round to nearest even
        const uint32_t r = bits + 0x7fffu + ((bits >> 16) & 1u);
        reinterpret_cast<uint16_t *>(img + f * img_bytes)[g % per] = (uint16_t)(r >> 16);
    }
    // FP32 output layer after the operands: [W][4] (weights of the 3 colours, pad 0), then bias[4]
    const int nout = 4 * W + 4;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < (int64_t)n_fields * nout;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = gi / nout;
        const int q = (int)(gi % nout);
        const float *wf = w32 + f * P;
        float v = 0.f;
        if (q < 4 * W) {
            const int k = q / 4, c = q % 4;
            if (c < 3) v = wf[o_out + (int64_t)c * W + k];
        } else if (q - 4 * W < 3) {
            v = wf[o_out + 3 * W + (q - 4 * W)];
        }
        reinterpret_cast<float *>(img + f * img_bytes + S::kMatBytes)[q] = v;
    }
    // unfolded widths: the FP32 bias table of the hidden and head layers
    if (S::kNTab > 0) {
        for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < (int64_t)n_fields * S::kNTab;
             gi += (int64_t)gridDim.x * blockDim.x) {
            const int64_t f = gi / S::kNTab;
            const int q = (int)(gi % S::kNTab);
            const float *wf = w32 + f * P;
            float v = 0.f;
            if (q < (H - 1) * W) v = wf[o_hid + (int64_t)(q / W) * (W * W + W) + (int64_t)W * W + q % W];
            else if (q < H * W) v = wf[o_head + (int64_t)(1 + W) * W + 1 + (q - (H - 1) * W)];
            else if (q == H * W) v = wf[o_head + (int64_t)(1 + W) * W];
            reinterpret_cast<float *>(img + f * img_bytes + S::kMatBytes + S::kOutBytes)[q] = v;
        }
    }
    // bias table: hidden (H-1)*W, head features W, head density 1, output 3
    const int64_t nbt = (int64_t)n_fields * nb;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nbt; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = g / nb;
        const int q = (int)(g % nb);
        const float *wf = w32 + f * P;
        float v = 0.f;
        if (q < (H - 1) * W) {
            const int l = q / W, o = q % W;
            v = wf[o_hid + (int64_t)l * (W * W + W) + (int64_t)W * W + o];
        } else if (q < (H - 1) * W + W) {
            v = wf[o_head + (int64_t)(1 + W) * W + 1 + (q - (H - 1) * W)];
        } else if (q == (H - 1) * W + W) {
            v = wf[o_head + (int64_t)(1 + W) * W];
        } else if (q < (H - 1) * W + W + 4) {
            v = wf[o_out + 3 * W + (q - (H - 1) * W - W - 1)];
        }
        bias[g] = v;
    }
}

template <int W, int H>
int tc_smem_bytes() { return 1024 + TcShape<W, H>::kImageAlloc; }

template <int W, int H>
void launch_t(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, float4 *out, int n_sm,
              cudaStream_t s)
{
    constexpr int kSlots = TcShape<W, H>::kSlots;
    const int smem = tc_smem_bytes<W, H>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_tc<W, H, kSlots>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    k_mlp_tc<W, H, kSlots><<<n_sm, kSlots * 128, smem, s>>>(w, src, b, ctr, out);
}

#define ROAM_TC_CASES                                                                                   \
    ROAM_CASE(32, 1) ROAM_CASE(32, 2) ROAM_CASE(32, 3) ROAM_CASE(32, 4) ROAM_CASE(64, 1) ROAM_CASE(64, 2) \
    ROAM_CASE(64, 3) ROAM_CASE(64, 4) ROAM_CASE(128, 1) ROAM_CASE(128, 2) ROAM_CASE(128, 3) ROAM_CASE(128, 4)

}  // namespace

bool tc_supported(int W, int H)
{
    if (H < 1 || H > 4) return false;
#define ROAM_CASE(WW, HH) \
    if (W == WW && H == HH) return tc_smem_bytes<WW, HH>() <= 227 * 1024;
    ROAM_TC_CASES
#undef ROAM_CASE
    return false;
}

int64_t tc_image_bytes(int W, int H)
{
#define ROAM_CASE(WW, HH) \
    if (W == WW && H == HH) return TcShape<WW, HH>::kImageBytes;
    ROAM_TC_CASES
#undef ROAM_CASE
    return 0;
}

int tc_bias_count(int W, int H) { return ((H - 1) * W + W + 1 + 3 + 3) & ~3; }

int tc_tile_samples() { return 128; }

int tc_tile_group(int W) { return W <= 64 ? TcShape<64, 1>::kSlots : TcShape<128, 1>::kSlots; }

void launch_pack_tc(const float *w32, int n_fields, int W, int H, int64_t P, void *wimg, int64_t img_bytes,
                    float *bias, int nb, cudaStream_t s)
{
#define ROAM_CASE(WW, HH) \
    if (W == WW && H == HH) { k_pack_tc<WW, HH><<<2048, 256, 0, s>>>(w32, n_fields, P, (uint8_t *)wimg, img_bytes, bias, nb); return; }
    ROAM_TC_CASES
#undef ROAM_CASE
}

void launch_mlp_tc(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, float4 *out,
                   int n_sm, cudaStream_t s)
{
#define ROAM_CASE(WW, HH) \
    if (w.W == WW && w.H == HH) { launch_t<WW, HH>(w, src, b, ctr, out, n_sm, s); return; }
    ROAM_TC_CASES
#undef ROAM_CASE
}

}  // namespace roam
