// Shared pieces of the tcgen05 MLP kernels (forward evaluation and the
// adjoint): the weight-image shapes, PTX wrappers for mbarriers, bulk
// copies, tcgen05 MMAs and TMEM access, BF16/E4M3 packing, the positional
// encoding and the per-sample gathers.  Everything sits in an anonymous
// namespace: each kernel file gets its own copy.
#pragma once

#include "internal.cuh"

namespace roam {

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }

// ---- shapes of the weight image ----
template <int W, int H, bool F8>
struct TcShape {
    static constexpr bool kFold = !F8 && W <= 64;    // hidden/head biases ride in the MMA
    static constexpr bool kTab = !kFold;             // FP32 per-layer scale/bias table in the image
    static constexpr int kEB = F8 ? 1 : 2;           // bytes per operand element
    static constexpr int kCE = 128 / kEB;            // K elements per 128-byte swizzle row (one chunk)
    static constexpr int kKS = 32 / kEB;             // K of one MMA instruction (32 bytes)
    static constexpr int N_HEAD = W + 16;
    static constexpr int K_COL = W + 32;
    static constexpr int K_HID = kFold ? W + 16 : W;
    static constexpr int kLayers = H + 2;      // L1, hidden, head, colour (the 3-output layer runs on CUDA cores)
    __host__ __device__ static constexpr int K(int l) { return l == 0 ? 64 : (l == H + 1 ? K_COL : K_HID); }
    __host__ __device__ static constexpr int N(int l) { return l == H ? N_HEAD : W; }
    __host__ __device__ static constexpr int chunks(int l) { return cdiv(K(l), kCE); }
    __host__ __device__ static constexpr int bytes(int l) { return chunks(l) * N(l) * 128; }
    __host__ __device__ static constexpr int offset(int l)
    {
        int o = 0;
        for (int i = 0; i < l; ++i) o += bytes(i);
        return o;
    }
    static constexpr int kMatBytes = offset(H + 2);
    // after the MMA operands: FP32 output layer, [4][W] (the 3 outputs' weight
    // rows over k, then a zero row: float4 loads along k) then bias[4]
    static constexpr int kOutBytes = (4 * W + 4) * 4;
    // then (kTab) per layer l: scale[kTabStride] and bias[kTabStride]; the
    // head's entry W is its density logit
    static constexpr int kTabStride = W + 4;
    static constexpr int kNTab = kTab ? kLayers * 2 * kTabStride : 0;
    static constexpr int kImageBytes = kMatBytes + kOutBytes + kNTab * 4;
    static constexpr int kImageAlloc = (kImageBytes + 1023) & ~1023;
    // TMEM of one slot: accumulator D (N_HEAD columns), then the activations A
    // of the next MMA (K_COL elements per row, 4 / kEB per 32-bit column)
    static constexpr int kDCols = N_HEAD;
    static constexpr int kACols = K_COL * kEB / 4;
    static constexpr int kSlotCols = kDCols + kACols;
    static constexpr int kSlots = 512 / kSlotCols >= 4 ? 4 : (512 / kSlotCols >= 2 ? 2 : 1);
};

// ---- PTX wrappers ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
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

// Waits for the phase of `parity` to complete; gives up after limit_ns or as
// soon as another thread has flagged an abort (a drain wait ignores the
// flag).  Returns false on give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint32_t *status, bool drain = false,
                                          unsigned long long limit_ns = kWaitNs)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag && !drain) return false;
        if (now_ns() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}

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

// instruction descriptors, D = F32, A and B K-major, M = 128:
// kind::f16 with A = B = BF16 (format 1); kind::f8f6f4 with A = B = E4M3 (format 0)
__host__ __device__ constexpr uint32_t idesc_bf16(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__host__ __device__ constexpr uint32_t idesc_e4m3(int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// D (TMEM) [+]= A (TMEM, 128 lanes, packed operand elements) * B (SMEM descriptor)
template <bool F8>
__device__ __forceinline__ void umma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if constexpr (F8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

// One layer's K loop with A in TMEM, fully unrolled: the B descriptor is
// built once and stepped by compile-time offsets (its 14-bit start-address
// field, in 16-byte units, cannot carry: every operand lies inside the CTA's
// shared memory).  A descriptor rebuilt for every instruction triples the
// issue time of an N <= 64 MMA (about 80 against 25 ns on GB300), which
// then bounds the whole chain.
template <bool F8, int K, int N>
__device__ __forceinline__ void umma_chain_ta(uint32_t d_tmem, uint32_t a_tmem, uint32_t b_saddr)
{
    constexpr int kKS = F8 ? 32 : 16;                // K of one MMA (32 bytes)
    constexpr uint32_t idesc = F8 ? idesc_e4m3(N) : idesc_bf16(N);
    static_assert(K % kKS == 0, "whole MMAs");
    const uint64_t db = sdesc(b_saddr);
#pragma unroll
    for (int ks = 0; ks < K / kKS; ++ks)
        umma_ta<F8>(d_tmem, a_tmem + (uint32_t)(ks * 8),
                    db + (uint64_t)(((ks >> 2) * N * 128 + (ks & 3) * 32) >> 4), idesc, ks > 0 ? 1u : 0u);
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

// 32 consecutive 32-bit TMEM columns of this thread's lane, one instruction
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 (8) consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// element 2c in the low half of 32-bit column c
__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

// element 4c + i in byte i of 32-bit column c; round to nearest even,
// magnitudes beyond 448 saturate
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d)
{
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(lo) : "f"(a), "f"(b));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(hi) : "f"(c), "f"(d));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b)
{
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

// Writes 32 activation values (elements [32c, 32c + 32) of A) to TMEM,
// through a ReLU when kRelu (fused into the BF16 conversion).
template <bool F8, bool kRelu>
__device__ __forceinline__ void st_act32(uint32_t tArow, int c, const float (&v)[32])
{
    if constexpr (F8) {
        uint32_t o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float a0 = kRelu ? fmaxf(v[4 * q], 0.f) : v[4 * q];
            const float a1 = kRelu ? fmaxf(v[4 * q + 1], 0.f) : v[4 * q + 1];
            const float a2 = kRelu ? fmaxf(v[4 * q + 2], 0.f) : v[4 * q + 2];
            const float a3 = kRelu ? fmaxf(v[4 * q + 3], 0.f) : v[4 * q + 3];
            o[q] = pack_e4m3x4(a0, a1, a2, a3);
        }
        tmem_st8(tArow + 8 * c, o);
    } else {
        uint32_t o[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            o[q] = kRelu ? pack_bf16_relu(v[2 * q], v[2 * q + 1]) : pack_bf16(v[2 * q], v[2 * q + 1]);
        tmem_st16(tArow + 16 * c, o);
    }
}

// sin(pi y), cos(pi y) for |y| up to 2^9: exact reduction of y to
// r in [-1, 1] (y - 2 rint(y/2) is exact in FP32), then the hardware
// approximations on [-pi, pi] (absolute error < 1e-6).
__device__ __forceinline__ void sincospi_fast(float y, float &s, float &c)
{
    const float r = y - 2.0f * rintf(0.5f * y);
    __sincosf(3.14159265358979f * r, &s, &c);
}

// Packs e[first .. first + n) into the MMA's A words (BF16: elements 2c and
// 2c + 1 in word c, low half first; E4M3: elements 4c .. 4c + 3 in word c);
// the words whose elements all lie in that range.
template <bool F8, int NW>
__device__ __forceinline__ void pack_range(const float *e, uint32_t (&w)[NW], int first, int n)
{
    constexpr int per = F8 ? 4 : 2;
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        if (c * per < first || c * per + per > first + n) continue;
        if constexpr (F8) w[c] = pack_e4m3x4(e[4 * c], e[4 * c + 1], e[4 * c + 2], e[4 * c + 3]);
        else w[c] = pack_bf16(e[2 * c], e[2 * c + 1]);
    }
}

// A block of the encoding F(v) = [v, sin(2^k pi v), cos(2^k pi v)] (k < L,
// three sines then three cosines per k), frequency after frequency so that
// each word is packed as soon as its elements exist (few live registers).
// Layout: `lead` leading constant-1 elements, then F(v) (3 + 6 L), then
// `trail_one` constant 1, then zeros up to 32 * NB elements.
template <bool F8, int L, int kLead, bool kTrailOne, int NE>
__device__ __forceinline__ void encode_packed(const float (&v)[3], uint32_t (&w)[F8 ? NE / 4 : NE / 2])
{
    constexpr int NW = F8 ? NE / 4 : NE / 2;
    float e[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) e[q] = 0.f;
#pragma unroll
    for (int q = 0; q < kLead; ++q) e[q] = 1.0f;
    e[kLead] = v[0]; e[kLead + 1] = v[1]; e[kLead + 2] = v[2];
    if (kTrailOne) e[kLead + 3 + 6 * L] = 1.0f;
    // (x, y) as packed pairs (each half rounded as the scalar operation), z alone
    float2 s01 = make_float2(0.f, 0.f), c01 = s01;
    float s2 = 0.f, c2 = 0.f;
#pragma unroll
    for (int k = 0; k < L; ++k) {
        // direct evaluation at k = 0 and k = 5, angle doubling in between
        if (k == 0 || k == 5) {
            sincospi_fast(v[0] * (float)(1 << k), s01.x, c01.x);
            sincospi_fast(v[1] * (float)(1 << k), s01.y, c01.y);
            sincospi_fast(v[2] * (float)(1 << k), s2, c2);
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
        e[kLead + 3 + 6 * k] = s01.x; e[kLead + 4 + 6 * k] = s01.y; e[kLead + 5 + 6 * k] = s2;
        e[kLead + 6 + 6 * k] = c01.x; e[kLead + 7 + 6 * k] = c01.y; e[kLead + 8 + 6 * k] = c2;
        pack_range<F8, NW>(e, w, 0, kLead + 9 + 6 * k);
    }
    pack_range<F8, NW>(e, w, 0, NE);
}

// log(1 + e^s) and 1 / (1 + e^-s) with the hardware exp2/log2 and the fast
// division (a few units of 2^-22 absolute: far inside the BF16/FP8 outputs'
// rounding); softplus(s) = s past s = 15 (the difference is below 4e-7)
__device__ __forceinline__ float softplus_f(float s) { return s > 15.f ? s : __logf(1.f + __expf(s)); }
__device__ __forceinline__ float sigmoid_f(float s) { return __fdividef(1.f, 1.f + __expf(-s)); }

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

// Everything the encoding of one sample needs, fetched a tile ahead.
struct SampleIn {
    uint32_t idx;
    float px, py, pz, dx, dy, dz;
};

// The next tile's sample, gathered in stages spread over this tile's layers
// (sorted index -> record and ray -> ray origin and direction), so that no
// stage waits on the previous one's load.
struct Pending {
    bool on;
    uint32_t idx, rec, ray;
    float4 o, d;
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

__device__ __forceinline__ void stage_index(Pending &q, const BucketBufs &b, const Tile &tl, int row, bool more)
{
    q.on = more && (uint32_t)row < tl.count;
    if (q.on) q.idx = b.sorted[tl.start + row];
}

__device__ __forceinline__ void stage_record(Pending &q, const SampleSrc &src)
{
    if (!q.on || src.mode != 0) return;
    const uint32_t col = q.idx >> 5;
    const uint32_t i = (col / (uint32_t)src.R) * 32u + (q.idx & 31u);
    q.rec = src.recs[q.idx];
    q.ray = src.live ? src.live[i] : i;
}

__device__ __forceinline__ void stage_ray(Pending &q, const SampleSrc &src)
{
    if (!q.on) return;
    if (src.mode == 0) {
        q.o = src.st.orig[q.ray];
        q.d = src.st.dir[q.ray];
    } else {
        const int64_t k = 3 * (int64_t)q.idx;
        q.o = make_float4(src.p[k], src.p[k + 1], src.p[k + 2], 0.f);
        q.d = make_float4(src.d[k], src.d[k + 1], src.d[k + 2], 0.f);
    }
}

__device__ __forceinline__ SampleIn stage_finish(const Pending &q, const SampleSrc &src)
{
    SampleIn r{0u, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    if (!q.on) return r;
    r.idx = q.idx;
    if (src.mode == 0) {
        const float tt = ((float)(q.rec & 0xffffu) + 0.5f) * src.delta;
        r.px = fmaf(tt, q.d.x, q.o.x); r.py = fmaf(tt, q.d.y, q.o.y); r.pz = fmaf(tt, q.d.z, q.o.z);
    } else {
        r.px = q.o.x; r.py = q.o.y; r.pz = q.o.z;
    }
    r.dx = q.d.x; r.dy = q.d.y; r.dz = q.d.z;
    return r;
}

// MN-major, 128-byte swizzle: 64-element MN blocks `lbo` bytes apart,
// 8-row K groups `sbo` bytes apart
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo = 1024u)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// kind::f16, D = F32, A = B = BF16, M = 128; a_mn / b_mn select the MN-major
// reading of A / B
__host__ __device__ constexpr uint32_t idesc_bf16_t(int N, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// kind::f16, D = F32, A = B = BF16, A K-major, any M (64 or 128); b_mn
// selects the MN-major reading of B
__host__ __device__ constexpr uint32_t idesc_bf16_m(int M, int N, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) [+]= A (SMEM descriptor) * B (SMEM descriptor)
__device__ __forceinline__ void umma_ss(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace

}  // namespace roam
