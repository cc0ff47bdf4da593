// The global 360NeRF (network table of the implementation details) as the
// distillation teacher of the local fields (Eq. 7): 8 fully connected layers
// of width 256 with F(x) concatenated to the input of layer 5, a density head
// (256 -> 1, ReLU), a feature head (256 -> 256, ReLU), a 128-wide colour
// layer on [feature; F(d)] (ReLU) and the 3-output layer (sigmoid).
//
// Two kernels of this file evaluate it:
//
// k_teacher_tc (BF16 operands, FP32 accumulation, tcgen05): a persistent
// kernel, one CTA per SM, one 128-point tile at a time.  The accumulator D
// (128 points x 256 outputs, FP32) and the next layer's input A (128 points x
// up to 320 BF16 features) live in TMEM; the weights stream from global
// memory (L2) through a ring of shared-memory stages, one 64-deep K-chunk of
// a layer (K = 64 x N = 256 BF16, 128-byte-swizzled K-major, 32 KB) per
// stage, copied by the bulk-copy (TMA) engine.  Warp roles:
//   warp 8     producer: one bulk copy per chunk into the next free stage;
//   warp 9     MMA issuer: per layer, waits for its input A, issues the
//              chunk's tcgen05.mma (M = 128, N = 256, K = 16 each) as its
//              stage lands, frees the stage with tcgen05.commit, and commits
//              the finished layer;
//   warps 0-7  epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its
//              points) and the output half w / 4 of D, adds the bias, applies
//              the activation, and writes the next layer's A with tcgen05.st;
//              they also encode F(x) and F(d), and form the density head and
//              the 3-output layer on the CUDA cores in FP32.
// A (element k of a point's row in 32-bit column k / 2 of the A region):
//   0 .. 255    the previous layer's output
//   256 .. 319  [F(d) (27) | 1 | 0 ...], read by layer 10 as its K 256 .. 287
//   320 .. 383  [F(x) (63) | 1], read by layer 1 and as layer 5's K 256 .. 319
// Layers 1, 5 and 10 take their bias through their constant-1 column; the
// other matrix layers add an FP32 bias in the epilogue.  The encodings use
// the accurate sincospif and are computed while the epilogue warps would
// otherwise wait for a layer's MMAs: the next tile's F(x) before layer 7's
// results (layer 5 has read the current one), its F(d) before layer 10's.
//
// k_teacher_simt (FP32): a plain SIMT evaluation for reference precision:
// a block of 256 threads takes 32 points, one output unit per thread, inputs
// in shared memory, weights read transposed ([K][N]) from global memory.
#include "tc_common.cuh"

namespace roam {

namespace {

constexpr int kTW = 256, kTC = 128;
constexpr int kTStages = 6;
constexpr int kTChunk = 32768;             // one stage: K = 64 x N = 256 BF16
constexpr int kTChunks = 39;               // weight chunks per tile (all layers)
constexpr int kTThreads = 320;             // 8 epilogue warps, producer, MMA issuer

// the API layers: 1-8, density head, feature head, 10, 11
constexpr int kTLayers = 12;
__host__ __device__ constexpr int t_out(int a)
{
    return a == 8 ? 1 : (a == 10 ? kTC : (a == 11 ? 3 : kTW));
}
__host__ __device__ constexpr int t_in(int a)
{
    return a == 0 ? kPeX : (a == 4 ? kTW + kPeX : (a == 10 ? kTW + kPeD : (a == 11 ? kTC : kTW)));
}
__host__ __device__ constexpr int64_t t_off(int a)
{
    int64_t o = 0;
    for (int i = 0; i < a; ++i) o += (int64_t)t_out(i) * t_in(i) + t_out(i);
    return o;
}

// ---- the tensor-core form -------------------------------------------------

// the ten matrix layers on the tensor cores: layers 1-8, the feature head,
// layer 10; their API layer, 64-deep K-chunks, N, first A column (32-bit
// TMEM columns), K-steps of 16, bias table (-1: folded) and ReLU
struct TcLayer {
    int api, chunks, N, a_col, ksteps, tab, relu;
};
constexpr int kColFd = 128, kColFx = 160;    // A columns of the F(d) and F(x) blocks
__host__ __device__ constexpr TcLayer tc_layer(int l)
{
    return l == 0   ? TcLayer{0, 1, kTW, kColFx, 4, -1, 1}
           : l <= 3 ? TcLayer{l, 4, kTW, 0, 16, l - 1, 1}
           : l == 4 ? TcLayer{4, 5, kTW, 0, 20, -1, 1}
           : l <= 7 ? TcLayer{l, 4, kTW, 0, 16, l - 2, l < 7 ? 1 : 0}
           : l == 8 ? TcLayer{9, 4, kTW, 0, 16, 6, 1}
                    : TcLayer{10, 5, kTC, 0, 18, -1, 1};
}
constexpr int kTcLayers = 10;

// A column of K-step ks of layer l: contiguous from a_col, except layer 5
// whose K 256 .. 319 is the F(x) block
__host__ __device__ constexpr int a_col_of(int l, int ks)
{
    return (l == 4 && ks >= 16) ? kColFx + (ks - 16) * 8 : tc_layer(l).a_col + ks * 8;
}

// the image: every chunk (N rows of 128 bytes) in layer order, then FP32
// tables: 7 biases x 256, density weights [256] and bias (4 floats), the
// 3-output layer as [128][4] (r, g, b, 0 per input) and its bias [4]
__host__ __device__ constexpr int64_t chunk_off(int c)
{
    int64_t o = 0;
    for (int l = 0, i = 0; l < kTcLayers; ++l)
        for (int k = 0; k < tc_layer(l).chunks; ++k, ++i) {
            if (i == c) return o;
            o += (int64_t)tc_layer(l).N * 128;
        }
    return o;
}
constexpr int64_t kTMatBytes = chunk_off(kTChunks);
constexpr int64_t kTTabOff = kTMatBytes;
constexpr int kTTabFloats = 7 * kTW + kTW + 4 + 4 * kTC + 4;
constexpr int64_t kTImageBytes = kTMatBytes + 4 * (int64_t)kTTabFloats;

// operand (n, k) of tensor-core layer l (B[k][n]), folded bias included
__device__ float tc_operand(const float *w, int l, int n, int k)
{
    const TcLayer L = tc_layer(l);
    const int a = L.api, K = t_in(a), N = t_out(a);
    if (n >= N) return 0.f;
    const float *Wa = w + t_off(a);
    if (k < K) return Wa[(int64_t)n * K + k];
    if (k == K && L.tab < 0) return Wa[(int64_t)N * K + n];
    return 0.f;
}

__global__ void k_teacher_pack_tc(const float *__restrict__ w, uint8_t *__restrict__ img)
{
    const int64_t n_el = kTMatBytes / 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t byte = 2 * e;
        int c = 0;
        while (c + 1 < kTChunks && chunk_off(c + 1) <= byte) ++c;
        int l = 0, first = 0;
        while (first + tc_layer(l).chunks <= c) first += tc_layer(l++).chunks;
        const int kc = c - first;
        const int in_chunk = (int)(byte - chunk_off(c));
        const int n = (in_chunk / 1024) * 8 + (in_chunk % 1024) / 128;
        const int u = (((in_chunk % 128) / 16) ^ (n & 7)) & 7;       // 16-byte unit before the swizzle
        const int k = kc * 64 + u * 8 + (in_chunk % 16) / 2;
        const float v = tc_operand(w, l, n, k);
        const uint32_t bits = __float_as_uint(v);
        reinterpret_cast<uint16_t *>(img)[e] = (uint16_t)((bits + 0x7fffu + ((bits >> 16) & 1u)) >> 16);
    }
    float *tab = reinterpret_cast<float *>(img + kTTabOff);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kTTabFloats; i += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < 7 * kTW) {
            const int t = i / kTW, n = i % kTW;
            const int a = t < 3 ? t + 1 : (t < 6 ? t + 2 : 9);          // layers 2-4, 6-8, feature head
            v = w[t_off(a) + (int64_t)kTW * kTW + n];
        } else if (i < 8 * kTW) {
            v = w[t_off(8) + (i - 7 * kTW)];                            // density weights
        } else if (i < 8 * kTW + 4) {
            v = i == 8 * kTW ? w[t_off(8) + kTW] : 0.f;                 // density bias
        } else if (i < 8 * kTW + 4 + 4 * kTC) {
            const int q = i - (8 * kTW + 4), k = q / 4, ch = q % 4;
            v = ch < 3 ? w[t_off(11) + (int64_t)ch * kTC + k] : 0.f;    // layer 11, [k][r g b 0]
        } else {
            const int ch = i - (8 * kTW + 4 + 4 * kTC);
            v = ch < 3 ? w[t_off(11) + 3 * kTC + ch] : 0.f;
        }
        tab[i] = v;
    }
}

struct TcSmem {
    uint64_t full[kTStages], empty[kTStages];
    uint64_t d_full, a_full, drain;
    uint32_t tmem;
    int abort_flag;
    float red[2][128][4];          // the epilogue halves' partial sums (density, colour logits)
};

// F(x) (L = 10, 63 features) or F(d) (L = 4, 27 features) and the constant 1,
// zero padded to 64 values, packed to BF16 pairs (element 2c in the low half
// of word c); sin and cos of every frequency by the accurate sincospif
template <int L>
__device__ __forceinline__ void encode_block(const float (&x)[3], uint32_t (&w)[32])
{
    float e[64];
    e[0] = x[0]; e[1] = x[1]; e[2] = x[2];
#pragma unroll
    for (int k = 0; k < L; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) sincospif(x[a] * (float)(1 << k), &e[3 + 6 * k + a], &e[6 + 6 * k + a]);
    constexpr int nf = 3 + 6 * L;
    e[nf] = 1.0f;
#pragma unroll
    for (int q = nf + 1; q < 64; ++q) e[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) w[q] = pack_bf16(e[2 * q], e[2 * q + 1]);
}

// a 64-element block of this thread's row at A column col (32 columns)
__device__ __forceinline__ void st_block(uint32_t tArow, int col, const uint32_t (&w)[32])
{
    uint32_t a[16], b[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) { a[q] = w[q]; b[q] = w[16 + q]; }
    tmem_st16(tArow + (uint32_t)col, a);
    tmem_st16(tArow + (uint32_t)col + 16u, b);
}

__device__ __forceinline__ void load_x(const float *p, TeacherAffine aff, int64_t i, int64_t n, float (&x)[3])
{
    x[0] = x[1] = x[2] = 0.f;
    if (i < n)
        for (int a = 0; a < 3; ++a) x[a] = fmaf(aff.v[a], p[3 * i + a], aff.v[3 + a]);
}

__device__ __forceinline__ void load_d(const float *d, int64_t i, int64_t n, float (&x)[3])
{
    x[0] = 0.f; x[1] = 0.f; x[2] = 1.f;
    if (i < n)
        for (int a = 0; a < 3; ++a) x[a] = d[3 * i + a];
}

__global__ void __launch_bounds__(kTThreads, 1)
    k_teacher_tc(const uint8_t *__restrict__ img, TeacherAffine aff, int64_t n, const float *__restrict__ p,
                 const float *__restrict__ d, float4 *__restrict__ out, uint32_t *status)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ TcSmem S;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t *ring = smem_raw + (base - smem_u32(smem_raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abortp = &S.abort_flag;
    const float *tab = reinterpret_cast<const float *>(img + kTTabOff);
    const int64_t n_tiles = (n + 127) / 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.d_full, 1);
        mbar_init(&S.a_full, 8);
        mbar_init(&S.drain, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tD = S.tmem, tA = S.tmem + 256;

    if (warp == 8) {
        // ---- producer ----
        if (lane == 0) {
            uint32_t i = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                // the chunks in image order: a running offset (N x 128 bytes each)
                int64_t off = 0;
                for (int l = 0; l < kTcLayers && ok; ++l) {
                    const TcLayer L = tc_layer(l);
                    const uint32_t bytes = (uint32_t)L.N * 128u;
                    for (int c = 0; c < L.chunks && ok; ++c, ++i, off += bytes) {
                        const uint32_t s = i % kTStages;
                        if (i >= (uint32_t)kTStages)
                            ok = mbar_wait(&S.empty[s], ((i / kTStages) - 1) & 1u, abortp, status);
                        if (!ok) break;
                        mbar_expect_tx(&S.full[s], bytes);
                        for (uint32_t b = 0; b < bytes; b += 16384)
                            bulk_g2s(ring + (size_t)s * kTChunk + b, img + off + b, 16384u, &S.full[s]);
                    }
                }
            }
            if (!ok) {
                // copies that may still be in flight: the last kTStages issued
                const uint32_t i0 = i > (uint32_t)kTStages ? i - kTStages : 0u;
                for (uint32_t j = i0; j < i; ++j)
                    mbar_wait(&S.full[j % kTStages], (j / kTStages) & 1u, abortp, status, true);
            }
        }
        __syncwarp();
    } else if (warp == 9) {
        // ---- MMA issuer ----
        if (lane == 0) {
            uint32_t i = 0, a_ph = 0;
            bool ok = true, any = false;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x)
                for (int l = 0; l < kTcLayers && ok; ++l) {
                    const TcLayer L = tc_layer(l);
                    ok = mbar_wait(&S.a_full, a_ph, abortp, status);
                    a_ph ^= 1u;
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t idesc = idesc_bf16(L.N);
                    for (int c = 0; c < L.chunks && ok; ++c, ++i) {
                        const uint32_t s = i % kTStages;
                        ok = mbar_wait(&S.full[s], (i / kTStages) & 1u, abortp, status);
                        if (!ok) break;
                        // the chunk's (up to) four K steps: consecutive A columns (the
                        // colour layer's F(x) block starts on a chunk boundary) and one
                        // B descriptor stepped by 32 bytes, unrolled
                        const uint64_t db = sdesc(smem_u32(ring + (size_t)s * kTChunk));
                        const uint32_t a0 = tA + (uint32_t)a_col_of(l, 4 * c);
                        const int ks = min(4, L.ksteps - 4 * c);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            if (kk < ks)
                                umma_ta<false>(tD, a0 + (uint32_t)(kk * 8), db + (uint64_t)(kk * 2), idesc,
                                               (c | kk) ? 1u : 0u);
                        umma_commit(&S.empty[s]);
                        any = true;
                    }
                    if (ok) umma_commit(&S.d_full);
                }
            // every MMA done before TMEM is freed
            if (any) {
                umma_commit(&S.drain);
                mbar_wait(&S.drain, 0, abortp, status, true);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps 0-7 ----
        const int q = warp & 3, h = warp >> 2;
        const int row = q * 32 + lane;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        const uint32_t tDrow = tD + lanes, tArow = tA + lanes;
        uint32_t d_ph = 0;
        bool aborted = false;
        float sigma = 0.f;
        int64_t t = blockIdx.x;
        // the first tile's encodings: F(x) by the first half, F(d) by the second
        if (t < n_tiles) {
            float x[3];
            uint32_t w[32];
            if (h == 0) {
                load_x(p, aff, t * 128 + row, n, x);
                encode_block<10>(x, w);
                st_block(tArow, kColFx, w);
            } else {
                load_d(d, t * 128 + row, n, x);
                encode_block<4>(x, w);
                st_block(tArow, kColFd, w);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S.a_full)) : "memory");
        }
        for (; t < n_tiles && !aborted; t += gridDim.x) {
            const int64_t pt = t * 128 + row;
            const int64_t tn = t + gridDim.x;
            for (int l = 0; l < kTcLayers; ++l) {
                const TcLayer L = tc_layer(l);
                // while layer l's MMAs run: the next tile's F(x) (layer 5 has
                // read this tile's) or F(d) (layer 10 is about to read this
                // tile's, so it is written after), kept packed until stored
                uint32_t enc[32];
                const bool enc_x = l == 6 && h == 0 && tn < n_tiles;
                const bool enc_d = l == 9 && h == 1 && tn < n_tiles;
                if (enc_x || enc_d) {
                    float x[3];
                    if (enc_x) {
                        load_x(p, aff, tn * 128 + row, n, x);
                        encode_block<10>(x, enc);
                    } else {
                        load_d(d, tn * 128 + row, n, x);
                        encode_block<4>(x, enc);
                    }
                }
                const bool got = mbar_wait(&S.d_full, d_ph, abortp, status);
                d_ph ^= 1u;
                // the eight warps leave together or not at all
                if (named_sync_or(1, 256, !got || *abortp)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                if (l < kTcLayers - 1) {
                    // 128 outputs of this half, in four passes of 32 (few live registers)
                    float ps = 0.f;
#pragma unroll 1
                    for (int g = 0; g < 4; ++g) {
                        const int c0 = h * 128 + g * 32;
                        uint32_t r0[16], r1[16];
                        tmem_ld16_nowait(tDrow + (uint32_t)c0, r0);
                        tmem_ld16_nowait(tDrow + (uint32_t)(c0 + 16), r1);
                        tmem_wait_ld();
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            v[j] = __uint_as_float(r0[j]);
                            v[16 + j] = __uint_as_float(r1[j]);
                        }
                        if (L.tab >= 0) {
                            const float4 *b4 = reinterpret_cast<const float4 *>(tab + L.tab * kTW + c0);
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float4 bb = __ldg(b4 + j);
                                v[4 * j] += bb.x; v[4 * j + 1] += bb.y; v[4 * j + 2] += bb.z; v[4 * j + 3] += bb.w;
                            }
                        }
                        if (l == 7) {
                            // density head on layer 8's FP32 output (no activation on it)
                            const float4 *w4 = reinterpret_cast<const float4 *>(tab + 7 * kTW + c0);
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float4 ww = __ldg(w4 + j);
                                ps = fmaf(ww.x, v[4 * j], ps);
                                ps = fmaf(ww.y, v[4 * j + 1], ps);
                                ps = fmaf(ww.z, v[4 * j + 2], ps);
                                ps = fmaf(ww.w, v[4 * j + 3], ps);
                            }
                        }
                        if (L.relu) st_act32<false, true>(tArow, c0 >> 5, v);
                        else st_act32<false, false>(tArow, c0 >> 5, v);
                    }
                    if (enc_x) st_block(tArow, kColFx, enc);
                    if (l == 7) {
                        S.red[h][row][0] = ps;
                        named_sync_or(2, 256, false);
                        if (h == 0) sigma = fmaxf(S.red[0][row][0] + S.red[1][row][0] + tab[8 * kTW], 0.f);
                    }
                } else {
                    // layer 10 (64 of its 128 outputs per half), ReLU, then this
                    // half's share of the 3-output layer in FP32, 16 columns a pass
                    const float4 *wo = reinterpret_cast<const float4 *>(tab + 8 * kTW + 4);
                    float ar = 0.f, ag = 0.f, ab = 0.f;
#pragma unroll 1
                    for (int c = 0; c < 4; ++c) {
                        uint32_t r[16];
                        tmem_ld16_nowait(tDrow + (uint32_t)(h * 64 + 16 * c), r);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float g = fmaxf(__uint_as_float(r[j]), 0.f);
                            const float4 ww = __ldg(wo + h * 64 + 16 * c + j);
                            ar = fmaf(ww.x, g, ar);
                            ag = fmaf(ww.y, g, ag);
                            ab = fmaf(ww.z, g, ab);
                        }
                    }
                    S.red[h][row][1] = ar;
                    S.red[h][row][2] = ag;
                    S.red[h][row][3] = ab;
                    // layer 10 has read this tile's F(d): the next tile's takes its place
                    if (enc_d) st_block(tArow, kColFd, enc);
                    named_sync_or(2, 256, false);
                    if (h == 0 && pt < n) {
                        const float4 bo = __ldg(wo + kTC);
                        const float zr = S.red[0][row][1] + S.red[1][row][1] + bo.x;
                        const float zg = S.red[0][row][2] + S.red[1][row][2] + bo.y;
                        const float zb = S.red[0][row][3] + S.red[1][row][3] + bo.z;
                        out[pt] = make_float4(sigma, sigmoid_f(zr), sigmoid_f(zg), sigmoid_f(zb));
                    }
                    // the red[] slots are read before the next tile writes them
                    named_sync_or(2, 256, false);
                    if (tn >= n_tiles) break;
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S.a_full)) : "memory");
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(512) : "memory");
    }
}

// ---- the FP32 SIMT form ----------------------------------------------------

constexpr int kSP = 32;          // points per block
constexpr int kSLd = 320;        // shared activation row: [layer input (<= 256) | F(x) (63) | 0]

// API layout -> every layer transposed ([K][N]) then its bias [N]
__global__ void k_teacher_pack_simt(const float *__restrict__ w, float *__restrict__ wt)
{
    for (int a = 0; a < kTLayers; ++a) {
        const int N = t_out(a), K = t_in(a);
        const float *src = w + t_off(a);
        float *dst = wt + t_off(a);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)N * K + N;
             e += (int64_t)gridDim.x * blockDim.x) {
            if (e < (int64_t)N * K) {
                const int k = (int)(e / N), nn = (int)(e % N);
                dst[e] = src[(int64_t)nn * K + k];
            } else {
                dst[e] = src[e];
            }
        }
    }
}

// one layer: Y[p][n] = act(b[n] + sum_k X[p][k] W[k][n]) for n < N, thread = n
__device__ __forceinline__ void simt_layer(const float *__restrict__ wt, int a, const float (*X)[kSLd], float (*Y)[kSLd],
                                           int relu)
{
    const int N = t_out(a), K = t_in(a);
    const float *Wt = wt + t_off(a);
    const int nn = threadIdx.x;
    if (nn < N) {
        float acc[kSP];
        const float b = Wt[(int64_t)N * K + nn];
#pragma unroll
        for (int q = 0; q < kSP; ++q) acc[q] = b;
        for (int k = 0; k < K; ++k) {
            const float wk = __ldg(Wt + (int64_t)k * N + nn);
#pragma unroll
            for (int q = 0; q < kSP; ++q) acc[q] = fmaf(X[q][k], wk, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < kSP; ++q) Y[q][nn] = relu ? fmaxf(acc[q], 0.f) : acc[q];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_teacher_simt(const float *__restrict__ wt, TeacherAffine aff, int64_t n,
                                                      const float *__restrict__ p, const float *__restrict__ d,
                                                      float4 *__restrict__ out)
{
    extern __shared__ float sm[];
    float(*X)[kSLd] = reinterpret_cast<float(*)[kSLd]>(sm);
    float(*Y)[kSLd] = reinterpret_cast<float(*)[kSLd]>(sm + kSP * kSLd);
    __shared__ float fd[kSP][kPeD];
    __shared__ float sig[kSP];
    for (int64_t base = (int64_t)blockIdx.x * kSP; base < n; base += (int64_t)gridDim.x * kSP) {
        // encodings: F(x) at columns 0..62 of X (layer 1's input) and again at
        // 256..318 of Y (the skip into layer 5); F(d) aside
        for (int q = threadIdx.x; q < kSP; q += blockDim.x) {
            const int64_t i = base + q;
            float x[3] = {0.f, 0.f, 0.f}, dv[3] = {0.f, 0.f, 1.f};
            if (i < n)
                for (int a = 0; a < 3; ++a) {
                    x[a] = fmaf(aff.v[a], p[3 * i + a], aff.v[3 + a]);
                    dv[a] = d[3 * i + a];
                }
            for (int a = 0; a < 3; ++a) {
                X[q][a] = x[a];
                fd[q][a] = dv[a];
            }
            for (int k = 0; k < 10; ++k)
                for (int a = 0; a < 3; ++a) {
                    float s, c;
                    sincospif(x[a] * (float)(1 << k), &s, &c);
                    X[q][3 + 6 * k + a] = s;
                    X[q][6 + 6 * k + a] = c;
                }
            for (int k = 0; k < 4; ++k)
                for (int a = 0; a < 3; ++a) {
                    float s, c;
                    sincospif(dv[a] * (float)(1 << k), &s, &c);
                    fd[q][3 + 6 * k + a] = s;
                    fd[q][6 + 6 * k + a] = c;
                }
            for (int k = 0; k < kPeX; ++k) Y[q][kTW + k] = X[q][k];
        }
        __syncthreads();
        simt_layer(wt, 0, X, Y, 1);                  // layer 1 -> Y[0..255]; Y keeps F(x) at 256..318
        simt_layer(wt, 1, Y, X, 1);
        simt_layer(wt, 2, X, Y, 1);
        // layer 4 writes X; layer 5 reads [X | F(x)]: copy F(x) beside it
        for (int e = threadIdx.x; e < kSP * kPeX; e += blockDim.x) X[e / kPeX][kTW + e % kPeX] = Y[e / kPeX][kTW + e % kPeX];
        simt_layer(wt, 3, Y, X, 1);
        simt_layer(wt, 4, X, Y, 1);                  // layer 5 on [h4 | F(x)]
        simt_layer(wt, 5, Y, X, 1);
        simt_layer(wt, 6, X, Y, 1);
        simt_layer(wt, 7, Y, X, 0);                  // layer 8, linear
        // density head: one warp per point group
        {
            const float *Wd = wt + t_off(8);
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int q = warp; q < kSP; q += blockDim.x >> 5) {
                float s = 0.f;
                for (int k = lane; k < kTW; k += 32) s = fmaf(X[q][k], Wd[k], s);
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) sig[q] = fmaxf(s + Wd[kTW], 0.f);
            }
        }
        simt_layer(wt, 9, X, Y, 1);                  // feature head -> Y[0..255]
        for (int e = threadIdx.x; e < kSP * kPeD; e += blockDim.x) Y[e / kPeD][kTW + e % kPeD] = fd[e / kPeD][e % kPeD];
        __syncthreads();
        simt_layer(wt, 10, Y, X, 1);                 // layer 10 on [feature | F(d)] -> X[0..127]
        {
            const float *Wo = wt + t_off(11);         // [128][3] then bias[3]
            for (int q = threadIdx.x; q < kSP; q += blockDim.x) {
                float z[3] = {Wo[3 * kTC], Wo[3 * kTC + 1], Wo[3 * kTC + 2]};
                for (int k = 0; k < kTC; ++k)
                    for (int c = 0; c < 3; ++c) z[c] = fmaf(X[q][k], Wo[3 * k + c], z[c]);
                const int64_t i = base + q;
                if (i < n)
                    out[i] = make_float4(sig[q], 1.f / (1.f + expf(-z[0])), 1.f / (1.f + expf(-z[1])),
                                         1.f / (1.f + expf(-z[2])));
            }
        }
        __syncthreads();
    }
}

}  // namespace

int64_t teacher_param_count() { return t_off(kTLayers); }

int64_t teacher_image_bytes() { return kTImageBytes; }

void launch_teacher_pack(const float *w, uint8_t *img, float *wt, cudaStream_t s)
{
    k_teacher_pack_tc<<<1024, 256, 0, s>>>(w, img);
    k_teacher_pack_simt<<<512, 256, 0, s>>>(w, wt);
}

void launch_teacher_tc(const uint8_t *img, TeacherAffine aff, int64_t n, const float *p, const float *d, float4 *out,
                       uint32_t *status, int n_sm, cudaStream_t s)
{
    const int smem = 1024 + kTStages * kTChunk;
    static int smem_set[kMaxDevices] = {};
    raise_smem_limit((const void *)k_teacher_tc, smem, smem_set);
    const int64_t tiles = (n + 127) / 128;
    const int grid = (int)(tiles < n_sm ? tiles : n_sm);
    if (grid > 0) k_teacher_tc<<<grid, kTThreads, smem, s>>>(img, aff, n, p, d, out, status);
}

void launch_teacher_simt(const float *wt, TeacherAffine aff, int64_t n, const float *p, const float *d, float4 *out,
                         int n_sm, cudaStream_t s)
{
    const int smem = 2 * kSP * kSLd * (int)sizeof(float);
    static int smem_set[kMaxDevices] = {};
    raise_smem_limit((const void *)k_teacher_simt, smem, smem_set);
    const int64_t blocks = (n + kSP - 1) / kSP;
    const int grid = (int)(blocks < 4 * n_sm ? blocks : 4 * n_sm);
    if (grid > 0) k_teacher_simt<<<grid, 256, smem, s>>>(wt, aff, n, p, d, out);
}

}  // namespace roam
