// FP32 SIMT evaluation of the per-field tiny MLPs (the plain FP32 form of
// querying many MLPs at once), one thread per sample, tiles of 128 samples
// of one field.  Positional encoding (Eq. 1's F(.)) is recomputed in the
// kernel.  Weights are read as a transposed FP32 copy ([in][out], padded to
// multiples of 4 outputs) through the read-only path; the whole warp reads
// the same weight, so every load is a broadcast.
#include "internal.cuh"

namespace roam {

namespace {

constexpr int kThreads = 128;

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// Parameter offsets of the transposed copy.
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

// acc[o] = b[o] + sum_i x[i] * WT[i][o]; x[i] lives in the thread's column
// of the shared buffer (sx[i * kThreads + tid]).
template <int K, int N>
__device__ __forceinline__ void dense(const float *__restrict__ sx, const float *__restrict__ wt,
                                      float (&acc)[N], int tid)
{
    static_assert(N % 4 == 0, "padded output count");
    const float4 *b4 = reinterpret_cast<const float4 *>(wt + (int64_t)K * N);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 b = __ldg(b4 + q);
        acc[4 * q + 0] = b.x; acc[4 * q + 1] = b.y; acc[4 * q + 2] = b.z; acc[4 * q + 3] = b.w;
    }
#pragma unroll 2
    for (int i = 0; i < K; ++i) {
        const float xi = sx[i * kThreads + tid];
        const float4 *wr = reinterpret_cast<const float4 *>(wt + (int64_t)i * N);
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 w = __ldg(wr + q);
            acc[4 * q + 0] = fmaf(w.x, xi, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(w.y, xi, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(w.z, xi, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(w.w, xi, acc[4 * q + 3]);
        }
    }
}

// F(x) = [x, sin(2^k pi x), cos(2^k pi x)]_k, three sines then three cosines
// per frequency; 2^k x is exact in FP32, sincospif reduces it exactly.
template <int L>
__device__ __forceinline__ void encode(float x0, float x1, float x2, float *sx, int base, int tid)
{
    sx[(base + 0) * kThreads + tid] = x0;
    sx[(base + 1) * kThreads + tid] = x1;
    sx[(base + 2) * kThreads + tid] = x2;
    const float xs[3] = {x0, x1, x2};
#pragma unroll
    for (int k = 0; k < L; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s, c;
            sincospif(ldexpf(xs[a], k), &s, &c);
            sx[(base + 3 + 6 * k + a) * kThreads + tid] = s;
            sx[(base + 6 + 6 * k + a) * kThreads + tid] = c;
        }
    }
}

template <int N>
__device__ __forceinline__ void store_relu(const float (&acc)[N], int n, float *sx, int base, int tid)
{
#pragma unroll
    for (int o = 0; o < N; ++o)
        if (o < n) sx[(base + o) * kThreads + tid] = fmaxf(acc[o], 0.f);
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

template <int W, int H>
__global__ void __launch_bounds__(kThreads) k_mlp_simt(MlpWeights w, SampleSrc src, BucketBufs b, Counters *ctr,
                                                       float4 *out)
{
    extern __shared__ float sx[];   // [(W + kPeD) or kPeX][kThreads]
    const int tid = threadIdx.x;
    // this width class's tiles
    const uint32_t c0 = ctr->class_tiles[w.cls], n_tiles = ctr->class_tiles[w.cls + 1] - c0;
    const uint32_t t0 = c0 + (uint32_t)((uint64_t)n_tiles * blockIdx.x / gridDim.x);
    const uint32_t t1 = c0 + (uint32_t)((uint64_t)n_tiles * (blockIdx.x + 1) / gridDim.x);
    const TLayout L(W, H);
    constexpr int NH = round4(1 + W);
    for (uint32_t t = t0; t < t1; ++t) {
        const Tile tl = b.tiles[t];
        const bool valid = (uint32_t)tid < tl.count;
        const uint32_t idx = valid ? b.sorted[tl.start + tid] : 0u;
        const float *aff = w.affine + 6 * (int64_t)tl.field;
        float xl0 = 0.f, xl1 = 0.f, xl2 = 0.f, dx = 0.f, dy = 0.f, dz = 1.f;
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
        const float *wf = w.wt + (int64_t)((int)tl.field - w.field_base) * w.Pt;

        encode<10>(xl0, xl1, xl2, sx, 0, tid);
        float h[W];
        dense<kPeX, W>(sx, wf + L.l1, h, tid);
        store_relu(h, W, sx, 0, tid);
#pragma unroll 1
        for (int k = 0; k < H - 1; ++k) {
            dense<W, W>(sx, wf + L.hid + (int64_t)k * (W * W + W), h, tid);
            store_relu(h, W, sx, 0, tid);
        }
        float hd[NH];
        dense<W, NH>(sx, wf + L.head, hd, tid);
        const float s = hd[0];
#pragma unroll
        for (int o = 0; o < W; ++o) sx[o * kThreads + tid] = hd[1 + o];   // features, no activation
        encode<4>(dx, dy, dz, sx, W, tid);
        dense<W + kPeD, W>(sx, wf + L.col, h, tid);
        store_relu(h, W, sx, 0, tid);
        float zo[4];
        dense<W, 4>(sx, wf + L.out, zo, tid);
        if (valid) {
            const float sigma = w.sigma_scale * (w.act == ROAM_RELU ? fmaxf(s, 0.f) : softplus_f(s));
            out[idx] = make_float4(sigma, sigmoid_f(zo[0]), sigmoid_f(zo[1]), sigmoid_f(zo[2]));
        }
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
            if (q < nw) {
                const int64_t o = q / n_in, i = q % n_in;
                dst = base + i * n_pad + o;
            } else if (q < nw + n_out) {
                dst = base + (int64_t)n_in * n_pad + (q - nw);
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
                     int grid, cudaStream_t s)
{
    const int kmax = (W + kPeD) > kPeX ? (W + kPeD) : kPeX;
    const size_t sh = (size_t)kmax * kThreads * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_simt<W, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        attr = true;
    }
    k_mlp_simt<W, H><<<grid, kThreads, sh, s>>>(w, src, b, ctr, out);
}

void launch_mlp_simt(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, float4 *out,
                     int grid, cudaStream_t s)
{
#define ROAM_CASE(WW, HH) \
    if (w.W == WW && w.H == HH) { launch_t<WW, HH>(w, src, b, ctr, out, grid, s); return; }
    ROAM_CASE(32, 1) ROAM_CASE(32, 2) ROAM_CASE(32, 3) ROAM_CASE(32, 4)
    ROAM_CASE(64, 1) ROAM_CASE(64, 2) ROAM_CASE(64, 3) ROAM_CASE(64, 4)
    ROAM_CASE(128, 1) ROAM_CASE(128, 2) ROAM_CASE(128, 3) ROAM_CASE(128, 4)
#undef ROAM_CASE
}

}  // namespace roam
