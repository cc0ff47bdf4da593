// Adjoint of the per-field tiny MLPs for the fine-tuning step (Sec.
// "Adaptive Radiance Fields Slimming and Fine-tuning": L2 loss on rendered
// pixels), FP32 SIMT: one thread per sample, tiles of 128 samples of one
// field.  Each thread recomputes its sample's encoding and activations (they
// are never stored between passes), then walks the layers backwards:
//   dgrad  dx = W^T dz            (per thread, weights from a row-padded copy)
//   wgrad  dW += dz^T x, db += dz (per tile: the 128 rows of x and dz are
//                                  staged in shared memory and each thread
//                                  owns a set of (out, in) entries)
// The field's gradient accumulates in shared memory while the CTA walks its
// contiguous run of tiles and is added to the global FP32 gradient (one
// atomic per parameter) whenever the field changes.  Also: the Adam update.
#include "internal.cuh"

namespace roam {

namespace {

constexpr int kThreads = 128;

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// offsets of the API layout
struct ALayout {
    int64_t l1, hid, head, col, out, total;
    __host__ __device__ ALayout(int W, int H)
    {
        int64_t o = 0;
        l1 = o;   o += (int64_t)W * kPeX + W;
        hid = o;  o += (int64_t)(H - 1) * ((int64_t)W * W + W);
        head = o; o += (int64_t)(1 + W) * W + (1 + W);
        col = o;  o += (int64_t)W * (W + kPeD) + W;
        out = o;  o += 3 * (int64_t)W + 3;
        total = o;
    }
};

// offsets of the row-padded copy [out][round4(in)] (matrices only)
struct RLayout {
    int64_t l1, hid, head, col, out, total;
    __host__ __device__ RLayout(int W, int H)
    {
        int64_t o = 0;
        l1 = o;   o += (int64_t)W * round4(kPeX);
        hid = o;  o += (int64_t)(H - 1) * W * W;
        head = o; o += (int64_t)(1 + W) * W;
        col = o;  o += (int64_t)W * round4(W + kPeD);
        out = o;  o += 3 * (int64_t)W;
        total = o;
    }
};

// offsets of the transposed copy used by the forward kernel (same as mlp_simt.cu;
// the head's row: W features, then the density logit, then zeros)
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

// acc[o] = b[o] + sum_i x[i] WT[i][o], x a per-thread array
template <int K, int N>
__device__ __forceinline__ void dense_arr(const float *x, const float *__restrict__ wt, float (&acc)[N])
{
    const float4 *b4 = reinterpret_cast<const float4 *>(wt + (int64_t)K * N);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 bb = __ldg(b4 + q);
        acc[4 * q + 0] = bb.x; acc[4 * q + 1] = bb.y; acc[4 * q + 2] = bb.z; acc[4 * q + 3] = bb.w;
    }
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
        const float xi = x[i];
        const float4 *wr = reinterpret_cast<const float4 *>(wt + (int64_t)i * N);
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 ww = __ldg(wr + q);
            acc[4 * q + 0] = fmaf(ww.x, xi, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(ww.y, xi, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(ww.z, xi, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(ww.w, xi, acc[4 * q + 3]);
        }
    }
}

// dx[k] = sum_n W[n][k] dz[n]; W row-padded [N][KP]; dz in the thread's
// shared-memory row
template <int N, int KP>
__device__ __forceinline__ void dgrad(const float *dz_row, const float *__restrict__ wr, float (&dx)[KP])
{
#pragma unroll
    for (int k = 0; k < KP; ++k) dx[k] = 0.f;
#pragma unroll 1
    for (int n = 0; n < N; ++n) {
        const float dn = dz_row[n];
        const float4 *w4 = reinterpret_cast<const float4 *>(wr + (int64_t)n * KP);
#pragma unroll
        for (int q = 0; q < KP / 4; ++q) {
            const float4 ww = __ldg(w4 + q);
            dx[4 * q + 0] = fmaf(ww.x, dn, dx[4 * q + 0]);
            dx[4 * q + 1] = fmaf(ww.y, dn, dx[4 * q + 1]);
            dx[4 * q + 2] = fmaf(ww.z, dn, dx[4 * q + 2]);
            dx[4 * q + 3] = fmaf(ww.w, dn, dx[4 * q + 3]);
        }
    }
}

// dW[n][k] += sum_s dz[s][n] x[s][k], db[n] += sum_s dz[s][n], over the
// tile's staged rows; each entry is owned by one thread
template <int N, int K, int XS, int DS>
__device__ __forceinline__ void wgrad(const float *xs, const float *dzs, float *gw, float *gb, int tid)
{
    for (int e = tid; e < N * K + N; e += kThreads) {
        float acc = 0.f;
        if (e < N * K) {
            const int n = e / K, k = e - n * K;
#pragma unroll 8
            for (int s = 0; s < kThreads; ++s) acc = fmaf(dzs[s * DS + n], xs[s * XS + k], acc);
            gw[e] += acc;
        } else {
            const int n = e - N * K;
#pragma unroll 8
            for (int s = 0; s < kThreads; ++s) acc += dzs[s * DS + n];
            gb[n] += acc;
        }
    }
}

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

template <int L>
__device__ __forceinline__ void encode_arr(float x0, float x1, float x2, float *e)
{
    e[0] = x0; e[1] = x1; e[2] = x2;
    const float xs[3] = {x0, x1, x2};
#pragma unroll
    for (int k = 0; k < L; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s, c;
            sincospif(ldexpf(xs[a], k), &s, &c);
            e[3 + 6 * k + a] = s;
            e[6 + 6 * k + a] = c;
        }
    }
}

template <int N>
__device__ __forceinline__ void stage_row(float *row, const float (&v)[N], int n)
{
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < n) row[i] = v[i];
}

template <int W, int H>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_bwd_simt(MlpWeights w, SampleSrc src, BucketBufs b,
                                                              Counters *ctr, const float4 *gsr, float *grad)
{
    constexpr int KC = W + kPeD;
    constexpr int KMAX = KC > kPeX ? KC : kPeX;
    constexpr int XS = KMAX + 1;
    constexpr int DS = W + 2;
    constexpr int NH = round4(1 + W);
    const ALayout A(W, H);
    const RLayout RL(W, H);
    const TLayout TL(W, H);
    const int P = (int)A.total;
    extern __shared__ float smem[];
    float *gacc = smem;                                   // [P] gradient of the current field
    float *xs = gacc + round4(P);                         // [128][XS]
    float *dzs = xs + kThreads * XS;                      // [128][DS]
    const int tid = threadIdx.x;
    float *xrow = xs + tid * XS;
    float *drow = dzs + tid * DS;

    for (int q = tid; q < P; q += kThreads) gacc[q] = 0.f;
    __syncthreads();
    const uint32_t n_tiles = ctr->n_tiles;
    const uint32_t t0 = (uint32_t)((uint64_t)n_tiles * blockIdx.x / gridDim.x);
    const uint32_t t1 = (uint32_t)((uint64_t)n_tiles * (blockIdx.x + 1) / gridDim.x);
    uint32_t cur = 0xffffffffu;
    for (uint32_t t = t0; t <= t1; ++t) {
        const uint32_t f = t < t1 ? b.tiles[t].field : 0xfffffffeu;
        if (f != cur) {
            if (cur != 0xffffffffu) {
                float *gf = grad + (int64_t)cur * w.P;
                for (int q = tid; q < P; q += kThreads) {
                    const float v = gacc[q];
                    if (v != 0.f) atomicAdd(gf + q, v);
                    gacc[q] = 0.f;
                }
                __syncthreads();
            }
            cur = f;
        }
        if (t == t1) break;
        const Tile tl = b.tiles[t];
        const bool valid = (uint32_t)tid < tl.count;
        const uint32_t idx = valid ? b.sorted[tl.start + tid] : 0u;
        const float *aff = w.affine + 6 * (int64_t)tl.field;
        float xl0 = 0.f, xl1 = 0.f, xl2 = 0.f, dx = 0.f, dy = 0.f, dz = 1.f;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid && src.mode == 1) {
            // direct points (distillation): world position and direction per sample
            const float px = src.p[3 * (int64_t)idx], py = src.p[3 * (int64_t)idx + 1], pz = src.p[3 * (int64_t)idx + 2];
            dx = src.d[3 * (int64_t)idx]; dy = src.d[3 * (int64_t)idx + 1]; dz = src.d[3 * (int64_t)idx + 2];
            xl0 = fmaf(aff[0], px, aff[3]);
            xl1 = fmaf(aff[1], py, aff[4]);
            xl2 = fmaf(aff[2], pz, aff[5]);
            g = gsr[idx];
        } else if (valid) {
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
            g = gsr[idx];
        }
        const float *wtf = w.wt + (int64_t)tl.field * w.Pt;
        const float *wrf = w.wr + (int64_t)tl.field * w.Pr;
        float *gf = gacc;

        // ---- forward recompute, activations kept per thread ----
        float pe[kPeX];
        encode_arr<10>(xl0, xl1, xl2, pe);
        float hs[H][W];
        {
            float acc[W];
            dense_arr<kPeX, W>(pe, wtf + TL.l1, acc);
#pragma unroll
            for (int o = 0; o < W; ++o) hs[0][o] = fmaxf(acc[o], 0.f);
        }
#pragma unroll
        for (int l = 1; l < H; ++l) {
            float acc[W];
            dense_arr<W, W>(hs[l - 1], wtf + TL.hid + (int64_t)(l - 1) * (W * W + W), acc);
#pragma unroll
            for (int o = 0; o < W; ++o) hs[l][o] = fmaxf(acc[o], 0.f);
        }
        float inc[KC];                    // [features; F(d)]
        float s_logit;
        {
            float acc[NH];
            dense_arr<W, NH>(hs[H - 1], wtf + TL.head, acc);
            s_logit = acc[W];             // the transposed head: features, then the density logit
#pragma unroll
            for (int o = 0; o < W; ++o) inc[o] = acc[o];
        }
        encode_arr<4>(dx, dy, dz, inc + W);
        float gg[W];
        {
            float acc[W];
            dense_arr<KC, W>(inc, wtf + TL.col, acc);
#pragma unroll
            for (int o = 0; o < W; ++o) gg[o] = fmaxf(acc[o], 0.f);
        }
        float rgb[3];
        {
            float acc[4];
            dense_arr<W, 4>(gg, wtf + TL.out, acc);
#pragma unroll
            for (int c = 0; c < 3; ++c) rgb[c] = 1.f / (1.f + expf(-acc[c]));
        }

        // ---- output layer: rgb = sigmoid(zo) ----
        float dzo[3] = {g.y * rgb[0] * (1.f - rgb[0]), g.z * rgb[1] * (1.f - rgb[1]), g.w * rgb[2] * (1.f - rgb[2])};
        stage_row(xrow, gg, W);
        stage_row(drow, dzo, 3);
        __syncthreads();
        wgrad<3, W, XS, DS>(xs, dzs, gf + A.out, gf + A.out + 3 * W, tid);
        float dv[round4(KC)];
        {
            float d_g[W];
            dgrad<3, W>(drow, wrf + RL.out, d_g);
#pragma unroll
            for (int k = 0; k < W; ++k) dv[k] = gg[k] > 0.f ? d_g[k] : 0.f;
        }
        __syncthreads();
        // ---- colour layer: g = relu(Wc [feat; F(d)] + bc) ----
        stage_row(xrow, inc, KC);
        {
            float t[W];
#pragma unroll
            for (int k = 0; k < W; ++k) t[k] = dv[k];
            stage_row(drow, t, W);
        }
        __syncthreads();
        wgrad<W, KC, XS, DS>(xs, dzs, gf + A.col, gf + A.col + (int64_t)W * KC, tid);
        {
            float d_in[round4(KC)];
            dgrad<W, round4(KC)>(drow, wrf + RL.col, d_in);
#pragma unroll
            for (int k = 0; k < W; ++k) dv[k] = d_in[k];       // d feat (features have no activation)
        }
        __syncthreads();
        // ---- head: [s; feat] = Wh h_H + bh, sigma = scale * softplus(s) ----
        {
            const float ds = g.x * w.sigma_scale *
                             (w.act == ROAM_RELU ? (s_logit > 0.f ? 1.f : 0.f) : 1.f / (1.f + expf(-s_logit)));
            float t[W + 1];
            t[0] = ds;
#pragma unroll
            for (int k = 0; k < W; ++k) t[1 + k] = dv[k];
            stage_row(xrow, hs[H - 1], W);
            stage_row(drow, t, W + 1);
        }
        __syncthreads();
        wgrad<W + 1, W, XS, DS>(xs, dzs, gf + A.head, gf + A.head + (int64_t)(1 + W) * W, tid);
        {
            float d_h[W];
            dgrad<W + 1, W>(drow, wrf + RL.head, d_h);
#pragma unroll
            for (int k = 0; k < W; ++k) dv[k] = hs[H - 1][k] > 0.f ? d_h[k] : 0.f;
        }
        __syncthreads();
        // ---- hidden layers H..2 ----
#pragma unroll
        for (int l = H - 1; l >= 1; --l) {
            {
                float t[W];
#pragma unroll
                for (int k = 0; k < W; ++k) t[k] = dv[k];
                stage_row(xrow, hs[l - 1], W);
                stage_row(drow, t, W);
            }
            __syncthreads();
            const int64_t ob = A.hid + (int64_t)(l - 1) * (W * W + W);
            wgrad<W, W, XS, DS>(xs, dzs, gf + ob, gf + ob + (int64_t)W * W, tid);
            {
                float d_h[W];
                dgrad<W, W>(drow, wrf + RL.hid + (int64_t)(l - 1) * W * W, d_h);
#pragma unroll
                for (int k = 0; k < W; ++k) dv[k] = hs[l - 1][k] > 0.f ? d_h[k] : 0.f;
            }
            __syncthreads();
        }
        // ---- layer 1 ----
        {
            float t[W];
#pragma unroll
            for (int k = 0; k < W; ++k) t[k] = dv[k];
            stage_row(xrow, pe, kPeX);
            stage_row(drow, t, W);
        }
        __syncthreads();
        wgrad<W, kPeX, XS, DS>(xs, dzs, gf + A.l1, gf + A.l1 + (int64_t)W * kPeX, tid);
        __syncthreads();
    }
}

// API layout -> row-padded copy (matrices only)
__global__ void k_pack_rows(const float *__restrict__ w32, int n_fields, int W, int H, int64_t P,
                            float *__restrict__ wr, int64_t Pr)
{
    const ALayout A(W, H);
    const RLayout RL(W, H);
    const int64_t n = (int64_t)n_fields * P;
    for (int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gidx < n;
         gidx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = gidx / P, q = gidx % P;
        int64_t src0, dst0;
        int n_out, n_in, kp;
        if (q < A.hid) { src0 = A.l1; dst0 = RL.l1; n_out = W; n_in = kPeX; }
        else if (q < A.head) {
            const int64_t l = (q - A.hid) / ((int64_t)W * W + W);
            src0 = A.hid + l * (W * W + W); dst0 = RL.hid + l * W * W; n_out = W; n_in = W;
        }
        else if (q < A.col) { src0 = A.head; dst0 = RL.head; n_out = 1 + W; n_in = W; }
        else if (q < A.out) { src0 = A.col; dst0 = RL.col; n_out = W; n_in = W + kPeD; }
        else { src0 = A.out; dst0 = RL.out; n_out = 3; n_in = W; }
        kp = round4(n_in);
        const int64_t r = q - src0;
        if (r >= (int64_t)n_out * n_in) continue;      // a bias
        const int64_t o = r / n_in, i = r % n_in;
        wr[f * Pr + dst0 + o * kp + i] = w32[gidx];
    }
}

__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        w[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// L2 photometric loss of the fine-tuning stage: loss += sum (rgb - target)^2
// / norm over the rays, and dl/drgb = 2 (rgb - target) / norm.
// One block: the loss is summed in a fixed order (per-thread strided sums,
// then a fixed tree), so the same inputs give the same bits on every run.
__global__ void __launch_bounds__(1024) k_l2_loss(int64_t n3, const float *__restrict__ rgb,
                                                  const float *__restrict__ target, float inv_norm,
                                                  float *__restrict__ dl, float *__restrict__ loss)
{
    __shared__ float part[32];
    float acc = 0.f;
    for (int64_t i = threadIdx.x; i < n3; i += blockDim.x) {
        const float e = rgb[i] - target[i];
        dl[i] = 2.f * e * inv_norm;
        acc = fmaf(e * inv_norm, e, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) *loss = v;
    }
}

template <int W, int H>
void launch_bwd_t(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr, const float4 *gsr,
                  float *grad, int grid, cudaStream_t s)
{
    constexpr int KC = W + kPeD;
    constexpr int KMAX = KC > kPeX ? KC : kPeX;
    const size_t sh = ((size_t)round4((int)ALayout(W, H).total) + (size_t)kThreads * (KMAX + 1) +
                       (size_t)kThreads * (W + 2)) * sizeof(float);
    static int smem_set[kMaxDevices] = {};
    raise_smem_limit((const void *)k_mlp_bwd_simt<W, H>, (int)sh, smem_set);
    k_mlp_bwd_simt<W, H><<<grid, kThreads, sh, s>>>(w, src, b, ctr, gsr, grad);
}

}  // namespace

bool mlp_bwd_supported(int W, int H) { return (W == 32 || W == 64) && H >= 1 && H <= 4; }

int64_t rows_padded_size(int W, int H) { return RLayout(W, H).total; }

void launch_pack_rows(const float *w32, int n_fields, int W, int H, int64_t P, float *wr, int64_t Pr, cudaStream_t s)
{
    cudaMemsetAsync(wr, 0, (size_t)n_fields * Pr * sizeof(float), s);
    k_pack_rows<<<1024, 256, 0, s>>>(w32, n_fields, W, H, P, wr, Pr);
}

void launch_mlp_bwd_simt(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr,
                         const float4 *gsr, float *grad, int grid, cudaStream_t s)
{
#define ROAM_CASE(WW, HH) \
    if (w.W == WW && w.H == HH) { launch_bwd_t<WW, HH>(w, src, b, ctr, gsr, grad, grid, s); return; }
    ROAM_CASE(32, 1) ROAM_CASE(32, 2) ROAM_CASE(32, 3) ROAM_CASE(32, 4)
    ROAM_CASE(64, 1) ROAM_CASE(64, 2) ROAM_CASE(64, 3) ROAM_CASE(64, 4)
#undef ROAM_CASE
}

// Eq. 7 over samples: sum [(sigma_s - sigma_t)^2 + |c_s - c_t|^2] / I, its
// gradient 2 (student - teacher) / I per component; one block, fixed order.
__global__ void __launch_bounds__(1024) k_distill_loss(int64_t n, const float4 *__restrict__ st,
                                                       const float4 *__restrict__ te, float inv_I,
                                                       float4 *__restrict__ dl, float *__restrict__ loss)
{
    __shared__ float part[32];
    float acc = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 a = st[i], b = te[i];
        const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
        dl[i] = make_float4(2.f * e0 * inv_I, 2.f * e1 * inv_I, 2.f * e2 * inv_I, 2.f * e3 * inv_I);
        acc = fmaf(e0 * inv_I, e0, acc);
        acc = fmaf(e1 * inv_I, e1, acc);
        acc = fmaf(e2 * inv_I, e2, acc);
        acc = fmaf(e3 * inv_I, e3, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) *loss = v;
    }
}

void launch_distill_loss(int64_t n, const float4 *student, const float4 *teacher, float I, float4 *dl, float *loss,
                         cudaStream_t s)
{
    k_distill_loss<<<1, 1024, 0, s>>>(n, student, teacher, 1.0f / I, dl, loss);
}

void launch_l2_loss(int64_t n_rays, const float *rgb, const float *target, float norm, float *dl, float *loss,
                    cudaStream_t s)
{
    k_l2_loss<<<1, 1024, 0, s>>>(3 * n_rays, rgb, target, 1.0f / norm, dl, loss);
}

void launch_adam(float *w32, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, cudaStream_t s)
{
    k_adam<<<2048, 256, 0, s>>>(w32, m, v, g, n, lr, b1, b2, eps, bc1, bc2);
}

}  // namespace roam
