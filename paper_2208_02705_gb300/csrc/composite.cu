// Volume rendering with early ray termination (Eq. 4 and Eq. 5, with the
// termination of Sec. "Related Work" / NSVF): per ray, in sample order,
//   alpha_i = 1 - exp(-sigma_i delta),  w_i = T_i alpha_i,
//   T_{i+1} = T_i exp(-sigma_i delta),
//   C += w_i c_i,  D += w_i t_i,
// stopping after the first sample whose T_{i+1} < t_stop; the background is
// added with the final transmittance.  All in FP32.
#include "internal.cuh"

namespace roam {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct RoundArgs {
    MarchParams mp;          // live list, counts, recs, ray state of the round
    const float4 *sr;        // (sigma, r, g, b) per slot
    uint32_t *next_live;
    uint32_t *next_count;
    float t_stop;
    float bg0, bg1, bg2;
    float *rgb, *depth, *opacity;
};

__device__ __forceinline__ void step(float4 v, float t, float delta, float &T, float &sw, float4 &acc)
{
    const float a = -expm1f(-v.x * delta);
    const float wgt = T * a;
    acc.x = fmaf(wgt, v.y, acc.x);
    acc.y = fmaf(wgt, v.z, acc.y);
    acc.z = fmaf(wgt, v.w, acc.z);
    acc.w = fmaf(wgt, t, acc.w);
    sw += wgt;
    T *= expf(-v.x * delta);
}

__global__ void __launch_bounds__(256) k_composite_round(RoundArgs a)
{
    const MarchParams &p = a.mp;
    const uint32_t n_live = p.live_count ? *p.live_count : p.n_rays;
    const uint32_t n_pad = (n_live + 31u) & ~31u;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t R = (uint32_t)p.R;
    uint32_t used_total = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
        bool keep = false;
        uint32_t ray = 0;
        if (i < n_live) {
            ray = p.live ? p.live[i] : i;
            float2 tw = p.st.tw[ray];
            float T = tw.x, sw = tw.y;
            float4 acc = p.st.acc[ray];
            const uint32_t c = p.cnt[i];
            bool done = false;
            for (uint32_t k = 0; k < c; ++k) {
                const uint32_t s = slot_of(i, k, R);
                const float4 v = a.sr[s];
                const uint32_t j = p.recs[s] & 0xffffu;
                step(v, ((float)j + 0.5f) * p.delta, p.delta, T, sw, acc);
                ++used_total;
                if (T < a.t_stop) { done = true; break; }
            }
            const bool exhausted = p.st.j_next[ray] >= p.st.j_end[ray] || p.st.n_kept[ray] >= (uint32_t)p.n_max;
            if (done || exhausted) {
                if (a.rgb) {
                    a.rgb[3 * (int64_t)ray + 0] = fmaf(T, a.bg0, acc.x);
                    a.rgb[3 * (int64_t)ray + 1] = fmaf(T, a.bg1, acc.y);
                    a.rgb[3 * (int64_t)ray + 2] = fmaf(T, a.bg2, acc.z);
                }
                if (a.depth) a.depth[ray] = acc.w;
                if (a.opacity) a.opacity[ray] = sw;
            } else {
                p.st.tw[ray] = make_float2(T, sw);
                p.st.acc[ray] = acc;
                keep = true;
            }
        }
        const unsigned m = __ballot_sync(kFull, keep);
        if (m) {
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(m) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.next_count, (uint32_t)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (keep) a.next_live[base + __popc(m & ((1u << lane) - 1u))] = ray;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) used_total += __shfl_down_sync(kFull, used_total, o);
    if ((threadIdx.x & 31) == 0 && used_total) atomicAdd(&p.ctr->n_used, (unsigned long long)used_total);
}

__global__ void k_composite_flat(int64_t n_rays, int n_max, const uint32_t *count, const float4 *sr, const float *t,
                                 float delta, float t_stop, float bg0, float bg1, float bg2, float *rgb, float *depth,
                                 float *opacity, uint32_t *n_used)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        float T = 1.f, sw = 0.f;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t c = min(count[r], (uint32_t)n_max);
        uint32_t used = 0;
        for (uint32_t k = 0; k < c; ++k) {
            step(sr[r * n_max + k], t[r * n_max + k], delta, T, sw, acc);
            used = k + 1;
            if (T < t_stop) break;
        }
        if (rgb) {
            rgb[3 * r + 0] = fmaf(T, bg0, acc.x);
            rgb[3 * r + 1] = fmaf(T, bg1, acc.y);
            rgb[3 * r + 2] = fmaf(T, bg2, acc.z);
        }
        if (depth) depth[r] = acc.w;
        if (opacity) opacity[r] = sw;
        if (n_used) n_used[r] = used;
    }
}

// Adjoint of the compositing for one ray (rays of a single round holding all
// their samples, slot layout with R = n_max).  With I the last composited
// sample, w_i = T_i alpha_i and C = sum_{i<=I} w_i c_i + T_end bg:
//   dC/dc_i     = w_i
//   dC/dsigma_i = delta (T_{i+1} c_i - sum_{i<j<=I} w_j c_j - T_end bg).
// Pass 1 repeats the forward arithmetic to find I, T_end and the composited
// colour; pass 2 emits per slot (dL/dsigma, dL/dc) and the used count.
// With `hist`, pass 1 also counts each composited sample's field (a block
// histogram added into hist), the histogram the backward bucketing needs.
__global__ void __launch_bounds__(256) k_composite_bwd(int64_t n_rays, int R, const uint32_t *cnt,
                                                       const uint32_t *recs, const float4 *sr, float delta,
                                                       float t_stop, float bg0, float bg1, float bg2,
                                                       const float *dl_drgb, float4 *gsr, uint32_t *cnt_used,
                                                       uint32_t *hist, int n_fields)
{
    extern __shared__ uint32_t s_hist[];
    if (hist) {
        for (int f = threadIdx.x; f < n_fields; f += blockDim.x) s_hist[f] = 0u;
        __syncthreads();
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cnt[i];
        float T = 1.f, sw = 0.f;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t used = 0;
        for (uint32_t k = 0; k < c; ++k) {
            const uint32_t s = slot_of((uint32_t)i, k, (uint32_t)R);
            const float4 v = sr[s];
            const uint32_t rec = recs[s];
            step(v, ((float)(rec & 0xffffu) + 0.5f) * delta, delta, T, sw, acc);
            if (hist) atomicAdd(&s_hist[rec >> 16], 1u);
            used = k + 1;
            if (T < t_stop) break;
        }
        const float T_end = T;
        const float g0 = dl_drgb[3 * i], g1 = dl_drgb[3 * i + 1], g2 = dl_drgb[3 * i + 2];
        const float bgterm = T_end * (bg0 * g0 + bg1 * g1 + bg2 * g2);
        float Tk = 1.f;
        float S0 = 0.f, S1 = 0.f, S2 = 0.f;
        for (uint32_t k = 0; k < used; ++k) {
            const uint32_t s = slot_of((uint32_t)i, k, (uint32_t)R);
            const float4 v = sr[s];
            const float a = -expm1f(-v.x * delta);
            const float wgt = Tk * a;
            const float Tn = Tk * expf(-v.x * delta);
            S0 = fmaf(wgt, v.y, S0);
            S1 = fmaf(wgt, v.z, S1);
            S2 = fmaf(wgt, v.w, S2);
            const float d0 = fmaf(Tn, v.y, -(acc.x - S0)), d1 = fmaf(Tn, v.z, -(acc.y - S1)),
                        d2 = fmaf(Tn, v.w, -(acc.z - S2));
            const float dsig = delta * (d0 * g0 + d1 * g1 + d2 * g2 - bgterm);
            gsr[s] = make_float4(dsig, wgt * g0, wgt * g1, wgt * g2);
            Tk = Tn;
        }
        cnt_used[i] = used;
    }
    if (hist) {
        __syncthreads();
        for (int f = threadIdx.x; f < n_fields; f += blockDim.x)
            if (s_hist[f]) atomicAdd(&hist[f], s_hist[f]);
    }
}

}  // namespace

void launch_composite_bwd(int64_t n_rays, int R, const uint32_t *cnt, const uint32_t *recs, const float4 *sr,
                          float delta, float t_stop, const float *bg, const float *dl_drgb, float4 *gsr,
                          uint32_t *cnt_used, uint32_t *hist, int n_fields, cudaStream_t s)
{
    int64_t blocks = (n_rays + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    const size_t smem = hist ? (size_t)n_fields * sizeof(uint32_t) : 0;
    k_composite_bwd<<<(unsigned)blocks, 256, smem, s>>>(n_rays, R, cnt, recs, sr, delta, t_stop, bg[0], bg[1], bg[2],
                                                        dl_drgb, gsr, cnt_used, hist, n_fields);
}

void launch_composite_round(const MarchParams &mp, const float4 *sr, uint32_t *next_live, uint32_t *next_count,
                            float t_stop, const float *bg, float *rgb, float *depth, float *opacity, int grid,
                            cudaStream_t s)
{
    RoundArgs a{mp, sr, next_live, next_count, t_stop, bg[0], bg[1], bg[2], rgb, depth, opacity};
    k_composite_round<<<grid, 256, 0, s>>>(a);
}

void launch_composite_flat(int64_t n_rays, int n_max, const uint32_t *count, const float4 *sr, const float *t,
                           float delta, float t_stop, const float *bg, float *rgb, float *depth, float *opacity,
                           uint32_t *n_used, cudaStream_t s)
{
    int64_t blocks = (n_rays + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    k_composite_flat<<<(unsigned)blocks, 256, 0, s>>>(n_rays, n_max, count, sr, t, delta, t_stop, bg[0], bg[1], bg[2],
                                                      rgb, depth, opacity, n_used);
}

}  // namespace roam
