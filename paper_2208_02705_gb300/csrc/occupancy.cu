// Progressive probabilistic occupancy (Eq. 6; Alg. 1 stage I): the log-odds
// of every voxel grows by the measurement of each scan (one rendered view:
// depth and the opacity that normalises the weights of Eq. 5), clamped to
// [l_min, l_max], and a voxel is occupied iff its log-odds exceed
// logit(p_occ).  Per scan:
//   k_occ_rays   one thread per pixel with opacity A >= a_min: the ray's end
//                point is o + (D / A) d; every voxel whose interior the
//                segment crosses is marked free (a bit per voxel), the voxel
//                of the end point takes the ray's A as its hit confidence
//                (atomic max)
//   k_occ_apply  one thread per voxel: hit -> L += logit(1/2 + (p_hit - 1/2) A),
//                else free -> L += logit(p_miss); clamp; clear the marks;
//                one ballot per warp writes the occupancy bits
// The traversal walks the segment's voxel-plane crossings in increasing
// order, defined in FP64: the first interval's voxel from its midpoint, then
// one voxel step on every axis that crosses at the next parameter (all at
// once when they tie), marking each interval's voxel unless the interval is
// shorter than 1e-9 voxel; free bits of one 32-voxel word are gathered in
// a register and flushed with one atomic when the word changes.  FP64 runs
// at a small fraction of the FP32 rate on this GPU, so the walk steps in
// FP32 while every decision is clear by a margin far above FP32 rounding
// (1e-3 voxel between the next crossing, the one after it and the end, and
// for the interval length) and hands the ray over to the FP64 walk, from
// the same integer state (plane indices, voxel), at the first step that is
// not: the voxels marked are those of the FP64 definition.
#include "internal.cuh"

namespace roam {

namespace {

__global__ void __launch_bounds__(256) k_occ_rays(GridDev g, const DevCamera *cams, int view, const float *depth,
                                                  const float *opacity, float a_min, uint32_t *hit,
                                                  uint32_t *free_bits)
{
    const DevCamera c = cams[view];
    const uint32_t n_pix = (uint32_t)c.width * (uint32_t)c.height;
    for (uint32_t pix = blockIdx.x * blockDim.x + threadIdx.x; pix < n_pix; pix += gridDim.x * blockDim.x) {
        const uint32_t gp = c.pix_start + pix;
        const float A = opacity[gp];
        if (!(A >= a_min)) continue;
        double3 d;
        make_ray64(c, pix, d);
        const double o[3] = {(double)c.o[0], (double)c.o[1], (double)c.o[2]};
        const double dv[3] = {d.x, d.y, d.z};
        const double t_end = (double)depth[gp] / (double)A;
        const double vox = (double)g.vox, ivox = 1.0 / vox;
        const double org[3] = {(double)g.origin[0], (double)g.origin[1], (double)g.origin[2]};
        const int dims[3] = {g.gx, g.gy, g.gz};
        const double len = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        // next crossing parameter, plane index and step per axis; crossing
        // parameters come from the plane index each time (no accumulated error)
        double tn[3], kn[3], inv[3];
        int step[3];
        for (int a = 0; a < 3; ++a) {
            tn[a] = 1e300;
            kn[a] = 0.0;
            inv[a] = 0.0;
            step[a] = 0;
            if (dv[a] != 0.0) {
                inv[a] = 1.0 / dv[a];
                step[a] = dv[a] > 0.0 ? 1 : -1;
                const double u0 = (o[a] - org[a]) * ivox;
                kn[a] = dv[a] > 0.0 ? floor(u0) + 1.0 : ceil(u0) - 1.0;
                double t = (org[a] + kn[a] * vox - o[a]) * inv[a];
                while (t <= 0.0) {                     // planes at the start are not crossings (t > 0)
                    kn[a] += (double)step[a];
                    t = (org[a] + kn[a] * vox - o[a]) * inv[a];
                }
                tn[a] = t;
            }
        }
        // the first interval's cell from its midpoint, then one step per crossing
        int64_t cc[3];
        {
            const double t1 = fmin(fmin(fmin(tn[0], tn[1]), tn[2]), t_end);
            const double tm = 0.5 * t1;
            for (int a = 0; a < 3; ++a) cc[a] = (int64_t)floor((o[a] + tm * dv[a] - org[a]) * ivox);
        }
        // free bits of the current 32-voxel word, flushed when the word changes;
        // every ray of a view starts at the camera, so the words near it are
        // hit by all of them: bits already set (they are only ever set during
        // a scan) skip the atomic
        int64_t word = -1;
        uint32_t mask = 0u;
        auto flush = [&]() {
            if (mask && (__ldcg(&free_bits[word]) & mask) != mask) atomicOr(&free_bits[word], mask);
        };
        auto mark_if_inside = [&]() {
            if (cc[0] < 0 || cc[0] >= dims[0] || cc[1] < 0 || cc[1] >= dims[1] || cc[2] < 0 || cc[2] >= dims[2])
                return;
            const int64_t v = (cc[2] * dims[1] + cc[1]) * dims[0] + cc[0];
            if ((v >> 5) != word) {
                flush();
                word = v >> 5;
                mask = 0u;
            }
            mask |= 1u << (v & 31);
        };
        // the walk: each step in FP32 when its decisions are clear, else that
        // one step in FP64 from the plane indices (then FP32 again)
        {
            const float eps = (float)(1e-3 * vox / len);           // 1e-3 voxel along the ray, as a parameter
            const float of[3] = {(float)o[0], (float)o[1], (float)o[2]};
            const float gf[3] = {(float)org[0], (float)org[1], (float)org[2]};
            const float vf = (float)vox, te = (float)t_end;
            float inf[3], tf[3];
            for (int q = 0; q < 3; ++q) {
                inf[q] = (float)inv[q];
                tf[q] = step[q] != 0 ? (float)tn[q] : 3.0e38f;
            }
            float t_cur32 = 0.f;
            for (int guard = 0; guard < 3 * 65536; ++guard) {
                // the next event (a crossing or the end) and its margin to the one after
                float m1 = te, m2 = 3.0e38f;
                int am = 3;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float x = tf[q];
                    if (x < m1) { m2 = m1; m1 = x; am = q; }
                    else if (x < m2) m2 = x;
                }
                if (m2 - m1 >= eps && m1 - t_cur32 >= eps) {
                    mark_if_inside();
                    if (am == 3) break;
                    t_cur32 = m1;
#pragma unroll
                    for (int q = 0; q < 3; ++q)        // (no dynamic indexing: the arrays stay in registers)
                        if (q == am) {
                            kn[q] += (double)step[q];
                            cc[q] += step[q];
                            tf[q] = fmaf((float)kn[q], vf, gf[q] - of[q]) * inf[q];
                        }
                    continue;
                }
                // FP64: the parameter of the last plane crossed (0 before any)
                // and every axis' next crossing, as the definition computes them
                double t_cur = 0.0, t_next = t_end;
                double t64[3];
                for (int q = 0; q < 3; ++q) {
                    t64[q] = 1e300;
                    if (step[q] == 0) continue;
                    const double tp = (org[q] + (kn[q] - (double)step[q]) * vox - o[q]) * inv[q];
                    if (tp > t_cur) t_cur = tp;
                    t64[q] = (org[q] + kn[q] * vox - o[q]) * inv[q];
                    t_next = fmin(t_next, t64[q]);
                }
                if (t_next > t_cur && (t_next - t_cur) * len >= 1e-9 * vox) mark_if_inside();
                if (t_next >= t_end) break;
                for (int q = 0; q < 3; ++q)
                    if (t64[q] == t_next) {
                        kn[q] += (double)step[q];
                        cc[q] += step[q];
                        tf[q] = fmaf((float)kn[q], vf, gf[q] - of[q]) * inf[q];
                    }
                t_cur32 = (float)t_next;
            }
        }
        flush();
        // the end point's voxel
        int64_t ce[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            ce[a] = (int64_t)floor((o[a] + t_end * dv[a] - org[a]) * ivox);
            if (ce[a] < 0 || ce[a] >= dims[a]) inside = false;
        }
        if (inside) atomicMax(&hit[(ce[2] * dims[1] + ce[1]) * dims[0] + ce[0]], __float_as_uint(A));
    }
}

__device__ __forceinline__ float logit_f(float p) { return logf(p / (1.f - p)); }

__global__ void __launch_bounds__(256) k_occ_apply(int64_t n_vox, roam_occ_params q, uint32_t *hit, uint32_t *free_bits,
                                                   float *logit, uint32_t *bits)
{
    const float l_thr = logit_f(q.p_occ), l_miss = logit_f(q.p_miss);
    const int64_t n_words = n_vox >> 5;
    // one warp per 32-voxel word
    const int lane = threadIdx.x & 31;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_words;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t v = (w << 5) + lane;
        const uint32_t fw = free_bits[w];
        const uint32_t h = hit[v];
        float L = logit[v];
        if (h != 0u) {
            const float A = __uint_as_float(h);
            L += logit_f(0.5f + (q.p_hit - 0.5f) * A);
            hit[v] = 0u;
        } else if ((fw >> lane) & 1u) {
            L += l_miss;
        }
        if (h != 0u || ((fw >> lane) & 1u)) {
            L = fminf(fmaxf(L, q.l_min), q.l_max);
            logit[v] = L;
        }
        const uint32_t occ = __ballot_sync(0xffffffffu, L > l_thr);
        if (lane == 0) {
            free_bits[w] = 0u;
            if (bits) bits[w] = occ;
        }
    }
}

}  // namespace

void launch_occupancy_scan(const GridDev &g, const DevCamera *cams, int view, int n_pix, const float *depth,
                           const float *opacity, const roam_occ_params &q, uint32_t *hit, uint32_t *free_bits,
                           float *logit, uint32_t *bits, int n_sm, cudaStream_t s)
{
    // one thread per pixel: the traversal lengths differ widely between rays
    int blocks_r = (n_pix + 255) / 256;
    if (blocks_r < 1) blocks_r = 1;
    k_occ_rays<<<blocks_r, 256, 0, s>>>(g, cams, view, depth, opacity, q.a_min, hit, free_bits);
    const int64_t n_vox = (int64_t)g.gx * g.gy * g.gz;
    int64_t blocks_a = (n_vox + 255) / 256;
    if (blocks_a > (int64_t)n_sm * 16) blocks_a = (int64_t)n_sm * 16;
    k_occ_apply<<<(unsigned)blocks_a, 256, 0, s>>>(n_vox, q, hit, free_bits, logit, bits);
}

}  // namespace roam
