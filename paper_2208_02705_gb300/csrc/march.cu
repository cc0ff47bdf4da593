// Ray generation, empty-space skipping march over the bit-packed occupancy
// grid and field lookup (Sec. "Real-time Rendering Speedup": rays are cast
// through a GPU-resident voxel structure to find occupied voxels, one ray
// per thread, each occupied voxel carrying the id of its tiny MLP), plus the
// load-time kernels that build the rank prefix and the brick distance map.
#include "internal.cuh"

namespace roam {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Exclusive scan of one value per thread over a block of 1024 threads.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t excl = x - v + (wid > 0 ? warp_sums[wid - 1] : 0u);
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

// prefix[w] = popcount of all words before w, in blocks of 4096 words
__global__ void k_prefix_local(const uint32_t *__restrict__ bits, uint32_t *__restrict__ prefix,
                               uint32_t *__restrict__ block_sums, int64_t n_words)
{
    const int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    uint32_t c[4], s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c[q] = base + q < n_words ? (uint32_t)__popc(bits[base + q]) : 0u;
        s += c[q];
    }
    uint32_t tot;
    uint32_t e = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q < n_words) prefix[base + q] = e;
        e += c[q];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_prefix_blocks(uint32_t *block_sums, int64_t n_blocks)
{
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < n_blocks; b0 += blockDim.x) {
        int64_t b = b0 + threadIdx.x;
        uint32_t v = b < n_blocks ? block_sums[b] : 0u;
        uint32_t tot;
        uint32_t e = block_exclusive_scan(v, &tot);
        if (b < n_blocks) block_sums[b] = e + carry;
        carry += tot;
    }
}

__global__ void k_prefix_add(uint32_t *prefix, const uint32_t *block_sums, int64_t n_words)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_words) prefix[i] += block_sums[i / 4096];
}

// one thread per 8^3 brick: 1 if any of its 512 voxels is occupied
__global__ void k_brick_occ(GridDev g, uint8_t *occ)
{
    const int64_t n = (int64_t)g.bx * g.by * g.bz;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(b % g.bx), by = (int)((b / g.bx) % g.by), bz = (int)(b / ((int64_t)g.bx * g.by));
        const int x0 = bx << kBrickShift;
        uint32_t any = 0;
        for (int z = bz * 8; z < bz * 8 + 8; ++z)
            for (int y = by * 8; y < by * 8 + 8; ++y) {
                const uint32_t w = g.bits[((int64_t)z * g.gy + y) * g.wpr + (x0 >> 5)];
                any |= (w >> (x0 & 31)) & 0xffu;
            }
        occ[b] = any ? 1 : 0;
    }
}

// Chebyshev (L-infinity) distance, in bricks, from every brick to the nearest
// occupied brick, separably: along x from the occupancy, then along y and z
// taking max(|offset|, previous distance).  0 marks an occupied brick.
__global__ void k_brick_dist(GridDev g, int axis, const uint8_t *occ, const uint16_t *src, uint16_t *dst)
{
    const int ext[3] = {g.bx, g.by, g.bz};
    const int64_t n = (int64_t)g.bx * g.by * g.bz;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        int c[3] = {(int)(b % g.bx), (int)((b / g.bx) % g.by), (int)(b / ((int64_t)g.bx * g.by))};
        const int64_t stride = axis == 0 ? 1 : (axis == 1 ? g.bx : (int64_t)g.bx * g.by);
        const int64_t b0 = b - (int64_t)c[axis] * stride;
        int best = 0xffff;
        for (int u = 0; u < ext[axis]; ++u) {
            const int off = u > c[axis] ? u - c[axis] : c[axis] - u;
            int v;
            if (axis == 0) v = occ[b0 + u * stride] ? off : 0xffff;
            else {
                const int prev = src[b0 + u * stride];
                v = prev == 0xffff ? 0xffff : (off > prev ? off : prev);
            }
            best = v < best ? v : best;
        }
        dst[b] = (uint16_t)best;
    }
}

__global__ void k_brick_final(int64_t n, const uint16_t *d16, uint8_t *dist)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x)
        dist[b] = (uint8_t)(d16[b] > 255 ? 255 : d16[b]);
}

// Pixel -> world ray.  Equirectangular: Eq. 2 gives longitude
// phi = 2 pi ((u + 1/2)/W - 1/2) and latitude theta = pi (1/2 - (v + 1/2)/H);
// Eq. 3 gives the camera-frame direction (cos t sin p, -sin t, cos t cos p).
// Perspective: pinhole, d_cam = normalise((u + 1/2 - W/2)/f, (v + 1/2 - H/2)/f, 1).
__device__ __forceinline__ void make_ray(const DevCamera &c, uint32_t pix, float3 &o, float3 &d)
{
    const uint32_t u = pix % (uint32_t)c.width, v = pix / (uint32_t)c.width;
    float d0, d1, d2;
    if (c.model == ROAM_EQUIRECT) {
        const float pu = 2.0f * (((float)u + 0.5f) / (float)c.width) - 1.0f;   // phi / pi
        const float tv = 0.5f - ((float)v + 0.5f) / (float)c.height;            // theta / pi
        float sp, cp, st, ct;
        sincospif(pu, &sp, &cp);
        sincospif(tv, &st, &ct);
        d0 = ct * sp;
        d1 = -st;
        d2 = ct * cp;
    } else {
        const float x = ((float)u + 0.5f - 0.5f * (float)c.width) * c.inv_f;
        const float y = ((float)v + 0.5f - 0.5f * (float)c.height) * c.inv_f;
        const float n = 1.0f / sqrtf(x * x + y * y + 1.0f);
        d0 = x * n;
        d1 = y * n;
        d2 = n;
    }
    d.x = c.R[0] * d0 + c.R[1] * d1 + c.R[2] * d2;
    d.y = c.R[3] * d0 + c.R[4] * d1 + c.R[5] * d2;
    d.z = c.R[6] * d0 + c.R[7] * d1 + c.R[8] * d2;
    o = make_float3(c.o[0], c.o[1], c.o[2]);
}

// The same ray direction in FP64, for the FP32 render path: its sample
// positions feed 2^9 pi frequencies, so the direction carries a residual.
__device__ __forceinline__ int view_of(const DevCamera *cams, int n_views, uint32_t gpix)
{
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].pix_start <= gpix) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The ray of live slot i (ray index `ray`) at the start of its round: on
// the first round built from its pixel and clipped against the grid box
// (state initialised), later read back from the ray state.  False for a bad
// (view, pixel) request, whose state is cleared and status flagged.  `lead`
// selects the thread that writes the state (all callers compute the same values).
__device__ __forceinline__ bool ray_begin(const GridDev &g, const MarchParams &p, uint32_t i, uint32_t ray, bool lead,
                                          float3 &o, float3 &d, uint32_t &jn, uint32_t &je, uint32_t &nk)
{
    const float delta = p.delta;
    if (p.init) {
        uint32_t view, pix;
        if (p.rays) {
            view = p.rays[2 * ray];
            pix = p.rays[2 * ray + 1];
            if (view >= (uint32_t)p.n_views ||
                pix >= (uint32_t)p.cams[view].width * (uint32_t)p.cams[view].height) {
                if (lead) atomicOr(&p.ctr->status, kStatusBadSample);
                if (lead) p.cnt[i] = 0;
                if (lead) p.st.j_next[ray] = 0;
                if (lead) p.st.j_end[ray] = 0;
                if (lead) p.st.n_kept[ray] = 0;
                if (lead) p.st.acc[ray] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (lead) p.st.tw[ray] = make_float2(1.f, 0.f);
                if (lead) p.st.orig[ray] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (lead) p.st.dir[ray] = make_float4(0.f, 0.f, 1.f, 0.f);
                return false;
            }
        } else {
            view = (uint32_t)view_of(p.cams, p.n_views, ray);
            pix = ray - p.cams[view].pix_start;
        }
        make_ray(p.cams[view], pix, o, d);
        if (p.accurate) {
            double3 dd;
            make_ray64(p.cams[view], pix, dd);
            d = make_float3((float)dd.x, (float)dd.y, (float)dd.z);
            if (lead)
                p.st.dir_lo[ray] = make_float4((float)(dd.x - (double)d.x), (float)(dd.y - (double)d.y),
                                               (float)(dd.z - (double)d.z), 0.f);
        }
        if (lead) p.st.orig[ray] = make_float4(o.x, o.y, o.z, 0.f);
        if (lead) p.st.dir[ray] = make_float4(d.x, d.y, d.z, 0.f);
        // clip against the grid box in voxel units
        const float og[3] = {(o.x - g.origin[0]) * g.inv_vox, (o.y - g.origin[1]) * g.inv_vox,
                             (o.z - g.origin[2]) * g.inv_vox};
        const float dg[3] = {d.x * g.inv_vox, d.y * g.inv_vox, d.z * g.inv_vox};
        const float ext[3] = {(float)g.gx, (float)g.gy, (float)g.gz};
        float t0 = 0.f, t1 = 3.0e38f;
        bool miss = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (dg[a] == 0.f) {
                if (og[a] < 0.f || og[a] >= ext[a]) miss = true;
            } else {
                float ta = (0.f - og[a]) / dg[a], tb = (ext[a] - og[a]) / dg[a];
                if (ta > tb) { const float s = ta; ta = tb; tb = s; }
                t0 = fmaxf(t0, ta);
                t1 = fminf(t1, tb);
            }
        }
        if (miss || t1 < t0) {
            jn = je = 0;
        } else {
            const float js = floorf(t0 / delta - 0.5f) - 1.0f;
            jn = js > 0.f ? (uint32_t)js : 0u;
            je = (uint32_t)fmaxf(ceilf(t1 / delta - 0.5f) + 2.0f, 0.f);
        }
        nk = 0;
        if (lead) p.st.j_end[ray] = je;
        if (lead) p.st.acc[ray] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lead) p.st.tw[ray] = make_float2(1.f, 0.f);
    } else {
        const float4 o4 = p.st.orig[ray], d4 = p.st.dir[ray];
        o = make_float3(o4.x, o4.y, o4.z);
        d = make_float3(d4.x, d4.y, d4.z);
        jn = p.st.j_next[ray];
        je = p.st.j_end[ray];
        nk = p.st.n_kept[ray];
    }
    return true;
}

// First sample past the empty space around sample j's voxel (ix, iy, iz)
// (clamped to je): out of an empty voxel to the first sample past its exit
// face; out of an empty brick to the first sample past the exit of the cube
// of bricks within Chebyshev distance dd - 1 (all empty; voxel units, clamped
// to the grid), minus one sample so that a sample rounded onto that face is
// still tested.  One code path for both jumps (fewer divergent branches).
__device__ __forceinline__ uint32_t empty_jump(const GridDev &g, int dd, int ix, int iy, int iz, float ogx, float ogy,
                                               float ogz, float dgx, float dgy, float dgz, float idx, float idy,
                                               float idz, float inv_delta, uint32_t je)
{
    const int bxi = ix >> kBrickShift, byi = iy >> kBrickShift, bzi = iz >> kBrickShift;
    float ex, ey, ez, back;
    if (dd > 0) {
        const int r = dd - 1;
        ex = dgx > 0.f ? (float)(min(bxi + r + 1, g.bx) << kBrickShift) : (float)(max(bxi - r, 0) << kBrickShift);
        ey = dgy > 0.f ? (float)(min(byi + r + 1, g.by) << kBrickShift) : (float)(max(byi - r, 0) << kBrickShift);
        ez = dgz > 0.f ? (float)(min(bzi + r + 1, g.bz) << kBrickShift) : (float)(max(bzi - r, 0) << kBrickShift);
        back = 1.0f;
    } else {
        ex = dgx > 0.f ? (float)(ix + 1) : (float)ix;
        ey = dgy > 0.f ? (float)(iy + 1) : (float)iy;
        ez = dgz > 0.f ? (float)(iz + 1) : (float)iz;
        back = 0.0f;
    }
    float te = 3.0e38f;
    if (dgx != 0.f) te = fminf(te, (ex - ogx) * idx);
    if (dgy != 0.f) te = fminf(te, (ey - ogy) * idy);
    if (dgz != 0.f) te = fminf(te, (ez - ogz) * idz);
    const float jf = ceilf(te * inv_delta - 0.5f) - back;
    return jf > (float)je ? je : (jf > 0.f ? (uint32_t)jf : 0u);
}

// Sample j of a ray sits at t_j = (j + 1/2) delta and is kept iff its voxel
// floor((o + t_j d - origin) / vox) is inside the grid and occupied.  The
// walk tests samples in occupied voxels one by one and jumps over empty
// space: out of an empty voxel to the first sample past its exit face, and
// out of an empty brick to the first sample past the exit of the largest
// empty cube of bricks around it (from the brick distance map), minus one
// sample so that a sample rounded onto that face is still tested.  Emitted
// records also feed a per-block field histogram for the bucketing.  Launched
// with about one thread per ray (the stride loop covers larger requests).
__global__ void __launch_bounds__(256) k_march(GridDev g, MarchParams p)
{
    extern __shared__ uint32_t s_hist[];      // per-block field histogram (when p.hist)
    if (p.hist) {
        for (int f = threadIdx.x; f < g.n_fields; f += blockDim.x) s_hist[f] = 0;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.live_count != nullptr) {
        // the count slot the composite of this round fills is the one the
        // previous round read: clear it for reuse
        uint32_t *other = (p.live_count == &p.ctr->live_count[0]) ? &p.ctr->live_count[1] : &p.ctr->live_count[0];
        *other = 0u;
    } else if (blockIdx.x == 0 && threadIdx.x == 0 && p.init && !p.flat) {
        p.ctr->live_count[1] = 0u;
    }
    const uint32_t n_live = p.live_count ? *p.live_count : p.n_rays;
    const uint32_t stride = gridDim.x * blockDim.x;
    const float delta = p.delta;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_live; i += stride) {
        const uint32_t ray = p.live ? p.live[i] : i;
        float3 o, d;
        uint32_t jn, je, nk;
        if (!ray_begin(g, p, i, ray, true, o, d, jn, je, nk)) continue;
        const float ogx = (o.x - g.origin[0]) * g.inv_vox, ogy = (o.y - g.origin[1]) * g.inv_vox,
                    ogz = (o.z - g.origin[2]) * g.inv_vox;
        const float dgx = d.x * g.inv_vox, dgy = d.y * g.inv_vox, dgz = d.z * g.inv_vox;
        const float idx = 1.0f / dgx, idy = 1.0f / dgy, idz = 1.0f / dgz;
        const float inv_delta = 1.0f / delta;   // (the jump's sample index: a product, not a division per step)
        uint32_t em = 0;
        const uint32_t R = (uint32_t)p.R, n_max = (uint32_t)p.n_max;
        // records this round may keep (the round's size and the ray's budget in one bound)
        const uint32_t lim = nk < n_max ? min(R, n_max - nk) : 0u;
        // slot of record em: s0 + em * s_step
        const uint32_t s0 = p.flat ? i * R : slot_of(i, 0u, R), s_step = p.flat ? 1u : 32u;
        // the histogram takes runs of one field (a ray crosses few fields),
        // not one shared-memory atomic per record
        uint32_t run_f = 0u, run_n = 0u;
        while (jn < je && em < lim) {
            const float t = ((float)jn + 0.5f) * delta;
            const float gxf = fmaf(t, dgx, ogx), gyf = fmaf(t, dgy, ogy), gzf = fmaf(t, dgz, ogz);
            const int ix = __float2int_rd(gxf), iy = __float2int_rd(gyf), iz = __float2int_rd(gzf);
            if ((unsigned)ix >= (unsigned)g.gx || (unsigned)iy >= (unsigned)g.gy || (unsigned)iz >= (unsigned)g.gz) {
                ++jn;
                continue;
            }
            const int bxi = ix >> kBrickShift, byi = iy >> kBrickShift, bzi = iz >> kBrickShift;
            // the brick's distance, the voxel's bit word and its rank prefix
            // side by side (the word is inside the grid), not one after the other
            // (grids are at most 2048^3 voxels: word and brick indices fit 32 bits)
            const uint32_t wi = ((uint32_t)iz * (uint32_t)g.gy + (uint32_t)iy) * (uint32_t)g.wpr + ((uint32_t)ix >> 5);
            const int dd = __ldg(&g.brick_dist[((uint32_t)bzi * (uint32_t)g.by + (uint32_t)byi) * (uint32_t)g.bx +
                                               (uint32_t)bxi]);
            const uint32_t wraw = __ldg(&g.bits[wi]);
            const uint32_t pre = __ldg(&g.prefix[wi]);
            const uint32_t b = (uint32_t)(ix & 31);
            const uint32_t w = dd > 0 ? 0u : wraw;
            if (!((w >> b) & 1u)) {
                const uint32_t jj =
                    empty_jump(g, dd, ix, iy, iz, ogx, ogy, ogz, dgx, dgy, dgz, idx, idy, idz, inv_delta, je);
                jn = jj > jn + 1 ? jj : jn + 1;
                continue;
            }
            {
                const uint32_t rank = pre + (uint32_t)__popc(w & ((1u << b) - 1u));
                uint32_t f = __ldg(&g.labels[rank]);
                if (f >= (uint32_t)g.n_fields) {
                    atomicOr(&p.ctr->status, kStatusBadLabel);
                    f = 0;
                }
                p.recs[s0 + em * s_step] = jn | (f << 16);
                if (p.hist) {
                    if (f != run_f) {
                        if (run_n) atomicAdd(&s_hist[run_f], run_n);
                        run_f = f;
                        run_n = 0u;
                    }
                    ++run_n;
                }
                ++em;
            }
            ++jn;
        }
        if (p.hist && run_n) atomicAdd(&s_hist[run_f], run_n);
        p.cnt[i] = em;
        p.st.j_next[ray] = jn;
        p.st.n_kept[ray] = nk + em;
    }
    if (p.hist) {
        __syncthreads();
        for (int f = threadIdx.x; f < g.n_fields; f += blockDim.x)
            if (s_hist[f]) atomicAdd(&p.hist[f], s_hist[f]);
    }
}


}  // namespace

void launch_grid_prefix(const uint32_t *bits, uint32_t *prefix, uint32_t *block_sums, int64_t n_words,
                        cudaStream_t s)
{
    const int64_t nb = (n_words + 4095) / 4096;
    k_prefix_local<<<(unsigned)nb, 1024, 0, s>>>(bits, prefix, block_sums, n_words);
    k_prefix_blocks<<<1, 1024, 0, s>>>(block_sums, nb);
    k_prefix_add<<<(unsigned)((n_words + 255) / 256), 256, 0, s>>>(prefix, block_sums, n_words);
}

void launch_brick_dist(GridDev g, uint8_t *occ, uint16_t *t0, uint16_t *t1, uint8_t *dist, cudaStream_t s)
{
    const int64_t n = (int64_t)g.bx * g.by * g.bz;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_brick_occ<<<blocks, 256, 0, s>>>(g, occ);
    k_brick_dist<<<blocks, 256, 0, s>>>(g, 0, occ, nullptr, t0);
    k_brick_dist<<<blocks, 256, 0, s>>>(g, 1, occ, t0, t1);
    k_brick_dist<<<blocks, 256, 0, s>>>(g, 2, occ, t1, t0);
    k_brick_final<<<blocks, 256, 0, s>>>(n, t0, dist);
}

void launch_march(const GridDev &g, const MarchParams &p, int grid, cudaStream_t s)
{
    k_march<<<grid, 256, p.hist ? (size_t)g.n_fields * sizeof(uint32_t) : 0, s>>>(g, p);
}

}  // namespace roam
