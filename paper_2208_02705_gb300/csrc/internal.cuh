// Internal declarations of the roam CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "roam.h"

namespace roam {

constexpr int kPeX = 63;          // 3 + 2*3*10 position features
constexpr int kPeD = 27;          // 3 + 2*3*4 direction features

// Kernel attributes are per device: a launcher raises a kernel's dynamic
// shared-memory limit on the current device the first time it needs more
// (`cached` holds the limit set so far per device ordinal; ordinals past
// the table are set on every launch).
constexpr int kMaxDevices = 64;
inline void raise_smem_limit(const void *kernel, int bytes, int (&cached)[kMaxDevices])
{
    int dev = -1;
    cudaGetDevice(&dev);
    const bool tracked = dev >= 0 && dev < kMaxDevices;
    if (tracked && cached[dev] >= bytes) return;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess && tracked)
        cached[dev] = bytes;
}
constexpr int kBrickShift = 3;    // 8^3-voxel bricks for empty-space skipping
constexpr int kMaxViews = 256;

// device status word bits
constexpr uint32_t kStatusBadLabel = 1u;
constexpr uint32_t kStatusTimeout = 2u;
constexpr uint32_t kStatusBadSample = 4u;

// Camera as the kernels use it.
struct DevCamera {
    int model, width, height, pad;
    float R[9];
    float o[3];
    float inv_f;          // perspective: 1 / focal length in pixels
    uint32_t pix_start;   // first global pixel index of this view
    double inv_f64;       // the same focal factor in FP64 (FP32 render path)
};

struct GridDev {
    int gx, gy, gz, wpr;          // wpr = gx / 32
    int bx, by, bz;               // brick grid (8^3 voxels per brick)
    float origin[3];
    float vox, inv_vox;
    const uint32_t *bits;         // [gz][gy][wpr]
    const uint32_t *prefix;       // exclusive popcount before each word
    const uint8_t *brick_dist;    // [bz][by][bx] Chebyshev distance (bricks) to an occupied brick, 0 = occupied
    const uint16_t *labels;       // field of each occupied voxel, rank order
    int n_fields;
};

// World direction of pixel `pix` of a view in FP64 (Eq. 2 and Eq. 3 for
// equirectangular views, the pinhole model for perspective ones).
__device__ __forceinline__ void make_ray64(const DevCamera &c, uint32_t pix, double3 &d)
{
    const uint32_t u = pix % (uint32_t)c.width, v = pix / (uint32_t)c.width;
    double d0, d1, d2;
    if (c.model == ROAM_EQUIRECT) {
        const double pu = 2.0 * (((double)u + 0.5) / (double)c.width) - 1.0;
        const double tv = 0.5 - ((double)v + 0.5) / (double)c.height;
        double sp, cp, st, ct;
        sincospi(pu, &sp, &cp);
        sincospi(tv, &st, &ct);
        d0 = ct * sp;
        d1 = -st;
        d2 = ct * cp;
    } else {
        const double x = ((double)u + 0.5 - 0.5 * (double)c.width) * c.inv_f64;
        const double y = ((double)v + 0.5 - 0.5 * (double)c.height) * c.inv_f64;
        const double n = 1.0 / sqrt(x * x + y * y + 1.0);
        d0 = x * n;
        d1 = y * n;
        d2 = n;
    }
    d.x = (double)c.R[0] * d0 + (double)c.R[1] * d1 + (double)c.R[2] * d2;
    d.y = (double)c.R[3] * d0 + (double)c.R[4] * d1 + (double)c.R[5] * d2;
    d.z = (double)c.R[6] * d0 + (double)c.R[7] * d1 + (double)c.R[8] * d2;
}

// Device counters of one render / training pass.
struct Counters {
    uint32_t live_count[2];
    uint32_t n_tiles;
    uint32_t status;
    unsigned long long n_samples;   // samples evaluated through the MLPs
    unsigned long long n_used;      // samples composited (up to termination)
    uint32_t fields_hit;
    uint32_t pad;
    uint32_t class_tiles[4];        // first tile of width class c; entry n_classes = n_tiles
};

// Width classes of a mixed-width field set: internal field ids are grouped by
// class; first[c] = first internal field of class c (n_fields past the last
// class).  A single width is one class: {0, F, F, F}.  group[c] > 0: the tile
// runs of class c's fields are padded to multiples of group[c] tiles (its
// MLP kernel's tiles in flight) instead of the bucketing call's own group.
struct ClassBounds {
    int first[4];
    int group[4];
};

// Ray state, structure of arrays, indexed by ray id.
struct RayState {
    float4 *orig;       // o (xyz), w unused
    float4 *dir;        // d (xyz), w unused
    float4 *dir_lo;     // FP64 direction minus d (FP32 render path only)
    uint32_t *j_next;   // next sample index to test
    uint32_t *j_end;    // first sample index past the grid
    uint32_t *n_kept;   // kept samples so far
    float4 *acc;        // (r, g, b, depth) accumulated
    float2 *tw;         // (transmittance, sum of weights)
};

// Slot of the k-th sample of live ray i in a round of R samples per ray:
// 32 consecutive rays share a 32-wide column so that per-k accesses coalesce.
__host__ __device__ inline uint32_t slot_of(uint32_t i, uint32_t k, uint32_t R)
{
    return ((i >> 5) * R + k) * 32u + (i & 31u);
}

// Inverse of the column part of slot_of: the 32-ray group of slot column col
// (= slot >> 5), i.e. col / R.  Power-of-two round sizes (the ones the round
// tuner picks) take a shift instead of the integer division.
__device__ __forceinline__ uint32_t group_of(uint32_t col, uint32_t R)
{
    return (R & (R - 1u)) == 0u ? col >> (31 - __clz(R)) : col / R;
}

struct MarchParams {
    const DevCamera *cams;
    int n_views;
    const uint32_t *rays;       // (view, pixel) pairs or nullptr (all pixels)
    uint32_t n_rays;
    const uint32_t *live;       // live ray ids or nullptr (round 0: identity)
    const uint32_t *live_count; // device count or nullptr (n_rays)
    int R;                      // samples per ray this round (flat: row length)
    int n_max;
    float delta;
    int init;                   // compute rays and reset state
    int flat;                   // recs laid out [n_rays][R] instead of slots
    int accurate;               // also keep the FP64 direction residual
    RayState st;
    uint32_t *cnt;              // per live index: samples emitted
    uint32_t *recs;             // j | field << 16
    Counters *ctr;
    uint32_t *hist;             // if set: field histogram of the emitted samples (added to)
};

// Sample source of the MLP kernels.
struct SampleSrc {
    int mode;                   // 0: render slots, 1: direct points
    // render slots
    const uint32_t *recs;
    const uint32_t *live;
    const uint32_t *live_count;
    int R;
    RayState st;
    float delta;
    int accurate;               // sample positions from the direction residual
    // direct points
    const float *p;             // [n][3]
    const float *d;             // [n][3]
};

struct Tile {
    uint32_t field, start, count, pad;
};

struct BucketBufs {
    uint32_t *hist;       // [F]
    uint32_t *offsets;    // [F + 1]
    uint32_t *cursor;     // [F]
    Tile *tiles;          // [max tiles]
    uint32_t *sorted;     // [max samples]
    uint32_t *tile_off;   // [F + 1] first tile of each field, or nullptr (tiles built by the scan)
};

struct MlpWeights {
    int W, H, act, n_fields;
    int64_t P;                 // parameters per field (API layout)
    float sigma_scale;
    const float *w32;          // FP32 masters [F][P]
    const float *wt;           // FP32 transposed/padded copy for SIMT [F][Pt]
    int64_t Pt;
    const float *wr;           // FP32 row-padded copy ([out][round4(in)]) for the SIMT adjoint [F][Pr]
    int64_t Pr;
    const void *wimg;          // BF16 tensor-core images [F][img_bytes]
    int64_t img_bytes;
    const void *wimg8;         // FP8 E4M3 tensor-core images [F][img8_bytes]
    int64_t img8_bytes;
    int cls;                   // width class: the kernels take tiles [class_tiles[cls], class_tiles[cls + 1])
    int field_base;            // first internal field id of the class (row 0 of the per-class arrays)
    const float *affine;       // [F][6]
    // self-test of the bounded waits (roam_selftest_wait_timeout): the limit of
    // every wait of the tensor-core kernel in ns (0: the 2 s default), and
    // whether the weight-image copies are withheld so that those waits run out
    unsigned long long wait_ns;
    int withhold_image;
};

// ---- kernels launched from the API layer -------------------------------

void launch_grid_prefix(const uint32_t *bits, uint32_t *prefix, uint32_t *block_sums,
                        int64_t n_words, cudaStream_t s);
void launch_brick_dist(GridDev g, uint8_t *occ, uint16_t *t0, uint16_t *t1, uint8_t *dist, cudaStream_t s);
void launch_march(const GridDev &g, const MarchParams &p, int grid, cudaStream_t s);
struct TeacherAffine {
    float v[6];      // global position -> [-1, 1]^3: scale xyz, offset xyz
};
int64_t teacher_param_count();
int64_t teacher_image_bytes();
// the caller's layout -> the tensor-core image and the transposed FP32 layers
void launch_teacher_pack(const float *w, uint8_t *img, float *wt, cudaStream_t s);
void launch_teacher_tc(const uint8_t *img, TeacherAffine aff, int64_t n, const float *p, const float *d, float4 *out,
                       uint32_t *status, int n_sm, cudaStream_t s);
void launch_teacher_simt(const float *wt, TeacherAffine aff, int64_t n, const float *p, const float *d, float4 *out,
                         int n_sm, cudaStream_t s);
void launch_distill_loss(int64_t n, const float4 *student, const float4 *teacher, float I, float4 *dl, float *loss,
                         cudaStream_t s);
size_t assign_scratch_bytes();
void launch_assign(const uint32_t *bits, const uint32_t *prefix, int64_t n_words, int gx, int gy, uint32_t S, int n,
                   uint32_t *vox, uint16_t *field, int32_t *boxes, void *scratch, int n_sm, cudaStream_t s);
uint32_t assign_status(const void *scratch);
void launch_occupancy_scan(const GridDev &g, const DevCamera *cams, int view, int n_pix, const float *depth,
                           const float *opacity, const roam_occ_params &q, uint32_t *hit, uint32_t *free_bits,
                           float *logit, uint32_t *bits, int n_sm, cudaStream_t s);
// tiles of `tile` samples, every non-empty field's tile count rounded up to a
// multiple of `group`; with hist_ready the histogram is already in b.hist
void launch_bucket_ready(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count,
                         uint32_t n_fixed, int R, int group, int n_fields, int tile, const BucketBufs &b,
                         Counters *ctr, int grid, cudaStream_t s, ClassBounds cb);
void launch_bucket(const uint32_t *cnt, const uint32_t *recs, const uint32_t *live_count,
                   uint32_t n_fixed, int R, int group, const uint16_t *keys16,
                   int n_fields, int tile, const BucketBufs &b, Counters *ctr, int grid,
                   cudaStream_t s, ClassBounds cb);
void launch_mlp_simt(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b,
                     Counters *ctr, float4 *out, int n_sm, cudaStream_t s);
void launch_pack_simt(const float *w32, int n_fields, int W, int H, int64_t P, float *wt,
                      int64_t Pt, cudaStream_t s);
int64_t simt_transposed_size(int W, int H);
void launch_composite_round(const MarchParams &mp, const float4 *sr, uint32_t *next_live,
                            uint32_t *next_count, float t_stop, const float *bg, float *rgb,
                            float *depth, float *opacity, int grid, cudaStream_t s);
void launch_composite_flat(int64_t n_rays, int n_max, const uint32_t *count, const float4 *sr,
                           const float *t, float delta, float t_stop, const float *bg, float *rgb,
                           float *depth, float *opacity, uint32_t *n_used, cudaStream_t s);

void launch_composite_bwd(int64_t n_rays, int R, const uint32_t *cnt, const uint32_t *recs, const float4 *sr,
                          float delta, float t_stop, const float *bg, const float *dl_drgb, float4 *gsr,
                          uint32_t *cnt_used, uint32_t *hist, int n_fields, cudaStream_t s);
void launch_mlp_bwd_simt(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr,
                         const float4 *gsr, float *grad, int grid, cudaStream_t s);
bool mlp_bwd_supported(int W, int H);
// tcgen05 BF16 adjoint (W <= 64 and the shared-memory budget: W = 32 with
// H <= 4, W = 64 with H <= 3); needs the BF16 weight images
bool mlp_bwd_tc_supported(int W, int H);
void launch_mlp_bwd_tc(const MlpWeights &w, const SampleSrc &src, const BucketBufs &b, Counters *ctr,
                       const float4 *gsr, float *grad, int n_sm, cudaStream_t s);
void launch_pack_rows(const float *w32, int n_fields, int W, int H, int64_t P, float *wr, int64_t Pr,
                      cudaStream_t s);
int64_t rows_padded_size(int W, int H);
void launch_l2_loss(int64_t n_rays, const float *rgb, const float *target, float norm, float *dl, float *loss,
                    cudaStream_t s);
void launch_adam(float *w32, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                 float eps, float bc1, float bc2, cudaStream_t s);

// sets the calling thread's roam_last_error() message
void set_error_message(const char *msg);

// tcgen05 BF16 path
bool tc_supported(int W, int H, bool f8);
int64_t tc_image_bytes(int W, int H, bool f8);
int tc_tile_samples();
int tc_tile_group(int W, bool f8);
void launch_pack_tc(const float *w32, int n_fields, int W, int H, int64_t P, void *wimg, int64_t img_bytes, bool f8,
                    cudaStream_t s);
// Adam fused with the BF16 image refresh (W <= 64); false: not available for this shape
bool launch_adam_tc(float *w32, float *m, float *v, const float *g, int n_fields, int W, int H, int64_t P, void *wimg,
                    int64_t img_bytes, float lr, float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s);
void launch_mlp_tc(const MlpWeights &w, bool f8, const SampleSrc &src, const BucketBufs &b, Counters *ctr,
                   float4 *out, int n_sm, cudaStream_t s);

}  // namespace roam
