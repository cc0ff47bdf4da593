// C ABI of the roam library: argument validation, device memory of the
// context, and the order of kernel launches for each entry point.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <vector>


#include "internal.cuh"

using namespace roam;

namespace {

thread_local char g_err[512] = "";

roam_status fail(roam_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define ROAM_CUDA(x)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) return fail(ROAM_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

#define ROAM_TRY(x)                          \
    do {                                     \
        roam_status s_ = (x);                \
        if (s_ != ROAM_OK) return s_;        \
    } while (0)

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
};

// bumped by every device (re)allocation: a captured render graph holds raw
// pointers and is re-captured when this moves
std::atomic<uint64_t> g_alloc_gen{0};

template <class T>
roam_status ensure(DBuf<T> &b, size_t n)
{
    if (n == 0) n = 1;
    if (b.p && b.n >= n) return ROAM_OK;
    ++g_alloc_gen;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    if (cudaMalloc(&b.p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(ROAM_ERR_OOM, "device allocation of %zu bytes failed", n * sizeof(T));
    }
    b.n = n;
    return ROAM_OK;
}

template <class T>
void release(DBuf<T> &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

bool finite(float x) { return std::isfinite(x); }

__global__ void k_check_finite(const float *w, int64_t n, uint32_t *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(w[i])) { atomicOr(bad, 1u); return; }
}

__global__ void k_check_labels(const uint16_t *lab, int64_t n, int n_fields, uint32_t *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (lab[i] >= n_fields) { atomicOr(bad, 1u); return; }
}

int64_t param_count(int W, int H)
{
    return (int64_t)W * kPeX + W + (int64_t)(H - 1) * ((int64_t)W * W + W) + (int64_t)(1 + W) * W + (1 + W) +
           (int64_t)W * (W + kPeD) + W + 3 * (int64_t)W + 3;
}

// Weights of the fields of one width: FP32 masters and the derived copies.
struct WSet {
    int W = 0, first = 0, n = 0;        // width; internal field ids [first, first + n)
    int64_t P = 0, Pt = 0, Pr = 0, img_bytes = 0, img8_bytes = 0;
    bool tc_ok = false, tc8_ok = false;
    uint32_t stale = 0;                 // derived copies older than w32 (kStale* bits)
    DBuf<float> w32, wt, wr;
    DBuf<uint8_t> wimg, wimg8;
};

}  // namespace

struct roam_ctx {
    int device = 0, n_sm = 0;
    // occupancy grid
    bool has_grid = false;
    roam_grid_desc gd{};
    GridDev g{};
    int64_t n_words = 0, n_occ = 0;
    DBuf<uint32_t> bits, prefix, block_sums;
    DBuf<uint8_t> brick_occ, brick_dist;
    DBuf<uint16_t> brick_t0, brick_t1;
    // fields
    bool has_fields = false;
    int n_fields = 0;
    DBuf<uint16_t> labels;
    DBuf<float> affine;
    // weights
    bool has_weights = false;
    roam_mlp_desc md{};
    // one weight set per width class; internal field ids are grouped by class
    // (a permutation of the caller's ids when the widths are mixed)
    WSet ws[3];
    int n_ws = 0;
    ClassBounds cb{{0, 0, 0, 0}, {0, 0, 0, 0}};
    bool permuted = false;
    DBuf<uint16_t> perm, inv, labels_orig, keys_tmp;
    std::vector<float> affine_orig;
    std::vector<int32_t> widths;            // caller's field order
    DBuf<float> adam_m, adam_v;
    bool adam_fresh = true;
    // per-call workspace
    DBuf<float4> orig, dir, dir_lo, acc, sr, gsr;
    DBuf<float2> tw;
    DBuf<uint32_t> j_next, j_end, n_kept, live0, live1, cnt, recs, sorted, hist, offsets, cursor, scratch_u32, tile_off;
    DBuf<Tile> tiles;
    DBuf<float> o_rgb, o_depth, o_op;
    DBuf<DevCamera> cams;
    DBuf<uint32_t> occ_hit, occ_free;        // occupancy update marks (per voxel, per 32 voxels)
    DBuf<uint32_t> assign_vox;               // occupied voxels' linear indices (field assignment)
    // distillation teacher (global 360NeRF)
    bool has_teacher = false;
    DBuf<uint8_t> teacher_img;              // BF16 tensor-core image (+ FP32 tables)
    DBuf<float> teacher_wt, teacher_ws;      // FP32 transposed layers; the caller's layout while loading
    TeacherAffine teacher_aff{};
    DBuf<uint8_t> assign_scratch;
    // pinned staging of the camera uploads: a ring, so that consecutive calls
    // (e.g. one per view) do not wait for each other's copies
    static constexpr int kCamRing = 8;
    DevCamera *h_cams_ring = nullptr;        // [kCamRing][kMaxViews]
    DevCamera *h_cams = nullptr;             // the slot filled by the current call
    cudaEvent_t cam_ev[kCamRing] = {};
    bool cam_pending[kCamRing] = {};
    int cam_slot = 0;
    std::vector<DevCamera> cams_dev;        // what the device camera buffer holds (the last copy)
    int cams_dev_n = 0;                     // its number of views (0: nothing copied yet)
    int cams_dev_slot = -1;                 // the ring slot whose event follows that copy
    Counters *ctr = nullptr;        // the last render / training forward (roam_get_stats)
    Counters *aux = nullptr;        // the other calls (single steps, backward passes): ctr + 1
    Counters *h_ctr = nullptr;
    uint32_t *d_flag = nullptr;
    cudaStream_t last = nullptr;
    int n_views = 0;
    int64_t last_rays = 0;
    int last_rounds = 0;
    // per-kernel event timing
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::vector<std::pair<int64_t, double>> prof_acc;
    // CUDA-graph replay of roam_render
    uint64_t gen = 0;                   // bumped whenever the grid, fields or weights are reloaded
    cudaGraphExec_t gexec = nullptr;
    std::vector<uint64_t> gkey;
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // training: state kept from roam_train_forward for roam_train_backward
    int64_t train_rays = 0;
    int train_R = 0;
    roam_render_opts train_opts{};
    int tile_pad = 0;                   // roam_set_tile_padding (0: each kernel's own tiles in flight)
    DBuf<float> selftest;               // roam_selftest_wait_timeout: points, directions, outputs
};

namespace {

const char *const kProfNames[] = {"march", "bucket", "mlp_f32_simt", "mlp_bf16_tcgen05", "composite",
                                  "composite_bwd", "mlp_bwd", "adam", "mlp_fp8_tcgen05", "mlp_bwd_bf16_tcgen05",
                                  "teacher_bf16_tcgen05", "teacher_f32_simt"};
constexpr int kProfKinds = (int)(sizeof(kProfNames) / sizeof(kProfNames[0]));
enum { P_MARCH, P_BUCKET, P_MLP_F32, P_MLP_BF16, P_COMPOSITE, P_COMPOSITE_BWD, P_MLP_BWD, P_ADAM, P_MLP_FP8,
       P_MLP_BWD_TC, P_TEACHER_TC, P_TEACHER_F32 };

cudaEvent_t pool_event(roam_ctx *c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch with events when profiling is on.
struct ProfScope {
    roam_ctx *c;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    ProfScope(roam_ctx *c_, int kind_, cudaStream_t s_) : c(c_), kind(kind_), s(s_)
    {
        if (c->prof) {
            a = pool_event(c);
            cudaEventRecord(a, s);
        }
    }
    ~ProfScope()
    {
        if (a) {
            cudaEvent_t b = pool_event(c);
            cudaEventRecord(b, s);
            c->prof_pending.push_back({kind, {a, b}});
        }
    }
};

roam_status set_dev(roam_ctx *c)
{
    if (!c) return fail(ROAM_ERR_ARG, "null context");
    ROAM_CUDA(cudaSetDevice(c->device));
    return ROAM_OK;
}

roam_status launched(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ROAM_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return ROAM_OK;
}

roam_status status_of(uint32_t st)
{
    if (st & kStatusTimeout) return fail(ROAM_ERR_TIMEOUT, "a device-side wait hit its iteration limit");
    if (st & (kStatusBadLabel | kStatusBadSample)) return fail(ROAM_ERR_DATA, "device found an invalid field id or sample");
    return ROAM_OK;
}

int grid_blocks(const roam_ctx *c, int per_sm) { return c->n_sm * per_sm; }

// The march runs one thread per ray (blocks of 256): rays differ widely in
// length, and many small blocks balance the SMs far better than a few
// blocks striding over many rays each (measured: half the march time).
int march_grid(int64_t n_rays) { return (int)std::max<int64_t>(1, std::min<int64_t>((n_rays + 255) / 256, 0x7fffffff)); }

MlpWeights weights_of(const roam_ctx *c, int k = 0)
{
    const WSet &q = c->ws[k];
    MlpWeights w{};
    w.W = q.W;
    w.H = c->md.n_hidden;
    w.act = c->md.density_act;
    w.n_fields = q.n;
    w.P = q.P;
    w.sigma_scale = c->md.sigma_scale;
    w.w32 = q.w32.p;
    w.wt = q.wt.p;
    w.Pt = q.Pt;
    w.wr = q.wr.p;
    w.Pr = q.Pr;
    w.wimg = q.wimg.p;
    w.img_bytes = q.img_bytes;
    w.wimg8 = q.wimg8.p;
    w.img8_bytes = q.img8_bytes;
    w.cls = k;
    w.field_base = q.first;
    w.affine = c->affine.p;
    return w;
}

bool all_tc(const roam_ctx *c, bool f8)
{
    for (int k = 0; k < c->n_ws; ++k)
        if (!(f8 ? c->ws[k].tc8_ok : c->ws[k].tc_ok)) return false;
    return c->n_ws > 0;
}

// Derived weight copies that an Adam step left stale are rebuilt before the
// first launch that reads them: the SIMT forward's transposed copy (FP32
// forward or SIMT adjoint), the SIMT adjoint's row-padded copy, the FP8
// images.  Adam rebuilds the BF16 images itself.
constexpr uint32_t kStaleWt = 1u, kStaleWr = 2u, kStaleImg8 = 4u;

roam_status refresh(roam_ctx *c, int precision, bool simt_adjoint, cudaStream_t s)
{
    for (int k = 0; k < c->n_ws; ++k) {
        WSet &q = c->ws[k];
        if (!q.stale) continue;
        const int H = c->md.n_hidden;
        if ((precision == ROAM_F32 || simt_adjoint) && (q.stale & kStaleWt)) {
            launch_pack_simt(q.w32.p, q.n, q.W, H, q.P, q.wt.p, q.Pt, s);
            q.stale &= ~kStaleWt;
        }
        if (simt_adjoint && (q.stale & kStaleWr)) {
            launch_pack_rows(q.w32.p, q.n, q.W, H, q.P, q.wr.p, q.Pr, s);
            q.stale &= ~kStaleWr;
        }
        if (precision == ROAM_FP8 && (q.stale & kStaleImg8)) {
            launch_pack_tc(q.w32.p, q.n, q.W, H, q.P, q.wimg8.p, q.img8_bytes, true, s);
            q.stale &= ~kStaleImg8;
        }
        ROAM_TRY(launched("weight refresh"));
    }
    return ROAM_OK;
}

roam_status check_ready(const roam_ctx *c)
{
    if (!c->has_grid) return fail(ROAM_ERR_STATE, "no occupancy grid loaded");
    if (!c->has_fields) return fail(ROAM_ERR_STATE, "no field labels loaded");
    if (!c->has_weights) return fail(ROAM_ERR_STATE, "no weights loaded");
    return ROAM_OK;
}

roam_status check_opts(const roam_ctx *c, const roam_render_opts *o)
{
    if (!o) return fail(ROAM_ERR_ARG, "null render options");
    if (!(o->delta > 0.f) || !finite(o->delta)) return fail(ROAM_ERR_ARG, "delta must be positive");
    if (o->n_max < 1 || o->n_max > 1024) return fail(ROAM_ERR_ARG, "n_max must be in [1, 1024]");
    if (!(o->t_stop >= 0.f && o->t_stop < 1.f)) return fail(ROAM_ERR_ARG, "t_stop must be in [0, 1)");
    for (int i = 0; i < 3; ++i)
        if (!finite(o->bg[i])) return fail(ROAM_ERR_ARG, "background must be finite");
    if (o->precision != ROAM_F32 && o->precision != ROAM_BF16 && o->precision != ROAM_FP8)
        return fail(ROAM_ERR_ARG, "unknown precision");
    if ((o->precision == ROAM_BF16 && !all_tc(c, false)) || (o->precision == ROAM_FP8 && !all_tc(c, true)))
        return fail(ROAM_ERR_UNSUPPORTED, "tensor-core path not available for W=%d H=%d", c->md.width, c->md.n_hidden);
    if (o->round_size < 0) return fail(ROAM_ERR_ARG, "round_size must be >= 0");
    if (o->first_round_size < 0) return fail(ROAM_ERR_ARG, "first_round_size must be >= 0");
    if (o->use_graph != 0 && o->use_graph != 1) return fail(ROAM_ERR_ARG, "use_graph must be 0 or 1");
    return ROAM_OK;
}

// Validates the cameras and copies them to the device; *n_pix = all pixels.
roam_status upload_cams(roam_ctx *c, const roam_camera *cams, int n_views, float delta, int64_t *n_pix,
                        cudaStream_t s)
{
    if (!cams) return fail(ROAM_ERR_ARG, "null cameras");
    if (n_views < 1 || n_views > kMaxViews) return fail(ROAM_ERR_ARG, "n_views must be in [1, %d]", kMaxViews);
    const int slot = c->cam_slot;
    c->cam_slot = (slot + 1) % roam_ctx::kCamRing;
    if (c->cam_pending[slot]) {
        cudaEventSynchronize(c->cam_ev[slot]);   // the copy that last used this staging slot
        c->cam_pending[slot] = false;
    }
    c->h_cams = c->h_cams_ring + (size_t)slot * kMaxViews;
    int64_t total = 0;
    const float ext[3] = {c->gd.dims[0] * c->gd.vox, c->gd.dims[1] * c->gd.vox, c->gd.dims[2] * c->gd.vox};
    for (int v = 0; v < n_views; ++v) {
        const roam_camera &k = cams[v];
        if (k.model != ROAM_EQUIRECT && k.model != ROAM_PERSPECTIVE) return fail(ROAM_ERR_ARG, "camera %d: bad model", v);
        if (k.width < 1 || k.height < 1 || k.width > 65536 || k.height > 65536)
            return fail(ROAM_ERR_ARG, "camera %d: bad size", v);
        if (k.model == ROAM_PERSPECTIVE && !(k.fov_h > 0.f && k.fov_h < 3.1f))
            return fail(ROAM_ERR_ARG, "camera %d: fov must be in (0, 3.1) rad", v);
        for (int i = 0; i < 9; ++i)
            if (!finite(k.R[i])) return fail(ROAM_ERR_ARG, "camera %d: non-finite rotation", v);
        double tmax = 0.0;
        for (int i = 0; i < 3; ++i)
            if (!finite(k.o[i])) return fail(ROAM_ERR_ARG, "camera %d: non-finite centre", v);
        for (int corner = 0; corner < 8; ++corner) {
            double d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const double e = c->gd.origin[a] + ((corner >> a) & 1) * ext[a] - k.o[a];
                d2 += e * e;
            }
            tmax = std::max(tmax, std::sqrt(d2));
        }
        if (tmax / delta + 8.0 > 65535.0)
            return fail(ROAM_ERR_ARG, "camera %d: more than 65535 sample positions per ray (delta too small)", v);
        DevCamera &d = c->h_cams[v];
        memset(&d, 0, sizeof(d));
        d.model = k.model;
        d.width = k.width;
        d.height = k.height;
        memcpy(d.R, k.R, sizeof(d.R));
        memcpy(d.o, k.o, sizeof(d.o));
        d.inv_f64 = k.model == ROAM_PERSPECTIVE ? std::tan(0.5 * (double)k.fov_h) / (0.5 * k.width) : 0.0;
        d.inv_f = (float)d.inv_f64;
        d.pix_start = (uint32_t)total;
        total += (int64_t)k.width * k.height;
        if (total > (int64_t)0x7fffffff) return fail(ROAM_ERR_ARG, "too many pixels");
    }
    const size_t bytes = sizeof(DevCamera) * (size_t)n_views;
    if (n_views == c->cams_dev_n && memcmp(c->h_cams, c->cams_dev.data(), bytes) == 0) {
        // the device already holds these cameras: order this stream after
        // that copy instead of copying again
        ROAM_CUDA(cudaStreamWaitEvent(s, c->cam_ev[c->cams_dev_slot], 0));
    } else {
        ROAM_TRY(ensure(c->cams, (size_t)n_views));
        ROAM_CUDA(cudaMemcpyAsync(c->cams.p, c->h_cams, bytes, cudaMemcpyHostToDevice, s));
        ROAM_CUDA(cudaEventRecord(c->cam_ev[slot], s));
        c->cam_pending[slot] = true;
        c->cams_dev.assign(c->h_cams, c->h_cams + n_views);
        c->cams_dev_n = n_views;
        c->cams_dev_slot = slot;
    }
    *n_pix = total;
    c->n_views = n_views;
    return ROAM_OK;
}

// tile records needed for `samples` samples: one per 128 plus padding of
// each field's run to a whole group
// tiles of 128 samples, each field's run rounded up to its padding (at most
// the larger of 8 and the forced padding)
size_t tile_capacity(const roam_ctx *c, size_t samples)
{
    return samples / 128 + (size_t)c->n_fields * (size_t)std::max(8, c->tile_pad) + 1;
}

roam_status ensure_rays(roam_ctx *c, int64_t n_rays, int R)
{
    const size_t n = (size_t)n_rays;
    ROAM_TRY(ensure(c->orig, n));
    ROAM_TRY(ensure(c->dir, n));
    ROAM_TRY(ensure(c->dir_lo, n));
    ROAM_TRY(ensure(c->acc, n));
    ROAM_TRY(ensure(c->tw, n));
    ROAM_TRY(ensure(c->j_next, n));
    ROAM_TRY(ensure(c->j_end, n));
    ROAM_TRY(ensure(c->n_kept, n));
    ROAM_TRY(ensure(c->live0, n));
    ROAM_TRY(ensure(c->live1, n));
    ROAM_TRY(ensure(c->cnt, n));
    const size_t slots = ((n + 31) & ~(size_t)31) * (size_t)R;
    ROAM_TRY(ensure(c->recs, slots));
    ROAM_TRY(ensure(c->sr, slots));
    ROAM_TRY(ensure(c->sorted, slots));
    ROAM_TRY(ensure(c->tiles, tile_capacity(c, slots)));
    return ROAM_OK;
}

roam_status ensure_fields_ws(roam_ctx *c)
{
    const size_t F = (size_t)c->n_fields;
    const bool fresh = !c->hist.p || c->hist.n < F;
    ROAM_TRY(ensure(c->hist, F));
    ROAM_TRY(ensure(c->offsets, F + 1));
    ROAM_TRY(ensure(c->cursor, F));
    ROAM_TRY(ensure(c->tile_off, F + 1));
    if (fresh) ROAM_CUDA(cudaMemset(c->hist.p, 0, F * sizeof(uint32_t)));
    return ROAM_OK;
}

RayState state_of(roam_ctx *c)
{
    RayState st;
    st.orig = c->orig.p;
    st.dir = c->dir.p;
    st.dir_lo = c->dir_lo.p;
    st.j_next = c->j_next.p;
    st.j_end = c->j_end.p;
    st.n_kept = c->n_kept.p;
    st.acc = c->acc.p;
    st.tw = c->tw.p;
    return st;
}

BucketBufs bucket_of(roam_ctx *c)
{
    BucketBufs b;
    b.hist = c->hist.p;
    b.offsets = c->offsets.p;
    b.cursor = c->cursor.p;
    b.tiles = c->tiles.p;
    b.sorted = c->sorted.p;
    b.tile_off = c->tile_off.p;
    return b;
}

int tile_of(int precision) { return precision != ROAM_F32 ? tc_tile_samples() : 128; }
// The classes with the tile padding of their MLP kernels: on the tensor cores
// every field's tile run is a multiple of its own kernel's tiles in flight
// (4, or 2 at W = 128), so that no group of tiles is empty throughout; the
// classes come in increasing width and the counts do not grow with width,
// so each class's range still starts on a group boundary of its kernel.
// FP32 (SIMT, one tile at a time): no padding.
ClassBounds classes_of(const roam_ctx *c, int precision)
{
    ClassBounds cb = c->cb;
    for (int k = 0; k < 4; ++k)
        cb.group[k] = (precision != ROAM_F32 && k < c->n_ws)
                          ? (c->tile_pad > 0 ? c->tile_pad : tc_tile_group(c->ws[k].W, precision == ROAM_FP8))
                          : 1;
    return cb;
}

roam_status run_mlp(roam_ctx *c, int precision, const SampleSrc &src, const BucketBufs &b, float4 *out,
                    Counters *ctr, cudaStream_t s)
{
    // one launch per width class over its own tile range
    for (int k = 0; k < c->n_ws; ++k) {
        const MlpWeights w = weights_of(c, k);
        if (precision != ROAM_F32) {
            launch_mlp_tc(w, precision == ROAM_FP8, src, b, ctr, out, c->n_sm, s);
            ROAM_TRY(launched("mlp_tc"));
        } else {
            launch_mlp_simt(w, src, b, ctr, out, c->n_sm, s);
            ROAM_TRY(launched("mlp_simt"));
        }
    }
    return ROAM_OK;
}

// The render / training-forward pipeline: rounds of march -> bucket -> MLP ->
// composite; each round marches at most R more kept samples of every live ray.
int n_rounds_of(int n_max, int R0, int R) { return 1 + (n_max > R0 ? (n_max - R0 + R - 1) / R : 0); }

// R0 kept samples per live ray in the first round, R in every later one
roam_status run_rounds(roam_ctx *c, const uint32_t *rays, int64_t n_rays, const roam_render_opts *o, float *rgb,
                       float *depth, float *opacity, int R0, int R, cudaStream_t s)
{
    const int n_rounds = n_rounds_of(o->n_max, R0, R);
    MarchParams mp{};
    mp.cams = c->cams.p;
    mp.n_views = c->n_views;
    mp.rays = rays;
    mp.n_rays = (uint32_t)n_rays;
    mp.R = R0;
    mp.n_max = o->n_max;
    mp.delta = o->delta;
    mp.flat = 0;
    mp.accurate = o->precision == ROAM_F32;
    mp.st = state_of(c);
    mp.cnt = c->cnt.p;
    mp.recs = c->recs.p;
    mp.ctr = c->ctr;
    mp.hist = c->hist.p;             // the march counts samples per field as it emits them
    const BucketBufs b = bucket_of(c);
    const int grid = grid_blocks(c, 4);
    uint32_t *lives[2] = {c->live0.p, c->live1.p};
    for (int r = 0; r < n_rounds; ++r) {
        const int Rr = r == 0 ? R0 : R;
        mp.R = Rr;
        mp.init = r == 0;
        mp.live = r == 0 ? nullptr : lives[r & 1];
        mp.live_count = r == 0 ? nullptr : &c->ctr->live_count[r & 1];
        {
            ProfScope ps(c, P_MARCH, s);
            launch_march(c->g, mp, march_grid(mp.n_rays), s);
        }
        ROAM_TRY(launched("march"));
        {
            ProfScope ps(c, P_BUCKET, s);
            launch_bucket_ready(mp.cnt, mp.recs, mp.live_count, mp.n_rays, Rr, 1, c->n_fields, tile_of(o->precision), b,
                                c->ctr, grid, s, classes_of(c, o->precision));
        }
        ROAM_TRY(launched("bucket"));
        SampleSrc src{};
        src.mode = 0;
        src.recs = mp.recs;
        src.live = mp.live;
        src.live_count = mp.live_count;
        src.R = Rr;
        src.st = mp.st;
        src.delta = o->delta;
        src.accurate = mp.accurate;
        {
            ProfScope ps(c, o->precision == ROAM_BF16 ? P_MLP_BF16 : (o->precision == ROAM_FP8 ? P_MLP_FP8 : P_MLP_F32), s);
            ROAM_TRY(run_mlp(c, o->precision, src, b, c->sr.p, c->ctr, s));
        }
        {
            ProfScope ps(c, P_COMPOSITE, s);
            launch_composite_round(mp, c->sr.p, lives[(r + 1) & 1], &c->ctr->live_count[(r + 1) & 1], o->t_stop,
                                   o->bg, rgb, depth, opacity, march_grid(mp.n_rays + 31), s);
        }
        ROAM_TRY(launched("composite"));
    }
    return ROAM_OK;
}

int round_size(const roam_render_opts *o, int64_t n_rays)
{
    int R = o->round_size > 0 ? o->round_size : 32;
    R = std::min(R, o->n_max);
    // slot indices are 32-bit
    while (R > 1 && (double)((n_rays + 31) & ~31LL) * R >= 4294967295.0) R >>= 1;
    return R;
}

// the first round's size: opts->first_round_size (0: the round size), at most
// the round size and n_max
int first_round_size(const roam_render_opts *o, int R)
{
    const int R0 = o->first_round_size > 0 ? o->first_round_size : R;
    return std::min(std::min(R0, R), o->n_max);
}

// The launch sequence of one render (counter resets + every round) as a CUDA
// graph on the context's own stream, captured for a configuration and
// replayed while it holds; forked from and joined back to the caller's stream.
roam_status render_graph(roam_ctx *c, int64_t n_pix, const roam_render_opts *o, float *rgb, float *depth,
                         float *opacity, int R0, int R, cudaStream_t s)
{
    if (!c->gstream) {
        ROAM_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        ROAM_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        ROAM_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    }
    uint32_t f[5];
    memcpy(&f[0], &o->delta, 4);
    memcpy(&f[1], &o->t_stop, 4);
    memcpy(&f[2], &o->bg[0], 4);
    memcpy(&f[3], &o->bg[1], 4);
    memcpy(&f[4], &o->bg[2], 4);
    const std::vector<uint64_t> key = {c->gen, g_alloc_gen.load(), (uint64_t)n_pix, (uint64_t)c->n_views, (uint64_t)R,
                                       (uint64_t)R0,
                                       (uint64_t)o->n_max, (uint64_t)o->precision, f[0], f[1], f[2], f[3], f[4],
                                       (uint64_t)(uintptr_t)rgb, (uint64_t)(uintptr_t)depth,
                                       (uint64_t)(uintptr_t)opacity};
    if (!c->gexec || key != c->gkey) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaStream_t g = c->gstream;
        ROAM_CUDA(cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(c->ctr, 0, sizeof(Counters), g);
        cudaMemsetAsync(c->hist.p, 0, (size_t)c->n_fields * sizeof(uint32_t), g);
        const roam_status st = run_rounds(c, nullptr, n_pix, o, rgb, depth, opacity, R0, R, g);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g, &graph);
        if (st != ROAM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return fail(ROAM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return fail(ROAM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
        }
        c->gkey = key;
    }
    ROAM_CUDA(cudaEventRecord(c->ev_fork, s));
    ROAM_CUDA(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0));
    ROAM_CUDA(cudaGraphLaunch(c->gexec, c->gstream));
    ROAM_CUDA(cudaEventRecord(c->ev_join, c->gstream));
    ROAM_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
    return ROAM_OK;
}

roam_status check_desc(const roam_mlp_desc *desc)
{
    if (desc->n_hidden < 1 || desc->n_hidden > 4) return fail(ROAM_ERR_ARG, "n_hidden must be in [1, 4]");
    if (!(desc->sigma_scale > 0.f) || !finite(desc->sigma_scale)) return fail(ROAM_ERR_ARG, "sigma_scale must be positive");
    if (desc->density_act != ROAM_SOFTPLUS && desc->density_act != ROAM_RELU)
        return fail(ROAM_ERR_ARG, "unknown density activation");
    return ROAM_OK;
}

__global__ void k_relabel(const uint16_t *src, const uint16_t *perm, int64_t n, uint16_t *dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = perm[src[i]];
}

// Internal field ids: perm[f] for the caller's field f (nullptr = identity).
// The device labels and the field affines follow; the caller's labels are
// kept aside while a permutation is in force.
roam_status set_field_order(roam_ctx *c, const uint16_t *perm)
{
    const int F = c->n_fields;
    if (!perm && !c->permuted) return ROAM_OK;
    if (!c->permuted && c->n_occ > 0) {
        ROAM_TRY(ensure(c->labels_orig, (size_t)c->n_occ));
        ROAM_CUDA(cudaMemcpy(c->labels_orig.p, c->labels.p, c->n_occ * sizeof(uint16_t), cudaMemcpyDeviceToDevice));
    }
    std::vector<float> aff(6 * (size_t)F);
    if (perm) {
        for (int f = 0; f < F; ++f) memcpy(&aff[6 * (size_t)perm[f]], &c->affine_orig[6 * (size_t)f], 6 * sizeof(float));
        ROAM_TRY(ensure(c->perm, (size_t)F));
        ROAM_CUDA(cudaMemcpy(c->perm.p, perm, F * sizeof(uint16_t), cudaMemcpyHostToDevice));
        if (c->n_occ > 0) {
            k_relabel<<<1024, 256>>>(c->labels_orig.p, c->perm.p, c->n_occ, c->labels.p);
            ROAM_TRY(launched("relabel"));
        }
    } else {
        aff = c->affine_orig;
        if (c->n_occ > 0)
            ROAM_CUDA(cudaMemcpy(c->labels.p, c->labels_orig.p, c->n_occ * sizeof(uint16_t), cudaMemcpyDeviceToDevice));
    }
    ROAM_CUDA(cudaMemcpy(c->affine.p, aff.data(), aff.size() * sizeof(float), cudaMemcpyHostToDevice));
    ROAM_CUDA(cudaDeviceSynchronize());
    c->permuted = perm != nullptr;
    return ROAM_OK;
}

// Loads weight set k: n fields of width W (internal ids first .. first + n - 1),
// FP32 masters in the API layout, and packs the SIMT and tensor-core copies.
roam_status load_set(roam_ctx *c, int k, int W, int H, int first, int n, const float *weights, bool on_device)
{
    WSet &q = c->ws[k];
    const int64_t P = param_count(W, H);
    const int64_t total = P * n;
    ROAM_TRY(ensure(q.w32, (size_t)total));
    ROAM_CUDA(cudaMemcpy(q.w32.p, weights, total * sizeof(float),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    ROAM_CUDA(cudaMemset(c->d_flag, 0, 4));
    k_check_finite<<<1024, 256>>>(q.w32.p, total, c->d_flag);
    ROAM_TRY(launched("weight check"));
    uint32_t bad = 0;
    ROAM_CUDA(cudaMemcpy(&bad, c->d_flag, 4, cudaMemcpyDeviceToHost));
    if (bad) return fail(ROAM_ERR_ARG, "weights contain NaN or Inf");
    q.W = W;
    q.first = first;
    q.n = n;
    q.P = P;
    q.stale = 0;
    q.Pt = simt_transposed_size(W, H);
    ROAM_TRY(ensure(q.wt, (size_t)(q.Pt * n)));
    launch_pack_simt(q.w32.p, n, W, H, P, q.wt.p, q.Pt, 0);
    ROAM_TRY(launched("pack simt"));
    q.Pr = rows_padded_size(W, H);
    ROAM_TRY(ensure(q.wr, (size_t)(q.Pr * n)));
    launch_pack_rows(q.w32.p, n, W, H, P, q.wr.p, q.Pr, 0);
    ROAM_TRY(launched("pack rows"));
    q.tc_ok = tc_supported(W, H, false);
    if (q.tc_ok) {
        q.img_bytes = tc_image_bytes(W, H, false);
        ROAM_TRY(ensure(q.wimg, (size_t)(q.img_bytes * n)));
        launch_pack_tc(q.w32.p, n, W, H, P, q.wimg.p, q.img_bytes, false, 0);
        ROAM_TRY(launched("pack tc"));
    }
    q.tc8_ok = tc_supported(W, H, true);
    if (q.tc8_ok) {
        q.img8_bytes = tc_image_bytes(W, H, true);
        ROAM_TRY(ensure(q.wimg8, (size_t)(q.img8_bytes * n)));
        launch_pack_tc(q.w32.p, n, W, H, P, q.wimg8.p, q.img8_bytes, true, 0);
        ROAM_TRY(launched("pack tc fp8"));
    }
    return ROAM_OK;
}

__global__ void k_unpermute_recs(const uint32_t *count, uint32_t *recs, int64_t n_rays, int n_max, const uint16_t *inv)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays * n_max;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n_max;
        if ((uint32_t)(i % n_max) < count[r]) recs[i] = (recs[i] & 0xffffu) | ((uint32_t)inv[recs[i] >> 16] << 16);
    }
}

__global__ void k_map_keys(const uint16_t *keys, int64_t n, const uint16_t *perm, int n_fields, uint16_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = keys[i] < n_fields ? perm[keys[i]] : keys[i];   // out-of-range ids stay invalid
}

}  // namespace

namespace roam {
void set_error_message(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace roam

extern "C" {

const char *roam_last_error(void) { return g_err; }

roam_status roam_create(roam_ctx **out, int device)
{
    if (!out) return fail(ROAM_ERR_ARG, "null output handle");
    *out = nullptr;
    int n_dev = 0;
    ROAM_CUDA(cudaGetDeviceCount(&n_dev));
    if (device < 0 || device >= n_dev) return fail(ROAM_ERR_ARG, "device %d out of range (%d devices)", device, n_dev);
    ROAM_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    ROAM_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(ROAM_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a only", device,
                    prop.major, prop.minor);
    roam_ctx *c = new roam_ctx();
    c->device = device;
    c->n_sm = prop.multiProcessorCount;
    bool ok = cudaMalloc(&c->ctr, 2 * sizeof(Counters)) == cudaSuccess &&
              cudaMallocHost(&c->h_ctr, 2 * sizeof(Counters)) == cudaSuccess &&
              cudaMallocHost(&c->h_cams_ring, sizeof(DevCamera) * kMaxViews * roam_ctx::kCamRing) == cudaSuccess &&
              cudaMalloc(&c->d_flag, sizeof(uint32_t)) == cudaSuccess;
    for (int i = 0; i < roam_ctx::kCamRing && ok; ++i)
        ok = cudaEventCreateWithFlags(&c->cam_ev[i], cudaEventDisableTiming) == cudaSuccess;
    c->h_cams = c->h_cams_ring;
    if (!ok) {
        cudaGetLastError();
        roam_destroy(c);
        return fail(ROAM_ERR_OOM, "context allocation failed");
    }
    c->aux = c->ctr + 1;
    cudaMemset(c->ctr, 0, 2 * sizeof(Counters));
    *out = c;
    return ROAM_OK;
}

roam_status roam_destroy(roam_ctx *c)
{
    if (!c) return ROAM_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    release(c->bits); release(c->prefix); release(c->block_sums);
    release(c->brick_occ); release(c->brick_dist); release(c->brick_t0); release(c->brick_t1);
    release(c->labels); release(c->affine);
    for (WSet &q : c->ws) {
        release(q.w32); release(q.wt); release(q.wr); release(q.wimg); release(q.wimg8);
    }
    release(c->occ_hit); release(c->occ_free); release(c->assign_vox); release(c->assign_scratch);
    release(c->teacher_img); release(c->teacher_wt); release(c->teacher_ws); release(c->selftest);
    release(c->perm); release(c->inv); release(c->labels_orig); release(c->keys_tmp);
    release(c->gsr); release(c->adam_m); release(c->adam_v);
    release(c->orig); release(c->dir); release(c->dir_lo); release(c->acc); release(c->sr); release(c->tw);
    release(c->j_next); release(c->j_end); release(c->n_kept); release(c->live0); release(c->live1);
    release(c->cnt); release(c->recs); release(c->sorted); release(c->hist); release(c->offsets);
    release(c->cursor); release(c->scratch_u32); release(c->tiles); release(c->tile_off);
    release(c->o_rgb); release(c->o_depth); release(c->o_op); release(c->cams);
    if (c->h_cams_ring) cudaFreeHost(c->h_cams_ring);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->ctr) cudaFree(c->ctr);
    if (c->d_flag) cudaFree(c->d_flag);
    for (cudaEvent_t e : c->cam_ev)
        if (e) cudaEventDestroy(e);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto &p : c->prof_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    delete c;
    return ROAM_OK;
}

roam_status roam_check(roam_ctx *c)
{
    ROAM_TRY(set_dev(c));
    ROAM_CUDA(cudaStreamSynchronize(c->last));
    ROAM_CUDA(cudaMemcpy(c->h_ctr, c->ctr, 2 * sizeof(Counters), cudaMemcpyDeviceToHost));
    return status_of(c->h_ctr[0].status | c->h_ctr[1].status);
}

roam_status roam_load_grid(roam_ctx *c, const roam_grid_desc *desc, const uint32_t *bits, int on_device)
{
    ROAM_TRY(set_dev(c));
    if (!desc || !bits) return fail(ROAM_ERR_ARG, "null grid descriptor or bits");
    for (int a = 0; a < 3; ++a)
        if (desc->dims[a] < 8 || desc->dims[a] > 2048 || desc->dims[a] % 8)
            return fail(ROAM_ERR_ARG, "grid dims must be multiples of 8 in [8, 2048]");
    if (desc->dims[0] % 32) return fail(ROAM_ERR_ARG, "grid x dimension must be a multiple of 32");
    if (!(desc->vox > 0.f) || !finite(desc->vox)) return fail(ROAM_ERR_ARG, "voxel size must be positive");
    for (int a = 0; a < 3; ++a)
        if (!finite(desc->origin[a])) return fail(ROAM_ERR_ARG, "grid origin must be finite");
    c->has_grid = c->has_fields = c->has_weights = false;
    ++c->gen;
    const int64_t n_words = (int64_t)desc->dims[0] / 32 * desc->dims[1] * desc->dims[2];
    ROAM_TRY(ensure(c->bits, (size_t)n_words));
    ROAM_TRY(ensure(c->prefix, (size_t)n_words));
    ROAM_TRY(ensure(c->block_sums, (size_t)((n_words + 4095) / 4096)));
    ROAM_CUDA(cudaMemcpy(c->bits.p, bits, n_words * sizeof(uint32_t),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    GridDev &g = c->g;
    g.gx = desc->dims[0]; g.gy = desc->dims[1]; g.gz = desc->dims[2];
    g.wpr = g.gx / 32;
    g.bx = g.gx >> kBrickShift; g.by = g.gy >> kBrickShift; g.bz = g.gz >> kBrickShift;
    for (int a = 0; a < 3; ++a) g.origin[a] = desc->origin[a];
    g.vox = desc->vox;
    g.inv_vox = 1.0f / desc->vox;
    const size_t n_bricks = (size_t)g.bx * g.by * g.bz;
    ROAM_TRY(ensure(c->brick_occ, n_bricks));
    ROAM_TRY(ensure(c->brick_dist, n_bricks));
    ROAM_TRY(ensure(c->brick_t0, n_bricks));
    ROAM_TRY(ensure(c->brick_t1, n_bricks));
    g.bits = c->bits.p;
    g.prefix = c->prefix.p;
    g.brick_dist = c->brick_dist.p;
    g.labels = nullptr;
    g.n_fields = 0;
    launch_grid_prefix(c->bits.p, c->prefix.p, c->block_sums.p, n_words, 0);
    ROAM_TRY(launched("grid prefix"));
    launch_brick_dist(g, c->brick_occ.p, c->brick_t0.p, c->brick_t1.p, c->brick_dist.p, 0);
    ROAM_TRY(launched("brick distance map"));
    uint32_t last_pre = 0, last_word = 0;
    ROAM_CUDA(cudaMemcpy(&last_pre, c->prefix.p + n_words - 1, 4, cudaMemcpyDeviceToHost));
    ROAM_CUDA(cudaMemcpy(&last_word, c->bits.p + n_words - 1, 4, cudaMemcpyDeviceToHost));
    c->n_words = n_words;
    c->n_occ = (int64_t)last_pre + __builtin_popcount(last_word);
    c->gd = *desc;
    c->has_grid = true;
    return ROAM_OK;
}

roam_status roam_load_fields(roam_ctx *c, int n_fields, const uint16_t *labels, int64_t n_occupied,
                             const float *affine, int on_device)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_grid) return fail(ROAM_ERR_STATE, "load the occupancy grid first");
    if (n_fields < 1 || n_fields > 8192) return fail(ROAM_ERR_ARG, "n_fields must be in [1, 8192]");
    if (n_occupied != c->n_occ)
        return fail(ROAM_ERR_ARG, "n_occupied=%lld but the grid has %lld occupied voxels", (long long)n_occupied,
                    (long long)c->n_occ);
    if ((n_occupied > 0 && !labels) || !affine) return fail(ROAM_ERR_ARG, "null labels or affine");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    std::vector<float> aff_h(6 * (size_t)n_fields);
    if (on_device) ROAM_CUDA(cudaMemcpy(aff_h.data(), affine, aff_h.size() * 4, cudaMemcpyDeviceToHost));
    else memcpy(aff_h.data(), affine, aff_h.size() * 4);
    for (float v : aff_h)
        if (!finite(v)) return fail(ROAM_ERR_ARG, "non-finite field affine");
    c->has_fields = c->has_weights = false;
    ++c->gen;
    ROAM_TRY(ensure(c->labels, (size_t)std::max<int64_t>(n_occupied, 1)));
    ROAM_TRY(ensure(c->affine, 6 * (size_t)n_fields));
    if (n_occupied > 0) ROAM_CUDA(cudaMemcpy(c->labels.p, labels, n_occupied * sizeof(uint16_t), kind));
    ROAM_CUDA(cudaMemcpy(c->affine.p, aff_h.data(), aff_h.size() * 4, cudaMemcpyHostToDevice));
    if (n_occupied > 0) {
        ROAM_CUDA(cudaMemset(c->d_flag, 0, 4));
        k_check_labels<<<256, 256>>>(c->labels.p, n_occupied, n_fields, c->d_flag);
        ROAM_TRY(launched("label check"));
        uint32_t bad = 0;
        ROAM_CUDA(cudaMemcpy(&bad, c->d_flag, 4, cudaMemcpyDeviceToHost));
        if (bad) return fail(ROAM_ERR_ARG, "a field label is >= n_fields");
    }
    c->n_fields = n_fields;
    c->g.labels = c->labels.p;
    c->g.n_fields = n_fields;
    c->permuted = false;
    release(c->labels_orig);
    c->affine_orig = aff_h;
    ROAM_TRY(ensure_fields_ws(c));
    c->has_fields = true;
    return ROAM_OK;
}

roam_status roam_load_weights(roam_ctx *c, const roam_mlp_desc *desc, const float *weights, int on_device)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_fields) return fail(ROAM_ERR_STATE, "load the field labels first");
    if (!desc || !weights) return fail(ROAM_ERR_ARG, "null MLP descriptor or weights");
    if (desc->width != 32 && desc->width != 64 && desc->width != 128)
        return fail(ROAM_ERR_ARG, "width must be 32, 64 or 128");
    ROAM_TRY(check_desc(desc));
    c->has_weights = false;
    ++c->gen;
    ROAM_TRY(set_field_order(c, nullptr));
    c->n_ws = 1;
    c->cb = ClassBounds{{0, c->n_fields, c->n_fields, c->n_fields}, {0, 0, 0, 0}};
    c->widths.assign(c->n_fields, desc->width);
    ROAM_TRY(load_set(c, 0, desc->width, desc->n_hidden, 0, c->n_fields, weights, on_device != 0));
    c->md = *desc;
    c->adam_fresh = true;
    c->train_rays = 0;
    ROAM_CUDA(cudaDeviceSynchronize());
    c->has_weights = true;
    return ROAM_OK;
}

roam_status roam_load_weights_mixed(roam_ctx *c, const roam_mlp_desc *desc, const int32_t *field_width,
                                    const float *weights, int on_device)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_fields) return fail(ROAM_ERR_STATE, "load the field labels first");
    if (!desc || !weights || !field_width) return fail(ROAM_ERR_ARG, "null descriptor, widths or weights");
    ROAM_TRY(check_desc(desc));
    const int F = c->n_fields, H = desc->n_hidden;
    const int kW[3] = {32, 64, 128};
    std::vector<int> cls(F);
    int count[3] = {0, 0, 0};
    int64_t total = 0;
    for (int f = 0; f < F; ++f) {
        const int w = field_width[f];
        cls[f] = w == 32 ? 0 : (w == 64 ? 1 : (w == 128 ? 2 : -1));
        if (cls[f] < 0) return fail(ROAM_ERR_ARG, "field %d: width must be 32, 64 or 128", f);
        ++count[cls[f]];
        total += param_count(w, H);
    }
    c->has_weights = false;
    ++c->gen;
    // the caller's weights, field after field (each in its own width's layout)
    std::vector<float> hw((size_t)total);
    ROAM_CUDA(cudaMemcpy(hw.data(), weights, (size_t)total * sizeof(float),
                         on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    std::vector<int64_t> off(F + 1, 0);
    for (int f = 0; f < F; ++f) off[f + 1] = off[f] + param_count(field_width[f], H);
    // internal ids: classes in width order, the caller's order inside a class
    std::vector<uint16_t> perm(F), inv(F);
    int n_ws = 0, next = 0, first[3] = {0, 0, 0}, wcls[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        if (!count[k]) continue;
        first[n_ws] = next;
        wcls[n_ws] = kW[k];
        for (int f = 0; f < F; ++f)
            if (cls[f] == k) {
                perm[f] = (uint16_t)next;
                inv[next] = (uint16_t)f;
                ++next;
            }
        ++n_ws;
    }
    ROAM_TRY(set_field_order(c, n_ws > 1 ? perm.data() : nullptr));
    if (n_ws > 1) {
        ROAM_TRY(ensure(c->inv, (size_t)F));
        ROAM_CUDA(cudaMemcpy(c->inv.p, inv.data(), F * sizeof(uint16_t), cudaMemcpyHostToDevice));
    }
    c->n_ws = n_ws;
    c->cb = ClassBounds{{0, F, F, F}, {0, 0, 0, 0}};
    for (int k = 0; k < n_ws; ++k) {
        c->cb.first[k] = first[k];
        const int n_k = (k + 1 < n_ws ? first[k + 1] : F) - first[k];
        const int64_t P = param_count(wcls[k], H);
        std::vector<float> part((size_t)(P * n_k));
        for (int q = 0; q < n_k; ++q) {
            const int f = n_ws > 1 ? inv[first[k] + q] : first[k] + q;
            memcpy(part.data() + (size_t)q * P, hw.data() + off[f], (size_t)P * sizeof(float));
        }
        ROAM_TRY(load_set(c, k, wcls[k], H, first[k], n_k, part.data(), false));
    }
    c->widths.assign(field_width, field_width + F);
    c->md = *desc;
    c->md.width = n_ws == 1 ? wcls[0] : 0;
    c->adam_fresh = true;
    c->train_rays = 0;
    ROAM_CUDA(cudaDeviceSynchronize());
    c->has_weights = true;
    return ROAM_OK;
}

roam_status roam_get_weights(roam_ctx *c, float *out, int on_device)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_weights) return fail(ROAM_ERR_STATE, "no weights loaded");
    if (!out) return fail(ROAM_ERR_ARG, "null output");
    ROAM_CUDA(cudaDeviceSynchronize());
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->n_ws == 1) {
        ROAM_CUDA(cudaMemcpy(out, c->ws[0].w32.p, (size_t)(c->ws[0].P * c->n_fields) * sizeof(float), kind));
        return ROAM_OK;
    }
    // mixed widths: field after field in the caller's order
    std::vector<uint16_t> perm(c->n_fields);
    ROAM_CUDA(cudaMemcpy(perm.data(), c->perm.p, c->n_fields * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    int64_t off = 0;
    for (int f = 0; f < c->n_fields; ++f) {
        const int i = perm[f];
        int k = 0;
        while (k + 1 < c->n_ws && i >= c->ws[k + 1].first) ++k;
        const WSet &q = c->ws[k];
        ROAM_CUDA(cudaMemcpy(out + off, q.w32.p + (int64_t)(i - q.first) * q.P, (size_t)q.P * sizeof(float), kind));
        off += q.P;
    }
    return ROAM_OK;
}

roam_status roam_render(roam_ctx *c, const roam_camera *cams, int n_views, const roam_render_opts *opts, float *rgb,
                        float *depth, float *opacity, int out_on_device, void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    ROAM_TRY(check_opts(c, opts));
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(refresh(c, opts->precision, false, s));
    int64_t n_pix = 0;
    ROAM_TRY(upload_cams(c, cams, n_views, opts->delta, &n_pix, s));
    const int R = round_size(opts, n_pix);
    const int R0 = first_round_size(opts, R);
    ROAM_TRY(ensure_rays(c, n_pix, R));
    float *d_rgb = rgb, *d_depth = depth, *d_op = opacity;
    if (!out_on_device) {
        if (rgb) { ROAM_TRY(ensure(c->o_rgb, 3 * (size_t)n_pix)); d_rgb = c->o_rgb.p; }
        if (depth) { ROAM_TRY(ensure(c->o_depth, (size_t)n_pix)); d_depth = c->o_depth.p; }
        if (opacity) { ROAM_TRY(ensure(c->o_op, (size_t)n_pix)); d_op = c->o_op.p; }
    }
    if (opts->use_graph && !c->prof) {
        ROAM_TRY(render_graph(c, n_pix, opts, d_rgb, d_depth, d_op, R0, R, s));
    } else {
        ROAM_CUDA(cudaMemsetAsync(c->ctr, 0, sizeof(Counters), s));
        ROAM_CUDA(cudaMemsetAsync(c->hist.p, 0, (size_t)c->n_fields * sizeof(uint32_t), s));
        ROAM_TRY(run_rounds(c, nullptr, n_pix, opts, d_rgb, d_depth, d_op, R0, R, s));
    }
    c->last = s;
    c->last_rays = n_pix;
    c->last_rounds = n_rounds_of(opts->n_max, R0, R);
    c->train_rays = 0;
    if (!out_on_device) {
        if (rgb) ROAM_CUDA(cudaMemcpyAsync(rgb, d_rgb, 12 * (size_t)n_pix, cudaMemcpyDeviceToHost, s));
        if (depth) ROAM_CUDA(cudaMemcpyAsync(depth, d_depth, 4 * (size_t)n_pix, cudaMemcpyDeviceToHost, s));
        if (opacity) ROAM_CUDA(cudaMemcpyAsync(opacity, d_op, 4 * (size_t)n_pix, cudaMemcpyDeviceToHost, s));
        ROAM_CUDA(cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
        ROAM_CUDA(cudaStreamSynchronize(s));
        return status_of(c->h_ctr->status);
    }
    return ROAM_OK;
}

roam_status roam_tune_round_size(roam_ctx *c, const roam_camera *cams, int n_views, const roam_render_opts *opts,
                                 int32_t *best_round_size, int32_t *best_first_round_size, float *best_ms,
                                 void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    ROAM_TRY(check_opts(c, opts));
    if (!best_round_size) return fail(ROAM_ERR_ARG, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(refresh(c, opts->precision, false, s));
    int64_t n_pix = 0;
    ROAM_TRY(upload_cams(c, cams, n_views, opts->delta, &n_pix, s));
    size_t free_b = 0, total_b = 0;
    ROAM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t have = c->recs.n + free_b / 24;          // slots the workspace can reach (24 B per slot)
    ROAM_TRY(ensure(c->o_rgb, 3 * (size_t)n_pix));
    cudaEvent_t e0, e1;
    ROAM_CUDA(cudaEventCreate(&e0));
    ROAM_CUDA(cudaEventCreate(&e1));
    roam_status st = ROAM_OK;
    // one warm-up render, then one timed render of this (first round, round) pair
    auto time_pair = [&](int R0, int R, float &t) {
        roam_render_opts o = *opts;
        o.round_size = R;
        o.first_round_size = R0;
        o.use_graph = 0;
        for (int rep = 0; rep < 2 && st == ROAM_OK; ++rep) {
            if ((st = ensure_rays(c, n_pix, R)) != ROAM_OK) break;
            cudaEventRecord(e0, s);
            cudaMemsetAsync(c->ctr, 0, sizeof(Counters), s);
            cudaMemsetAsync(c->hist.p, 0, (size_t)c->n_fields * sizeof(uint32_t), s);
            st = run_rounds(c, nullptr, n_pix, &o, c->o_rgb.p, nullptr, nullptr, R0, R, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ROAM_ERR_CUDA, "tuning render failed");
            cudaEventElapsedTime(&t, e0, e1);
        }
    };
    int best = 0, best0 = 0;
    float best_t = 0.f;
    // the round size, every round alike
    for (int R = 4; R <= opts->n_max && R <= 256 && st == ROAM_OK; R *= 2) {
        roam_render_opts o = *opts;
        o.round_size = R;
        if (round_size(&o, n_pix) != R) break;                                // 32-bit slot ids
        if ((size_t)((n_pix + 31) & ~31LL) * (size_t)R > have / 2) break;   // leave half the memory free
        float t = 0.f;
        time_pair(R, R, t);
        if (st == ROAM_OK && (best == 0 || t < best_t)) {
            best = best0 = R;
            best_t = t;
        }
    }
    // then a smaller first round: most rays stop at their first surface, and
    // the samples a round marches past a ray's termination are evaluated for
    // nothing
    for (int R0 = 4; best > 0 && R0 < best && st == ROAM_OK; R0 *= 2) {
        float t = 0.f;
        time_pair(R0, best, t);
        if (st == ROAM_OK && t < best_t) {
            best0 = R0;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ROAM_TRY(st);
    if (best == 0) return fail(ROAM_ERR_OOM, "no round size fits the device");
    c->last = s;
    c->last_rays = n_pix;
    *best_round_size = best;
    if (best_first_round_size) *best_first_round_size = best0;
    if (best_ms) *best_ms = best_t;
    ROAM_CUDA(cudaMemcpy(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
    return status_of(c->h_ctr->status);
}

roam_status roam_occupancy_update(roam_ctx *c, const roam_camera *cams, int n_views, const float *depth,
                                  const float *opacity, const roam_occ_params *q, float *logit, uint32_t *bits,
                                  void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_grid) return fail(ROAM_ERR_STATE, "load the occupancy grid first (it fixes the voxel lattice)");
    if (!q || !depth || !opacity || !logit) return fail(ROAM_ERR_ARG, "null pointer");
    if (!(q->p_hit > 0.5f && q->p_hit < 1.f) || !(q->p_miss > 0.f && q->p_miss < 0.5f) || !(q->l_min < 0.f) ||
        !(q->l_max > 0.f) || !(q->p_occ > 0.f && q->p_occ < 1.f) || !(q->a_min > 0.f && q->a_min <= 1.f) ||
        !finite(q->l_min) || !finite(q->l_max))
        return fail(ROAM_ERR_ARG, "bad occupancy parameters");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n_pix = 0;
    ROAM_TRY(upload_cams(c, cams, n_views, 0.25f * c->gd.vox, &n_pix, s));
    const int64_t n_vox = (int64_t)c->g.gx * c->g.gy * c->g.gz;
    ROAM_TRY(ensure(c->occ_hit, (size_t)n_vox));
    ROAM_TRY(ensure(c->occ_free, (size_t)(n_vox / 32)));
    ROAM_CUDA(cudaMemsetAsync(c->occ_hit.p, 0, (size_t)n_vox * 4, s));
    ROAM_CUDA(cudaMemsetAsync(c->occ_free.p, 0, (size_t)(n_vox / 32) * 4, s));
    for (int v = 0; v < n_views; ++v) {
        launch_occupancy_scan(c->g, c->cams.p, v, cams[v].width * cams[v].height, depth, opacity, *q, c->occ_hit.p,
                              c->occ_free.p, logit, bits, c->n_sm, s);
        ROAM_TRY(launched("occupancy scan"));
    }
    c->last = s;
    return ROAM_OK;
}

roam_status roam_assign_fields(roam_ctx *c, int n_fields, uint16_t *labels, int32_t *boxes, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_grid) return fail(ROAM_ERR_STATE, "load the occupancy grid first");
    if (!labels) return fail(ROAM_ERR_ARG, "null labels");
    const int64_t S = c->n_occ;
    if (n_fields < 1 || n_fields > 8192 || n_fields > S)
        return fail(ROAM_ERR_ARG, "n_fields must be in [1, min(8192, occupied voxels = %lld)]", (long long)S);
    if (S >= (int64_t)1 << 27) return fail(ROAM_ERR_ARG, "at most 2^27 - 1 occupied voxels");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(ensure(c->assign_vox, (size_t)S));
    ROAM_TRY(ensure(c->assign_scratch, assign_scratch_bytes()));
    launch_assign(c->bits.p, c->prefix.p, c->n_words, c->g.gx, c->g.gy, (uint32_t)S, n_fields, c->assign_vox.p,
                  labels, boxes, c->assign_scratch.p, c->n_sm, s);
    ROAM_TRY(launched("field assignment"));
    ROAM_CUDA(cudaStreamSynchronize(s));
    if (assign_status(c->assign_scratch.p)) return fail(ROAM_ERR_DATA, "field assignment ran out of voxels");
    return ROAM_OK;
}

roam_status roam_teacher_load(roam_ctx *c, const float *weights, const float *affine, int on_device)
{
    ROAM_TRY(set_dev(c));
    if (!weights || !affine) return fail(ROAM_ERR_ARG, "null weights or affine");
    const int64_t P = teacher_param_count();
    c->has_teacher = false;
    // the caller's layout lands in the workspace, is checked, then packed
    // into the tensor-core image and the transposed FP32 layers
    ROAM_TRY(ensure(c->teacher_ws, (size_t)P));
    ROAM_TRY(ensure(c->teacher_wt, (size_t)P));
    ROAM_TRY(ensure(c->teacher_img, (size_t)teacher_image_bytes()));
    ROAM_CUDA(cudaMemcpy(c->teacher_ws.p, weights, (size_t)P * sizeof(float),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    ROAM_CUDA(cudaMemset(c->d_flag, 0, 4));
    k_check_finite<<<1024, 256>>>(c->teacher_ws.p, P, c->d_flag);
    ROAM_TRY(launched("teacher weight check"));
    uint32_t bad = 0;
    ROAM_CUDA(cudaMemcpy(&bad, c->d_flag, 4, cudaMemcpyDeviceToHost));
    if (bad) return fail(ROAM_ERR_ARG, "teacher weights contain NaN or Inf");
    launch_teacher_pack(c->teacher_ws.p, c->teacher_img.p, c->teacher_wt.p, 0);
    ROAM_TRY(launched("teacher pack"));
    ROAM_CUDA(cudaDeviceSynchronize());
    for (int i = 0; i < 6; ++i) {
        if (!finite(affine[i])) return fail(ROAM_ERR_ARG, "non-finite teacher affine");
        c->teacher_aff.v[i] = affine[i];
    }
    c->has_teacher = true;
    return ROAM_OK;
}

roam_status roam_teacher_eval(roam_ctx *c, const float *p, const float *d, int64_t n, int precision, float *out,
                              void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_teacher) return fail(ROAM_ERR_STATE, "no teacher loaded");
    if (precision != ROAM_F32 && precision != ROAM_BF16) return fail(ROAM_ERR_ARG, "precision: ROAM_F32 or ROAM_BF16");
    if (n < 0 || n > 0x7fffffff) return fail(ROAM_ERR_ARG, "bad sample count");
    if (n == 0) return ROAM_OK;
    if (!p || !d || !out) return fail(ROAM_ERR_ARG, "null pointer");
    if (((uintptr_t)out) & 15) return fail(ROAM_ERR_ARG, "out must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == ROAM_BF16) {
        ProfScope ps(c, P_TEACHER_TC, s);
        launch_teacher_tc(c->teacher_img.p, c->teacher_aff, n, p, d, reinterpret_cast<float4 *>(out), &c->aux->status,
                          c->n_sm, s);
    } else {
        ProfScope ps(c, P_TEACHER_F32, s);
        launch_teacher_simt(c->teacher_wt.p, c->teacher_aff, n, p, d, reinterpret_cast<float4 *>(out), c->n_sm, s);
    }
    c->last = s;
    return launched("teacher");
}

roam_status roam_distill_loss(roam_ctx *c, const float *student, const float *teacher, int64_t n, float I,
                              float *dl_dout, float *loss, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (n < 0 || !(I > 0.f)) return fail(ROAM_ERR_ARG, "bad sizes");
    if (!student || !teacher || !dl_dout) return fail(ROAM_ERR_ARG, "null pointer");
    if ((((uintptr_t)student) | ((uintptr_t)teacher) | ((uintptr_t)dl_dout)) & 15)
        return fail(ROAM_ERR_ARG, "arrays must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    launch_distill_loss(n, reinterpret_cast<const float4 *>(student), reinterpret_cast<const float4 *>(teacher), I,
                        reinterpret_cast<float4 *>(dl_dout), loss, s);
    c->last = s;
    return launched("distill loss");
}

roam_status roam_mlp_backward(roam_ctx *c, const float *p, const float *d, const uint16_t *field, int64_t n,
                              int precision, const float *dl_dout, float *grad, void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    if (c->n_ws != 1) return fail(ROAM_ERR_UNSUPPORTED, "training needs one MLP width for every field");
    if (!mlp_bwd_supported(c->md.width, c->md.n_hidden))
        return fail(ROAM_ERR_UNSUPPORTED, "training supports W = 32 or 64");
    if (precision != ROAM_F32 && precision != ROAM_BF16) return fail(ROAM_ERR_ARG, "precision: ROAM_F32 or ROAM_BF16");
    const bool tc = precision == ROAM_BF16;
    if (tc && (!mlp_bwd_tc_supported(c->md.width, c->md.n_hidden) || !c->ws[0].tc_ok))
        return fail(ROAM_ERR_UNSUPPORTED, "the BF16 adjoint supports W = 32 (H <= 4) and W = 64 (H <= 3)");
    if (n < 0 || n > 0x7fffffff) return fail(ROAM_ERR_ARG, "bad sample count");
    if (!grad) return fail(ROAM_ERR_ARG, "null gradient");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(refresh(c, precision, !tc, s));
    ROAM_CUDA(cudaMemsetAsync(grad, 0, (size_t)(c->ws[0].P * c->n_fields) * sizeof(float), s));
    if (n == 0) return ROAM_OK;
    if (!p || !d || !field || !dl_dout) return fail(ROAM_ERR_ARG, "null pointer");
    if (((uintptr_t)dl_dout) & 15) return fail(ROAM_ERR_ARG, "dl_dout must be 16-byte aligned");
    ROAM_TRY(ensure(c->sorted, (size_t)n));
    ROAM_TRY(ensure(c->tiles, tile_capacity(c, (size_t)n)));
    const BucketBufs b = bucket_of(c);
    ROAM_CUDA(cudaMemsetAsync(c->aux, 0, sizeof(Counters), s));
    launch_bucket(nullptr, nullptr, nullptr, (uint32_t)n, 1, 1, field, c->n_fields, 128, b, c->aux, grid_blocks(c, 2),
                  s, c->cb);
    ROAM_TRY(launched("bucket"));
    SampleSrc src{};
    src.mode = 1;
    src.p = p;
    src.d = d;
    if (tc) {
        ProfScope ps(c, P_MLP_BWD_TC, s);
        launch_mlp_bwd_tc(weights_of(c), src, b, c->aux, reinterpret_cast<const float4 *>(dl_dout), grad, c->n_sm, s);
    } else {
        ProfScope ps(c, P_MLP_BWD, s);
        launch_mlp_bwd_simt(weights_of(c), src, b, c->aux, reinterpret_cast<const float4 *>(dl_dout), grad, c->n_sm,
                            s);
    }
    c->last = s;
    return launched("mlp_bwd");
}

roam_status roam_get_stats(roam_ctx *c, roam_stats *st)
{
    ROAM_TRY(set_dev(c));
    if (!st) return fail(ROAM_ERR_ARG, "null stats");
    ROAM_CUDA(cudaStreamSynchronize(c->last));
    ROAM_CUDA(cudaMemcpy(c->h_ctr, c->ctr, 2 * sizeof(Counters), cudaMemcpyDeviceToHost));
    st->n_samples = (int64_t)c->h_ctr->n_samples;
    st->n_used = (int64_t)c->h_ctr->n_used;
    st->n_fields_hit = (int32_t)c->h_ctr->fields_hit;
    st->n_rays = c->last_rays;
    st->n_rounds = c->last_rounds;
    return status_of(c->h_ctr[0].status | c->h_ctr[1].status);
}

roam_status roam_set_tile_padding(roam_ctx *c, int tiles)
{
    ROAM_TRY(set_dev(c));
    // a multiple of every tensor-core kernel's tiles in flight (4, 2 or 1),
    // so that every width class's range still starts on a group boundary
    if (tiles != 0 && (tiles < 4 || tiles > 64 || tiles % 4))
        return fail(ROAM_ERR_ARG, "tile padding must be 0 or a multiple of 4 in [4, 64]");
    c->tile_pad = tiles;
    ++c->gen;                          // a captured render graph holds the old padding
    return ROAM_OK;
}

roam_status roam_selftest_wait_timeout(roam_ctx *c, uint64_t limit_ns, int32_t *observed, void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    if (!observed) return fail(ROAM_ERR_ARG, "null output");
    if (limit_ns < 1000000ull || limit_ns > 10000000000ull) return fail(ROAM_ERR_ARG, "limit_ns must be in [1e6, 1e10]");
    if (!all_tc(c, false)) return fail(ROAM_ERR_UNSUPPORTED, "needs the tensor-core MLP of the loaded weights");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(refresh(c, ROAM_BF16, false, s));
    // one tile of points of internal field 0 (the first field of width class 0)
    const int64_t n = 128;
    ROAM_TRY(ensure(c->selftest, (size_t)(10 * n + n / 2)));
    ROAM_TRY(ensure(c->sorted, (size_t)n));
    ROAM_TRY(ensure(c->tiles, tile_capacity(c, (size_t)n)));
    float *p = c->selftest.p, *d = p + 3 * n, *out = d + 3 * n;
    uint16_t *keys = reinterpret_cast<uint16_t *>(out + 4 * n);
    ROAM_CUDA(cudaMemsetAsync(c->selftest.p, 0, (size_t)(10 * n + n / 2) * sizeof(float), s));
    const BucketBufs b = bucket_of(c);
    ROAM_CUDA(cudaMemsetAsync(c->aux, 0, sizeof(Counters), s));
    launch_bucket(nullptr, nullptr, nullptr, (uint32_t)n, 1, 1, keys, c->n_fields, tile_of(ROAM_BF16), b, c->aux,
                  grid_blocks(c, 2), s, classes_of(c, ROAM_BF16));
    ROAM_TRY(launched("bucket"));
    SampleSrc src{};
    src.mode = 1;
    src.p = p;
    src.d = d;
    MlpWeights w = weights_of(c, 0);
    w.wait_ns = limit_ns;
    w.withhold_image = 1;
    launch_mlp_tc(w, false, src, b, c->aux, reinterpret_cast<float4 *>(out), c->n_sm, s);
    ROAM_TRY(launched("mlp_tc"));
    ROAM_CUDA(cudaStreamSynchronize(s));
    ROAM_CUDA(cudaMemcpy(&c->h_ctr[1], c->aux, sizeof(Counters), cudaMemcpyDeviceToHost));
    *observed = (int32_t)status_of(c->h_ctr[1].status);
    // the context stays usable: the self-test's status does not outlive it
    ROAM_CUDA(cudaMemset(c->aux, 0, sizeof(Counters)));
    c->last = s;
    return ROAM_OK;
}

roam_status roam_profile(roam_ctx *c, int enable)
{
    ROAM_TRY(set_dev(c));
    ROAM_CUDA(cudaDeviceSynchronize());
    for (auto &p : c->prof_pending) {
        c->ev_pool.push_back(p.second.first);
        c->ev_pool.push_back(p.second.second);
    }
    c->prof_pending.clear();
    c->prof_acc.assign(kProfKinds, {0, 0.0});
    c->prof = enable != 0;
    return ROAM_OK;
}

roam_status roam_profile_read(roam_ctx *c, roam_kernel_time *out, int max_entries, int *n_entries)
{
    ROAM_TRY(set_dev(c));
    if (!out || !n_entries || max_entries < 0) return fail(ROAM_ERR_ARG, "null output");
    ROAM_CUDA(cudaDeviceSynchronize());
    if (c->prof_acc.size() != (size_t)kProfKinds) c->prof_acc.assign(kProfKinds, {0, 0.0});
    for (auto &p : c->prof_pending) {
        float ms = 0.f;
        ROAM_CUDA(cudaEventElapsedTime(&ms, p.second.first, p.second.second));
        c->prof_acc[p.first].first += 1;
        c->prof_acc[p.first].second += ms;
        c->ev_pool.push_back(p.second.first);
        c->ev_pool.push_back(p.second.second);
    }
    c->prof_pending.clear();
    int n = 0;
    for (int k = 0; k < kProfKinds && n < max_entries; ++k) {
        if (!c->prof_acc[k].first) continue;
        memset(out[n].name, 0, sizeof(out[n].name));
        strncpy(out[n].name, kProfNames[k], sizeof(out[n].name) - 1);
        out[n].launches = c->prof_acc[k].first;
        out[n].total_ms = c->prof_acc[k].second;
        ++n;
    }
    *n_entries = n;
    return ROAM_OK;
}

roam_status roam_march(roam_ctx *c, const roam_camera *cams, int n_views, const uint32_t *rays, int64_t n_rays,
                       const roam_render_opts *opts, uint32_t *count, uint32_t *recs, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_grid || !c->has_fields) return fail(ROAM_ERR_STATE, "load grid and fields first");
    if (!opts || !(opts->delta > 0.f) || opts->n_max < 1 || opts->n_max > 1024)
        return fail(ROAM_ERR_ARG, "bad options");
    if (!count || !recs) return fail(ROAM_ERR_ARG, "null outputs");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n_pix = 0;
    ROAM_TRY(upload_cams(c, cams, n_views, opts->delta, &n_pix, s));
    if (!rays) n_rays = n_pix;
    if (n_rays < 0 || n_rays > 0x7fffffff) return fail(ROAM_ERR_ARG, "bad ray count");
    if (n_rays == 0) return ROAM_OK;
    ROAM_TRY(ensure_rays(c, n_rays, 1));
    MarchParams mp{};
    mp.cams = c->cams.p;
    mp.n_views = n_views;
    mp.rays = rays;
    mp.n_rays = (uint32_t)n_rays;
    mp.R = opts->n_max;
    mp.n_max = opts->n_max;
    mp.delta = opts->delta;
    mp.init = 1;
    mp.flat = 1;
    mp.accurate = opts->precision == ROAM_F32;      // the ray directions roam_render uses
    mp.st = state_of(c);
    mp.cnt = count;
    mp.recs = recs;
    mp.ctr = c->aux;
    ROAM_CUDA(cudaMemsetAsync(c->aux, 0, sizeof(Counters), s));
    launch_march(c->g, mp, march_grid(mp.n_rays), s);
    ROAM_TRY(launched("march"));
    if (c->permuted) {
        // records carry the caller's field ids
        k_unpermute_recs<<<grid_blocks(c, 4), 256, 0, s>>>(count, recs, n_rays, opts->n_max, c->inv.p);
        ROAM_TRY(launched("march field ids"));
    }
    c->last = s;
    return ROAM_OK;
}

roam_status roam_bucket(roam_ctx *c, const uint16_t *keys, int64_t n, uint32_t *perm, uint32_t *offsets, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_fields) return fail(ROAM_ERR_STATE, "load field labels first");
    if (n < 0 || n > 0x7fffffff) return fail(ROAM_ERR_ARG, "bad sample count");
    if (!offsets || (n > 0 && (!keys || !perm))) return fail(ROAM_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(ensure(c->tiles, tile_capacity(c, (size_t)n)));
    BucketBufs b = bucket_of(c);
    b.offsets = offsets;
    b.sorted = perm;
    ROAM_CUDA(cudaMemsetAsync(c->aux, 0, sizeof(Counters), s));
    launch_bucket(nullptr, nullptr, nullptr, (uint32_t)n, 1, 1, keys, c->n_fields, 128, b, c->aux, grid_blocks(c, 2), s,
                  ClassBounds{{0, c->n_fields, c->n_fields, c->n_fields}, {0, 0, 0, 0}});
    c->last = s;
    return launched("bucket");
}

roam_status roam_mlp_eval(roam_ctx *c, const float *p, const float *d, const uint16_t *field, int64_t n, int precision,
                          float *out, void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    if (n < 0 || n > 0x7fffffff) return fail(ROAM_ERR_ARG, "bad sample count");
    if (n == 0) return ROAM_OK;
    if (!p || !d || !field || !out) return fail(ROAM_ERR_ARG, "null pointer");
    if (precision != ROAM_F32 && precision != ROAM_BF16 && precision != ROAM_FP8)
        return fail(ROAM_ERR_ARG, "unknown precision");
    if ((precision == ROAM_BF16 && !all_tc(c, false)) || (precision == ROAM_FP8 && !all_tc(c, true)))
        return fail(ROAM_ERR_UNSUPPORTED, "tensor-core path not available");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(refresh(c, precision, false, s));
    ROAM_TRY(ensure(c->sorted, (size_t)n));
    ROAM_TRY(ensure(c->tiles, tile_capacity(c, (size_t)n)));
    const BucketBufs b = bucket_of(c);
    ROAM_CUDA(cudaMemsetAsync(c->aux, 0, sizeof(Counters), s));
    const uint16_t *keys = field;
    if (c->permuted) {
        ROAM_TRY(ensure(c->keys_tmp, (size_t)n));
        k_map_keys<<<grid_blocks(c, 2), 256, 0, s>>>(field, n, c->perm.p, c->n_fields, c->keys_tmp.p);
        ROAM_TRY(launched("field ids"));
        keys = c->keys_tmp.p;
    }
    launch_bucket(nullptr, nullptr, nullptr, (uint32_t)n, 1, 1, keys, c->n_fields, tile_of(precision), b, c->aux,
                  grid_blocks(c, 2), s, classes_of(c, precision));
    ROAM_TRY(launched("bucket"));
    SampleSrc src{};
    src.mode = 1;
    src.p = p;
    src.d = d;
    c->last = s;
    return run_mlp(c, precision, src, b, reinterpret_cast<float4 *>(out), c->aux, s);
}

roam_status roam_composite(roam_ctx *c, int64_t n_rays, int n_max, const uint32_t *count, const float *sigma_rgb,
                           const float *t, const roam_render_opts *opts, float *rgb, float *depth, float *opacity,
                           uint32_t *n_used, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!opts || !(opts->delta > 0.f) || !(opts->t_stop >= 0.f && opts->t_stop < 1.f))
        return fail(ROAM_ERR_ARG, "bad options");
    if (n_rays < 0 || n_max < 1) return fail(ROAM_ERR_ARG, "bad sizes");
    if (n_rays == 0) return ROAM_OK;
    if (!count || !sigma_rgb || !t) return fail(ROAM_ERR_ARG, "null input");
    if (((uintptr_t)sigma_rgb) & 15) return fail(ROAM_ERR_ARG, "sigma_rgb must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    launch_composite_flat(n_rays, n_max, count, reinterpret_cast<const float4 *>(sigma_rgb), t, opts->delta,
                          opts->t_stop, opts->bg, rgb, depth, opacity, n_used, s);
    c->last = s;
    return launched("composite");
}

roam_status roam_train_forward(roam_ctx *c, const roam_camera *cams, int n_views, const uint32_t *rays, int64_t n_rays,
                               const roam_render_opts *opts, float *rgb, void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    ROAM_TRY(check_opts(c, opts));
    if (opts->precision == ROAM_FP8) return fail(ROAM_ERR_UNSUPPORTED, "training runs in FP32 or BF16");
    if (!rays || !rgb) return fail(ROAM_ERR_ARG, "null rays or rgb");
    if (n_rays < 1 || n_rays > 0x7fffffff) return fail(ROAM_ERR_ARG, "bad ray count");
    if (c->n_ws != 1) return fail(ROAM_ERR_UNSUPPORTED, "training needs one MLP width for every field");
    if (!mlp_bwd_supported(c->md.width, c->md.n_hidden))
        return fail(ROAM_ERR_UNSUPPORTED, "training supports W = 32 or 64");
    cudaStream_t s = (cudaStream_t)stream;
    ROAM_TRY(refresh(c, opts->precision, false, s));
    int64_t n_pix = 0;
    ROAM_TRY(upload_cams(c, cams, n_views, opts->delta, &n_pix, s));
    // one round holding every kept sample of every ray, so the backward pass
    // finds each ray's samples in one place
    const int R = opts->n_max;
    if ((double)((n_rays + 31) & ~31LL) * R >= 4294967295.0) return fail(ROAM_ERR_ARG, "too many rays x samples");
    ROAM_TRY(ensure_rays(c, n_rays, R));
    ROAM_CUDA(cudaMemsetAsync(c->ctr, 0, sizeof(Counters), s));
    ROAM_CUDA(cudaMemsetAsync(c->hist.p, 0, (size_t)c->n_fields * sizeof(uint32_t), s));
    ROAM_TRY(run_rounds(c, rays, n_rays, opts, rgb, nullptr, nullptr, R, R, s));
    c->last = s;
    c->last_rays = n_rays;
    c->last_rounds = 1;
    c->train_rays = n_rays;
    c->train_R = R;
    c->train_opts = *opts;
    return ROAM_OK;
}

roam_status roam_train_backward(roam_ctx *c, const float *dl_drgb, float *grad, void *stream)
{
    ROAM_TRY(set_dev(c));
    ROAM_TRY(check_ready(c));
    if (c->train_rays <= 0) return fail(ROAM_ERR_STATE, "call roam_train_forward first");
    if (!dl_drgb || !grad) return fail(ROAM_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->train_rays;
    const int R = c->train_R;
    const roam_render_opts &o = c->train_opts;
    const size_t slots = ((size_t)(n + 31) & ~(size_t)31) * (size_t)R;
    ROAM_TRY(ensure(c->gsr, slots));
    // the composite's adjoint also counts the composited samples per field,
    // so the backward bucketing needs no histogram pass of its own
    const bool fused_hist = (size_t)c->n_fields * sizeof(uint32_t) <= 48 * 1024;
    if (fused_hist) ROAM_CUDA(cudaMemsetAsync(c->hist.p, 0, (size_t)c->n_fields * sizeof(uint32_t), s));
    {
        ProfScope ps(c, P_COMPOSITE_BWD, s);
        launch_composite_bwd(n, R, c->cnt.p, c->recs.p, c->sr.p, o.delta, o.t_stop, o.bg, dl_drgb, c->gsr.p,
                             c->live1.p, fused_hist ? c->hist.p : nullptr, c->n_fields, s);
    }
    ROAM_TRY(launched("composite_bwd"));
    ROAM_CUDA(cudaMemsetAsync(c->aux, 0, sizeof(Counters), s));
    const BucketBufs b = bucket_of(c);
    {
        ProfScope ps(c, P_BUCKET, s);
        if (fused_hist)
            launch_bucket_ready(c->live1.p, c->recs.p, nullptr, (uint32_t)n, R, 1, c->n_fields, 128, b, c->aux,
                                grid_blocks(c, 4), s, c->cb);
        else
            launch_bucket(c->live1.p, c->recs.p, nullptr, (uint32_t)n, R, 1, nullptr, c->n_fields, 128, b, c->aux,
                          grid_blocks(c, 4), s, c->cb);
    }
    ROAM_TRY(launched("bucket"));
    ROAM_CUDA(cudaMemsetAsync(grad, 0, (size_t)(c->ws[0].P * c->n_fields) * sizeof(float), s));
    SampleSrc src{};
    src.mode = 0;
    src.recs = c->recs.p;
    src.live = nullptr;
    src.live_count = nullptr;
    src.R = R;
    src.st = state_of(c);
    src.delta = o.delta;
    src.accurate = o.precision == ROAM_F32;
    const bool tc = o.precision == ROAM_BF16 && mlp_bwd_tc_supported(c->md.width, c->md.n_hidden) && c->ws[0].tc_ok;
    if (!tc) ROAM_TRY(refresh(c, o.precision, true, s));
    if (tc) {
        ProfScope ps(c, P_MLP_BWD_TC, s);
        launch_mlp_bwd_tc(weights_of(c), src, b, c->aux, c->gsr.p, grad, c->n_sm, s);
    } else {
        ProfScope ps(c, P_MLP_BWD, s);
        launch_mlp_bwd_simt(weights_of(c), src, b, c->aux, c->gsr.p, grad, c->n_sm, s);
    }
    c->last = s;
    return launched("mlp_bwd");
}

roam_status roam_l2_loss(roam_ctx *c, const float *rgb, const float *target, int64_t n_rays, float norm,
                         float *dl_drgb, float *loss, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (n_rays < 0) return fail(ROAM_ERR_ARG, "bad ray count");
    if (!(norm > 0.f) || !finite(norm)) return fail(ROAM_ERR_ARG, "norm must be positive");
    if (n_rays == 0) return ROAM_OK;
    if (!rgb || !target || !dl_drgb) return fail(ROAM_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    launch_l2_loss(n_rays, rgb, target, norm, dl_drgb, loss, s);
    c->last = s;
    return launched("l2_loss");
}

roam_status roam_adam_step(roam_ctx *c, const float *grad, const roam_adam_cfg *cfg, void *stream)
{
    ROAM_TRY(set_dev(c));
    if (!c->has_weights) return fail(ROAM_ERR_STATE, "no weights loaded");
    if (!grad || !cfg) return fail(ROAM_ERR_ARG, "null pointer");
    if (!(cfg->lr >= 0.f) || !finite(cfg->lr) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
        !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f) || cfg->step < 1)
        return fail(ROAM_ERR_ARG, "bad Adam configuration");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->n_ws != 1) return fail(ROAM_ERR_UNSUPPORTED, "training needs one MLP width for every field");
    WSet &q = c->ws[0];
    const int64_t n = q.P * c->n_fields;
    ROAM_TRY(ensure(c->adam_m, (size_t)n));
    ROAM_TRY(ensure(c->adam_v, (size_t)n));
    if (c->adam_fresh) {
        ROAM_CUDA(cudaMemsetAsync(c->adam_m.p, 0, n * sizeof(float), s));
        ROAM_CUDA(cudaMemsetAsync(c->adam_v.p, 0, n * sizeof(float), s));
        c->adam_fresh = false;
    }
    const float bc1 = (float)(1.0 - std::pow((double)cfg->beta1, (double)cfg->step));
    const float bc2 = (float)(1.0 - std::pow((double)cfg->beta2, (double)cfg->step));
    {
        ProfScope ps(c, P_ADAM, s);
        // the BF16 images now (in the same pass where they fold every bias);
        // the other derived copies when a launch needs them
        const int W = c->md.width, H = c->md.n_hidden;
        const bool fused = q.tc_ok && launch_adam_tc(q.w32.p, c->adam_m.p, c->adam_v.p, grad, c->n_fields, W, H, q.P,
                                                     q.wimg.p, q.img_bytes, cfg->lr, cfg->beta1, cfg->beta2, cfg->eps,
                                                     bc1, bc2, s);
        if (!fused) {
            launch_adam(q.w32.p, c->adam_m.p, c->adam_v.p, grad, n, cfg->lr, cfg->beta1, cfg->beta2, cfg->eps, bc1,
                        bc2, s);
            if (q.tc_ok) launch_pack_tc(q.w32.p, c->n_fields, W, H, q.P, q.wimg.p, q.img_bytes, false, s);
        }
        q.stale |= kStaleWt | kStaleWr | (q.tc8_ok ? kStaleImg8 : 0u);
        if (!q.tc_ok) ROAM_TRY(refresh(c, ROAM_F32, true, s));
    }
    c->last = s;
    return launched("adam");
}

}  // extern "C"
