/*
 * roam.h -- C ABI of the GB300 renderer for geometry-aware local radiance
 * fields (360Roam, arXiv 2208.02705): an occupancy grid whose occupied voxels
 * are labelled with one of n tiny MLPs, rendered by ray casting with
 * empty-space skipping, parallel per-field MLP queries and volume rendering
 * with early termination, plus the training step of the fine-tuning stage.
 *
 * Conventions for every entry point:
 *   - Plain pointers and sizes only.  Arguments documented "device" are
 *     CUDA device pointers on the context's device; "host" are host pointers.
 *     The caller owns every buffer it passes; the library owns its own copies
 *     of the grid, labels and weights, and its workspace, and frees them in
 *     roam_destroy.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued asynchronously unless the entry point says it synchronises.
 *   - Every call validates its arguments and returns a roam_status; it never
 *     aborts the process.  roam_last_error() gives a message for the calling
 *     thread's last failure.  Kernels that detect bad data or a timed-out wait
 *     record it in a device status word; synchronising calls (and
 *     roam_check()) turn it into ROAM_ERR_DATA / ROAM_ERR_TIMEOUT.
 *   - A context is bound to one device and must be used by one host thread at
 *     a time.
 */
#ifndef ROAM_H
#define ROAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct roam_ctx roam_ctx;

typedef enum {
    ROAM_OK = 0,
    ROAM_ERR_ARG = -1,         /* invalid argument (size, pointer, alignment, id) */
    ROAM_ERR_OOM = -2,         /* device allocation failed */
    ROAM_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    ROAM_ERR_STATE = -4,       /* call out of order (e.g. render before load) */
    ROAM_ERR_TIMEOUT = -5,     /* a device-side wait hit its iteration limit */
    ROAM_ERR_DATA = -6,        /* inconsistent data found on the device */
    ROAM_ERR_UNSUPPORTED = -7  /* valid request with no kernel for it (shape or precision) */
} roam_status;

enum { ROAM_F32 = 0, ROAM_BF16 = 1, ROAM_FP8 = 2 };   /* arithmetic */
enum { ROAM_EQUIRECT = 0, ROAM_PERSPECTIVE = 1 };     /* camera models */
enum { ROAM_SOFTPLUS = 0, ROAM_RELU = 1 };            /* density activation */

/* Occupancy grid geometry.  dims = (Gx, Gy, Gz), Gx a multiple of 32, each
 * dimension a multiple of 8 and at most 2048.  Voxel (x, y, z) covers
 * [origin + i*vox, origin + (i+1)*vox) on each axis. */
typedef struct {
    int32_t dims[3];
    float origin[3];
    float vox;
} roam_grid_desc;

/* Tiny-MLP architecture shared by all fields (slim-network table of the
 * paper's appendix, read as: layer 1 (63 -> W), n_hidden - 1 layers W -> W,
 * head W -> 1 + W (density logit, then W features, no activation on the
 * features), colour layer (W + 27 -> W, ReLU), output W -> 3 (sigmoid)).
 * Positional encodings: 63 features of the field-local position (L = 10)
 * and 27 of the world view direction (L = 4), each [x, sin(2^k pi x),
 * cos(2^k pi x)], three sines then three cosines per frequency.
 * density = sigma_scale * softplus(s)  (or ReLU(s) with ROAM_RELU). */
typedef struct {
    int32_t width;        /* W: 32, 64 or 128 */
    int32_t n_hidden;     /* H: 1..4 trunk layers */
    float sigma_scale;
    int32_t density_act;  /* ROAM_SOFTPLUS or ROAM_RELU */
} roam_mlp_desc;

/* Camera (Eq. 2 and Eq. 3 for equirectangular views; pinhole with square
 * pixels and focal length (width/2)/tan(fov_h/2) for perspective views).
 * Camera frame: x right, y down, z forward; pixel (u, v) has its centre at
 * (u + 1/2, v + 1/2); the world ray is o + t * R d_cam, t >= 0. */
typedef struct {
    int32_t model;        /* ROAM_EQUIRECT or ROAM_PERSPECTIVE */
    int32_t width, height;
    float fov_h;          /* radians, perspective only */
    float R[9];           /* camera-to-world rotation, row-major */
    float o[3];           /* camera centre, world units */
} roam_camera;

/* Sampling and compositing options.  Sample j of a ray sits at
 * t_j = (j + 1/2) * delta and is kept iff its voxel is occupied (dense
 * sampling of occupied voxels only); at most n_max kept samples per ray.
 * Compositing (Eq. 4-5) stops after the first sample whose transmittance
 * falls below t_stop; the background bg is added with the final
 * transmittance. */
typedef struct {
    float delta;          /* > 0, world units */
    int32_t n_max;        /* 1..1024 */
    float t_stop;         /* e.g. 1e-4; 0 disables early termination */
    float bg[3];
    int32_t precision;    /* ROAM_F32 (SIMT FP32), ROAM_BF16 (tcgen05 BF16, FP32 accumulate) or
                             ROAM_FP8 (tcgen05 E4M3 weights with one FP32 scale per output
                             channel, E4M3 activations, FP32 accumulate, FP32 biases; render
                             and roam_mlp_eval only) */
    int32_t round_size;   /* kept samples marched per ray per round, 0 = library default */
    int32_t use_graph;    /* 1: roam_render captures its launch sequence into a CUDA graph
                             (once per configuration: view sizes, options, output pointers)
                             and replays it on later calls; 0: plain launches */
    int32_t first_round_size; /* kept samples marched per ray in the first round (at most
                             round_size), 0 = round_size.  The render's result does not
                             depend on the round sizes; the work does: samples marched past
                             a ray's termination within a round are evaluated for nothing */
} roam_render_opts;

/* Counters of the last render / training forward (read with a sync). */
typedef struct {
    int64_t n_rays;
    int64_t n_samples;    /* kept samples evaluated through the MLPs */
    int64_t n_used;       /* samples composited (up to each ray's termination) */
    int32_t n_rounds;
    int32_t n_fields_hit; /* sum over rounds of fields with at least one sample */
} roam_stats;

/* Device time of one kind of kernel launch, from CUDA events recorded on the
 * launching stream around each launch while profiling is on. */
typedef struct {
    char name[24];
    int64_t launches;
    double total_ms;
} roam_kernel_time;

/* Adam (Sec. "Training Details and Parameters": beta = (0.9, 0.99), learning
 * rate decaying exponentially from 1e-3 to 5e-5). */
typedef struct {
    float lr;             /* learning rate of this step */
    float beta1, beta2, eps;
    int32_t step;         /* 1-based step number, for bias correction */
} roam_adam_cfg;

/* ---- context --------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  *ctx receives the handle. */
roam_status roam_create(roam_ctx **ctx, int device);
/* Frees every allocation of the context; NULL is accepted. */
roam_status roam_destroy(roam_ctx *ctx);
/* Message of the calling thread's last failed call ("" if none). */
const char *roam_last_error(void);
/* Synchronises the context's last stream and reports any device status. */
roam_status roam_check(roam_ctx *ctx);

/* ---- scene ----------------------------------------------------------- */

/* Loads the occupancy map O (Alg. 1 stage I output; voxels with occupied
 * probability above 0.97, Sec. "Progressive Probabilistic Geometry
 * Estimation").  bits: uint32[Gz][Gy][Gx/32], bit b of word w in a row is
 * voxel x = 32 w + b.  bits_on_device selects device or host memory.
 * Builds the per-word rank prefix and an 8^3 brick occupancy map on the
 * device.  Invalidates loaded fields.  Synchronises. */
roam_status roam_load_grid(roam_ctx *ctx, const roam_grid_desc *desc, const uint32_t *bits,
                           int bits_on_device);

/* Loads the voxel-to-field labelling (Alg. 1 stage II output: every occupied
 * voxel names the tiny MLP that models it, Sec. "Real-time Rendering
 * Speedup").  field_of_rank[r] (uint16) is the field of the r-th
 * occupied voxel in linear order (z*Gy + y)*Gx + x; n_occupied must equal the
 * number of set bits.  affine: float[n_fields][6] = (scale xyz, offset xyz),
 * the field-local position being scale * p + offset.  Arrays are device
 * memory iff on_device.  Labels >= n_fields give ROAM_ERR_ARG.  Synchronises. */
roam_status roam_load_fields(roam_ctx *ctx, int n_fields, const uint16_t *field_of_rank,
                             int64_t n_occupied, const float *affine, int on_device);

/* Loads per-field MLP weights: float[n_fields][P] in layer order W1, b1,
 * (Wk, bk) x (H-1), Wh, bh, Wc, bc, Wo, bo, matrices row-major [out][in]
 * (P = 6,212 for W=32/H=2).  Keeps FP32 masters and builds the BF16 tensor
 * core images.  Device memory iff on_device.  Synchronises. */
roam_status roam_load_weights(roam_ctx *ctx, const roam_mlp_desc *desc, const float *weights,
                              int on_device);

/* Loads per-field MLPs of mixed widths (each field 32, 64 or 128 wide, all
 * with desc->n_hidden hidden layers; desc->width is ignored).  field_width:
 * host int32[n_fields]; weights: host or device (on_device) float32, field
 * after field in the caller's field order, each field in the layout of
 * roam_load_weights for its own width.
 * Internally the fields are grouped by width and each group runs its own
 * kernel over its own tiles; field ids seen through the ABI (roam_march
 * records, roam_mlp_eval keys, roam_get_weights order) stay the caller's.
 * Rendering and roam_mlp_eval accept every precision; training
 * (roam_train_forward, roam_adam_step) needs a single width.  Synchronous. */
roam_status roam_load_weights_mixed(roam_ctx *ctx, const roam_mlp_desc *desc, const int32_t *field_width,
                                    const float *weights, int on_device);

/* Copies the FP32 master weights (same layout as roam_load_weights, or as
 * roam_load_weights_mixed when the widths are mixed) to `out` (device memory
 * iff on_device).  Synchronises. */
roam_status roam_get_weights(roam_ctx *ctx, float *out, int on_device);

/* ---- rendering (Sec. "Real-time Rendering Speedup", Eq. 2-5) ---------- */

/* Renders n_views cameras (host array).  Pixels of all views are
 * concatenated in view order, row-major within a view: rgb float[N][3],
 * depth float[N], opacity float[N] (either may be NULL), N = sum of
 * width*height.  out_on_device = 1: outputs are device pointers and the call
 * is asynchronous on `stream`; 0: host pointers, the library copies the
 * result back and synchronises `stream`. */
roam_status roam_render(roam_ctx *ctx, const roam_camera *cams, int n_views,
                        const roam_render_opts *opts, float *rgb, float *depth, float *opacity,
                        int out_on_device, void *stream);

/* Parameters of the occupancy update (Eq. 6): measurement probabilities of
 * a confident end point (p_hit) and of a crossed voxel (p_miss), the
 * log-odds clamp [l_min, l_max], the occupancy threshold p_occ, and the
 * opacity below which a pixel carries no measurement (a_min).  The paper's
 * values: l_min = -2, l_max = 3.5, p_occ = 0.97; the library's defaults
 * p_hit = 0.7, p_miss = 0.4, a_min = 0.5 (24 bytes). */
typedef struct {
    float p_hit, p_miss, l_min, l_max, p_occ, a_min;
} roam_occ_params;

/* Progressive probabilistic occupancy update (Eq. 6; Alg. 1 stage I) on the
 * loaded grid's voxel lattice, one scan per camera in order.  depth and
 * opacity: device float per pixel of every view in order (roam_render's
 * depth and opacity outputs: D = sum w t, A = sum w).  Each pixel with
 * A >= a_min measures its ray's end point o + (D / A) d: the voxels whose
 * interior the segment crosses are observed free, the end point's voxel
 * occupied with confidence A (occupied wins; one update per voxel per scan:
 * L += logit(1/2 + (p_hit - 1/2) A_max) or L += logit(p_miss)), then L is
 * clamped to [l_min, l_max].  logit: device float[gz][gy][gx], in/out.
 * bits (device, may be NULL): the occupancy bit grid (same layout as
 * roam_load_grid; bit set iff L > logit(p_occ)) after the last scan.
 * Asynchronous on `stream`. */
roam_status roam_occupancy_update(roam_ctx *ctx, const roam_camera *cams, int n_views, const float *depth,
                                  const float *opacity, const roam_occ_params *params, float *logit,
                                  uint32_t *bits, void *stream);

/* Adaptive assignment of the loaded grid's occupied voxels to n_fields
 * networks (Alg. 1 stage II): network k takes the smallest unassigned voxel
 * (lexicographic (z, y, x): the smallest linear index) as its anchor and
 * the s - 1 unassigned voxels nearest to it (squared distance in voxel
 * units, ties to the smaller linear index), s = S / n_fields; the last
 * network takes every voxel left.  labels: device uint16[S], the network of
 * every occupied voxel in rank order (the layout roam_load_fields takes);
 * boxes (device int32[n_fields][6], may be NULL): each network's voxel
 * bounding box (min x, y, z, max x, y, z exclusive).  Synchronises. */
roam_status roam_assign_fields(roam_ctx *ctx, int n_fields, uint16_t *labels, int32_t *boxes, void *stream);

/* Distillation of the local fields from the global 360NeRF (Eq. 7).
 *
 * roam_teacher_load: the teacher's FP32 parameters (host, or device when
 * on_device) in its layer order -- layers 1-4 (63 -> 256, 256 -> 256 x 3),
 * layer 5 on [layer 4 (256); F(x) (63)], layers 6-8, the density head
 * (256 -> 1), the feature head (256 -> 256), layer 10 on [feature (256);
 * F(d) (27)] -> 128, layer 11 (128 -> 3); each layer row-major [out][in]
 * then its bias -- 595,844 floats; affine (host float[6]): the global
 * position's map onto [-1, 1]^3 (scale xyz, offset xyz).  Synchronous. */
roam_status roam_teacher_load(roam_ctx *ctx, const float *weights, const float *affine, int on_device);

/* The teacher at n points: p, d device float[n][3] (world position, view
 * direction); out device float[n][4] = (sigma, r, g, b), 16-byte aligned.
 * precision ROAM_BF16: the matrix layers on the tensor cores (tcgen05, BF16
 * inputs and weights, FP32 accumulation; layers 1, 5 and 10 take their bias
 * as a BF16 product term, the others add it in FP32), the density head and
 * layer 11 in FP32 on the CUDA cores; ROAM_F32: every layer in FP32 on the
 * CUDA cores.  The encodings are FP32 in both.  Asynchronous. */
roam_status roam_teacher_eval(roam_ctx *ctx, const float *p, const float *d, int64_t n, int precision, float *out,
                              void *stream);

/* Eq. 7 over n samples: *loss (device, may be NULL) = sum over samples of
 * [(sigma_s - sigma_t)^2 + |c_s - c_t|^2] / I, and dl_dout = 2 (student -
 * teacher) / I per component; student, teacher, dl_dout device
 * float[n][4], 16-byte aligned.  The sum runs in a fixed order.
 * Asynchronous. */
roam_status roam_distill_loss(roam_ctx *ctx, const float *student, const float *teacher, int64_t n, float I,
                              float *dl_dout, float *loss, void *stream);

/* Gradient of the loaded fields' weights at n points given the loss
 * gradient of every sample's output: p, d device float[n][3], field device
 * uint16[n], dl_dout device float[n][4] (d loss / d (sigma, r, g, b));
 * grad device float[n_fields][P] (overwritten), the layout of
 * roam_load_weights.  One MLP width (32 or 64) for every field.
 * precision ROAM_F32: FP32 SIMT adjoint (recomputes the forward pass in
 * FP32); ROAM_BF16: tcgen05 adjoint of the BF16 forward pass (BF16
 * operands, FP32 accumulation; W = 32 with H <= 4 or W = 64 with H <= 3,
 * else ROAM_ERR_UNSUPPORTED).  Asynchronous. */
roam_status roam_mlp_backward(roam_ctx *ctx, const float *p, const float *d, const uint16_t *field, int64_t n,
                              int precision, const float *dl_dout, float *grad, void *stream);

/* Chooses the round sizes (kept samples marched per live ray per round) for
 * this camera batch and these options: renders the batch once per candidate
 * round size (4, 8, 16, ... up to n_max, while the workspace fits in half
 * the free device memory and slot ids in 32 bits), then, with the fastest,
 * once per smaller first-round size (4, 8, ...), each after one warm-up
 * render, timing with CUDA events on `stream`.  Returns the fastest pair in
 * *best_round_size and *best_first_round_size (may be NULL), its time in
 * *best_ms (may be NULL).  Pass them back as roam_render_opts.round_size and
 * .first_round_size.  Synchronous. */
roam_status roam_tune_round_size(roam_ctx *ctx, const roam_camera *cams, int n_views, const roam_render_opts *opts,
                                 int32_t *best_round_size, int32_t *best_first_round_size, float *best_ms,
                                 void *stream);

/* Counters of the last roam_render / roam_train_forward (synchronises); the
 * single-step entry points and the backward passes keep counters of their
 * own and leave these as they are. */
roam_status roam_get_stats(roam_ctx *ctx, roam_stats *stats);

/* Pads every field's run of 128-sample tiles on the tensor-core paths to a
 * multiple of `tiles` (a multiple of 4 in [4, 64]) instead of each MLP
 * kernel's own tiles in flight (0, the default).  Results do not depend on
 * it: the padding tiles hold no samples, and a kernel then meets groups of
 * tiles in which no slot has work.  Meant for testing that every kernel
 * handles such groups; it only adds work.  ROAM_ERR_ARG for other values. */
roam_status roam_set_tile_padding(roam_ctx *ctx, int tiles);

/* Self-test of the bounded device-side waits: runs the tensor-core MLP
 * kernel of the loaded weights once over a tile of 128 points of one field
 * with the copy of that field's weight image withheld, so that every wait
 * for the image runs out after limit_ns (1e6 .. 1e10 ns) instead of the
 * 2 s the kernels otherwise allow.  The kernel then flags the timeout in
 * its status word, lets its other threads leave at their next barrier,
 * finishes the commits it issued, frees its tensor memory and returns;
 * nothing is copied or computed on the withheld image.  Synchronises.
 * *observed receives the status a synchronising call reports for that
 * launch (ROAM_ERR_TIMEOUT when the path works); the flag is then cleared,
 * so the context stays usable.  ROAM_ERR_UNSUPPORTED without tensor-core
 * weights. */
roam_status roam_selftest_wait_timeout(roam_ctx *ctx, uint64_t limit_ns, int32_t *observed, void *stream);

/* Turns per-kernel event timing on (clearing earlier records) or off.  While
 * on, every kernel launch of roam_render / roam_train_* is bracketed by two
 * CUDA events on its stream (a small overhead). */
roam_status roam_profile(roam_ctx *ctx, int enable);

/* Reads the accumulated per-kernel times (synchronises): up to max_entries
 * entries into out, *n_entries receives the number written. */
roam_status roam_profile_read(roam_ctx *ctx, roam_kernel_time *out, int max_entries, int *n_entries);

/* ---- the steps of the render path, exposed one by one ----------------- */

/* Ray generation + DDA march + field lookup for n_rays rays (view, pixel)
 * pairs (device uint32[n_rays][2]; NULL = every pixel of every view in
 * order).  No compositing, no termination: per ray, the first n_max kept
 * samples.  count: device uint32[n_rays]; recs: device uint32[n_rays][n_max],
 * entry = j | field << 16.  The rays are generated as roam_render generates
 * them under the same options (opts->precision selects the FP32 render's
 * directions, rounded from FP64, or the reduced-precision renders' FP32
 * ones), so the records are exactly the samples roam_render composites, up
 * to each ray's termination.  Asynchronous. */
roam_status roam_march(roam_ctx *ctx, const roam_camera *cams, int n_views, const uint32_t *rays,
                       int64_t n_rays, const roam_render_opts *opts, uint32_t *count,
                       uint32_t *recs, void *stream);

/* Buckets n samples by field: keys device uint16[n] (field ids < n_fields);
 * perm device uint32[n] receives the sample indices grouped by field in
 * increasing field order (order within a field unspecified); offsets device
 * uint32[n_fields + 1] the group boundaries.  Asynchronous. */
roam_status roam_bucket(roam_ctx *ctx, const uint16_t *keys, int64_t n, uint32_t *perm,
                        uint32_t *offsets, void *stream);

/* Positional encoding + per-field MLP at n world points: p, d device
 * float[n][3] (d the world view direction), field device uint16[n];
 * out device float[n][4] = (sigma, r, g, b).  precision ROAM_F32, ROAM_FP8 or
 * ROAM_BF16.  Asynchronous. */
roam_status roam_mlp_eval(roam_ctx *ctx, const float *p, const float *d, const uint16_t *field,
                          int64_t n, int precision, float *out, void *stream);

/* Allocation-free variant of roam_bucket, for callers that may not allocate
 * device memory: hosts whose own pool allocator owns every device byte, or
 * frame loops that cannot afford the device-wide synchronisation cudaFree
 * brings.  (The paper has no counterpart: this is a service of the library.)
 * Needs no context and never calls cudaMalloc, cudaFree or an allocating
 * library routine: its scratch is a fixed array of about 96 KiB in device
 * memory, created when the library is loaded and held by every GPU that
 * loads it until the process exits.
 *   keys    device uint16[n], field ids; ids >= n_fields are dropped
 *   n       0 .. 2^31 - 1
 *   n_fields 1 .. 4096; more gives ROAM_ERR_ARG (the scratch is sized for 4096)
 *   perm    device uint32[n]: sample indices grouped by field, fields in
 *           increasing order (order within a field unspecified); entries
 *           from offsets[n_fields] (the number of samples kept) to n - 1
 *           are left unwritten when ids were dropped
 *   offsets device uint32[n_fields + 1]: group boundaries
 * Works on the calling thread's current device and is asynchronous on
 * `stream`.  The first successful call on each device looks up the scratch
 * array's device address (cudaGetSymbolAddress) and keeps it; make that
 * first call before any stream capture, and do not use this entry point
 * after a cudaDeviceReset of the device (the kept address would be stale).
 * All calls share the one array and it keeps the previous call's contents
 * (each call clears what must start at zero), so calls whose work overlaps
 * on the GPU -- e.g. on two streams -- race: serialise them. */
roam_status roam_bucket_static(const uint16_t *keys, int64_t n, int n_fields, uint32_t *perm,
                               uint32_t *offsets, void *stream);

/* Compositing with early termination (Eq. 4-5) of n_rays rays holding
 * count[r] <= n_max samples: sigma_rgb device float[n_rays][n_max][4]
 * (sigma, r, g, b), t device float[n_rays][n_max] sample depths; outputs as
 * roam_render (device), n_used device uint32[n_rays] (may be NULL) = samples
 * composited before termination.  Uses opts->delta, t_stop, bg.
 * Asynchronous. */
roam_status roam_composite(roam_ctx *ctx, int64_t n_rays, int n_max, const uint32_t *count,
                           const float *sigma_rgb, const float *t, const roam_render_opts *opts,
                           float *rgb, float *depth, float *opacity, uint32_t *n_used, void *stream);

/* ---- training (Sec. "Adaptive Radiance Fields Slimming and Fine-tuning":
 *      L2 photometric loss over rendered pixels, dense sampling of occupied
 *      voxels) ---------------------------------------------------------- */

/* Forward pass of the fine-tuning step for n_rays rays (device
 * uint32[n_rays][2] of (view, pixel)); rgb device float[n_rays][3].  Keeps
 * what the backward pass needs inside the context.  Asynchronous. */
roam_status roam_train_forward(roam_ctx *ctx, const roam_camera *cams, int n_views,
                               const uint32_t *rays, int64_t n_rays, const roam_render_opts *opts,
                               float *rgb, void *stream);

/* Backward pass of the last roam_train_forward: dl_drgb device
 * float[n_rays][3]; grad device float[n_fields][P] receives d(loss)/d(weights)
 * (overwritten), in the layout of roam_load_weights.  Recomputes the
 * positional encodings and MLP activations instead of storing them.  The
 * MLP adjoint follows the forward's precision: FP32 SIMT after a ROAM_F32
 * forward, tcgen05 BF16 after a ROAM_BF16 one (FP32 SIMT where the shape is
 * outside the tensor-core adjoint's, see roam_mlp_backward).  Asynchronous. */
roam_status roam_train_backward(roam_ctx *ctx, const float *dl_drgb, float *grad, void *stream);

/* L2 photometric loss of the fine-tuning stage on device arrays rgb and
 * target (float[n_rays][3]): *loss (device float, may be NULL) receives
 * sum (rgb - target)^2 / norm and dl_drgb (device float[n_rays][3])
 * 2 (rgb - target) / norm.  norm = 3 n for the mean over a batch of n rays;
 * with data parallelism, 3 n over the global batch so that summed per-rank
 * gradients equal the global one.  The sum runs in a fixed order: the same
 * inputs give the same bits.  Asynchronous. */
roam_status roam_l2_loss(roam_ctx *ctx, const float *rgb, const float *target, int64_t n_rays, float norm,
                         float *dl_drgb, float *loss, void *stream);

/* Adam update of the FP32 master weights with grad (device, layout of
 * roam_load_weights); refreshes the BF16 images.  Asynchronous. */
roam_status roam_adam_step(roam_ctx *ctx, const float *grad, const roam_adam_cfg *cfg, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ROAM_H */
