/*
 * FP64 CPU oracle for the geometry-aware local-MLP renderer (360Roam, arXiv
 * 2208.02705).  TEST INFRASTRUCTURE ONLY: the tests, the package's smoke
 * check and the benchmark's CPU-baseline leg may call it; the rendering
 * library never does.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Every function is the plain definition of one step of the method, written
 * as loops in double precision, with no bucketing, skipping structure,
 * blocking or fusion:
 *
 *   orc_ray          pixel -> ray (Eq. 2 and Eq. 3; pinhole model for
 *                    perspective views)
 *   orc_label_map    rank of an occupied voxel -> its field label, by a
 *                    linear scan of the grid (Sec. "Real-time Rendering
 *                    Speedup": every occupied voxel is labelled with its MLP)
 *   orc_march        regular samples t_j = (j + 1/2) * delta kept iff their
 *                    voxel is occupied (Sec. "Adaptive Radiance Fields
 *                    Slimming and Fine-tuning": dense sampling of occupied
 *                    voxels only), brute force over every j
 *   orc_mlp          positional encoding (Eq. 1 and its encoding F(.)) and the
 *                    tiny MLP of the slim-network table (Appendix, network
 *                    architecture details)
 *   orc_composite    Eq. 4 / Eq. 5 with early ray termination
 *   orc_render       all of the above per ray
 *   orc_loss_grad    L2 photometric loss of the fine-tuning stage and its
 *                    analytic reverse-mode gradient w.r.t. every MLP weight
 *   orc_occupancy_update  the log-odds occupancy recursion of Eq. 6 over
 *                    scans of rendered depth and opacity (Alg. 1 stage I)
 *   orc_assign_fields  the anchor + nearest-neighbour assignment of occupied
 *                    voxels to networks (Alg. 1 stage II)
 *   orc_teacher_eval   the global 360NeRF of the implementation details (the
 *                    distillation teacher)
 *   orc_distill_loss_grad  the distillation loss of Eq. 7 and its gradient
 *
 * Readings of the paper taken here (the paper is silent or garbled on these):
 *   - pixel centres at (u + 1/2, v + 1/2);
 *   - camera frame x right, y down, z forward; world direction d = R d_cam;
 *   - delta_i = delta for every kept sample (samples in empty voxels carry
 *     zero density and are skipped);
 *   - the paper's per-sample weight "T_i" of Eq. 5 is called w_i here and T
 *     is the transmittance;
 *   - termination after the first sample whose post-sample transmittance is
 *     below t_stop; background colour added with the final transmittance;
 *   - F(x) = [x, sin(2^k pi x), cos(2^k pi x)] for k < L, grouped per
 *     frequency (three sines, then three cosines), L = 10 for the field-local
 *     position and L = 4 for the world view direction (63 and 27 features,
 *     which reproduce the paper's 6,212 parameters per tiny network);
 *   - density = sigma_scale * softplus(s) (or ReLU(s) when act == 1);
 *     the feature branch of the head has no activation; colour = sigmoid.
 *
 * The reduced-precision reading (quant == 1, the library's FP8 path; the
 * paper fixes no arithmetic format): every matrix layer but the 3-output
 * one takes its inputs rounded to FP8 E4M3 and its weights rounded to E4M3
 * after division by a per-output-row scale s = max |row| / 448 (s and the
 * division in FP32), then y = bias + s * sum(products), everything else in
 * FP64 as above.
 *
 * The BF16 reading (quant == 2, the library's BF16 tensor-core path at
 * W <= 64, where every bias rides in the matrix product): every matrix
 * layer but the 3-output one takes its inputs, weights and bias rounded to
 * BF16 (8 significant bits, nearest, ties to even) and sums in FP64; the
 * 3-output layer stays FP64 on the FP32 weights.  Its adjoint rounds to BF16
 * what that path keeps as BF16 operands: each layer's output gradient dz
 * (after the ReLU mask), the layer inputs it multiplies, and the weights of
 * the products that carry dz down; the 3-output layer's dz and its input g
 * enter its weight gradient rounded too.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PE_POS 63
#define ORC_PE_DIR 27
#define ORC_TIE_EPS 1e-3   /* voxel units: FP32 coordinates carry ~1e-4 */

/* ------------------------------------------------------------------ */
/* parameters                                                           */
/* ------------------------------------------------------------------ */

/* Parameter count of one tiny MLP: layer 1 (63 -> W), H-1 hidden layers
 * (W -> W), head (W -> 1 + W), colour layer (W + 27 -> W), output (W -> 3),
 * each with a bias. */
int64_t orc_param_count(int W, int H)
{
    int64_t p = 0;
    p += (int64_t)W * ORC_PE_POS + W;
    p += (int64_t)(H - 1) * ((int64_t)W * W + W);
    p += (int64_t)(1 + W) * W + (1 + W);
    p += (int64_t)W * (W + ORC_PE_DIR) + W;
    p += 3 * (int64_t)W + 3;
    return p;
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Number of host threads the parallel loops use from now on (timing only) */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* ray generation: Eq. 2 (pixel <-> longitude/latitude) and Eq. 3       */
/* ------------------------------------------------------------------ */

/* cam = (model, width, height, fov_h, R[9] row-major camera-to-world, o[3]).
 * (uc, vc) are continuous pixel coordinates; a pixel's centre is u + 1/2. */
void orc_ray(const double *cam, double uc, double vc, double *o, double *d)
{
    int model = (int)cam[0];
    double W = cam[1], H = cam[2], fov = cam[3];
    const double *R = cam + 4;
    double dc[3];
    if (model == 0) {
        /* Eq. 2 inverted: phi = 2 pi (u - W/2) / W, theta = pi (H/2 - v) / H */
        double phi = 2.0 * M_PI * (uc - W / 2.0) / W;
        double theta = M_PI * (H / 2.0 - vc) / H;
        /* Eq. 3 */
        dc[0] = cos(theta) * sin(phi);
        dc[1] = -sin(theta);
        dc[2] = cos(theta) * cos(phi);
    } else {
        double f = (W / 2.0) / tan(fov / 2.0);
        dc[0] = (uc - W / 2.0) / f;
        dc[1] = (vc - H / 2.0) / f;
        dc[2] = 1.0;
        double n = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
        dc[0] /= n; dc[1] /= n; dc[2] /= n;
    }
    for (int i = 0; i < 3; ++i) {
        d[i] = R[3 * i + 0] * dc[0] + R[3 * i + 1] * dc[1] + R[3 * i + 2] * dc[2];
        o[i] = cam[13 + i];
    }
}

/* ------------------------------------------------------------------ */
/* occupancy and labels                                                 */
/* ------------------------------------------------------------------ */

static int bit_at(const uint32_t *bits, int gx, int gy, int x, int y, int z)
{
    int64_t words_per_row = gx / 32;
    uint32_t w = bits[((int64_t)z * gy + y) * words_per_row + x / 32];
    return (int)((w >> (x % 32)) & 1u);
}

/* label[v] = field of voxel v (linear index (z*gy + y)*gx + x), -1 if empty.
 * The rank of an occupied voxel is the number of occupied voxels before it in
 * linear order.  Returns the number of occupied voxels, or -1 if it differs
 * from n_occ. */
int64_t orc_label_map(int gx, int gy, int gz, const uint32_t *bits,
                      const uint16_t *field_of_rank, int64_t n_occ, int32_t *label)
{
    int64_t rank = 0;
    for (int z = 0; z < gz; ++z)
        for (int y = 0; y < gy; ++y)
            for (int x = 0; x < gx; ++x) {
                int64_t v = ((int64_t)z * gy + y) * gx + x;
                if (bit_at(bits, gx, gy, x, y, z)) {
                    if (rank >= n_occ) return -1;
                    label[v] = field_of_rank[rank];
                    ++rank;
                } else {
                    label[v] = -1;
                }
            }
    return rank == n_occ ? rank : -1;
}

/* ------------------------------------------------------------------ */
/* sampling of occupied voxels                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    int dims[3];
    double origin[3];
    double vox;
    const int32_t *label;     /* dense map from orc_label_map */
} orc_grid;

static int32_t state_at(const orc_grid *g, const int64_t i[3])
{
    for (int a = 0; a < 3; ++a)
        if (i[a] < 0 || i[a] >= g->dims[a]) return -1;
    return g->label[(i[2] * g->dims[1] + i[1]) * g->dims[0] + i[0]];
}

/* exit distance of the ray from the grid box (slab method); -1 if missed */
static double grid_exit(const orc_grid *g, const double *o, const double *d)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = g->origin[a], hi = g->origin[a] + g->dims[a] * g->vox;
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] >= hi) return -1.0;
            continue;
        }
        double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t1 < t0 || t1 < 0.0) return -1.0;
    return t1;
}

/* Keeps sample j (t_j = (j + 1/2) delta) iff the voxel floor((p - origin)/vox)
 * of p = o + t_j d is inside the grid and occupied; first n_max kept samples.
 * Writes js[k], fields[k]; returns the count.  *ties counts tested samples
 * (up to the last one that could matter) lying within ORC_TIE_EPS voxels of
 * a face whose two sides differ in occupancy or field. */
static int march_ray(const orc_grid *g, const double *o, const double *d, double delta,
                     int n_max, int32_t *js, int32_t *fields, int *ties)
{
    int n = 0, nt = 0;
    double t_out = grid_exit(g, o, d);
    if (t_out >= 0.0) {
        for (int64_t j = 0; n < n_max; ++j) {
            double t = ((double)j + 0.5) * delta;
            if (t > t_out + delta) break;
            double gc[3];
            int64_t iv[3];
            for (int a = 0; a < 3; ++a) {
                gc[a] = (o[a] + t * d[a] - g->origin[a]) / g->vox;
                iv[a] = (int64_t)floor(gc[a]);
            }
            int32_t s = state_at(g, iv);
            for (int a = 0; a < 3; ++a) {
                double fr = gc[a] - (double)iv[a];
                int step = fr < ORC_TIE_EPS ? -1 : (fr > 1.0 - ORC_TIE_EPS ? 1 : 0);
                if (step) {
                    int64_t nb[3] = {iv[0], iv[1], iv[2]};
                    nb[a] += step;
                    if (state_at(g, nb) != s) ++nt;
                }
            }
            if (s >= 0) {
                if (js) js[n] = (int32_t)j;
                if (fields) fields[n] = s;
                ++n;
            }
        }
    }
    if (ties) *ties = nt;
    return n;
}

int orc_march(const int32_t *dims, const double *origin, double vox, const int32_t *label,
              const double *o, const double *d, double delta, int n_max,
              int32_t *js, int32_t *fields, int32_t *ties)
{
    orc_grid g = {{dims[0], dims[1], dims[2]}, {origin[0], origin[1], origin[2]}, vox, label};
    int nt = 0;
    int n = march_ray(&g, o, d, delta, n_max, js, fields, &nt);
    if (ties) *ties = nt;
    return n;
}

/* ------------------------------------------------------------------ */
/* positional encoding and the tiny MLP                                 */
/* ------------------------------------------------------------------ */

/* F(x) for a 3-vector: [x, sin(2^k pi x), cos(2^k pi x)], k = 0..L-1 */
static void encode(const double *x, int L, double *out)
{
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2];
    for (int k = 0; k < L; ++k) {
        double f = ldexp(M_PI, k);
        for (int a = 0; a < 3; ++a) {
            out[3 + 6 * k + a] = sin(f * x[a]);
            out[3 + 6 * k + 3 + a] = cos(f * x[a]);
        }
    }
}

typedef struct {
    int W, H, act;
    double sigma_scale;
    int quant;                  /* 1: the FP8 E4M3 reading, 2: the BF16 reading */
} orc_arch;

/* y[o] = b[o] + sum_i Wm[o][i] x[i] */
static void dense(const float *Wm, const float *b, int n_out, int n_in, const double *x, double *y)
{
    for (int r = 0; r < n_out; ++r) {
        double acc = (double)b[r];
        for (int c = 0; c < n_in; ++c) acc += (double)Wm[(int64_t)r * n_in + c] * x[c];
        y[r] = acc;
    }
}

/* Nearest value of the 8-bit E4M3 floating-point format (1 sign bit, 4
 * exponent bits with bias 7, 3 mantissa bits; normal numbers from 2^-6,
 * subnormal spacing 2^-9, largest finite value 448, no infinities), ties to
 * even; magnitudes beyond 448 saturate to 448. */
static double e4m3(double x)
{
    double a = fabs(x);
    if (a == 0.0) return x;
    int e;
    frexp(a, &e);                 /* a = m 2^e, m in [0.5, 1): leading bit 2^(e-1) */
    int lead = e - 1;
    if (lead < -6) lead = -6;     /* subnormal range keeps the spacing of 2^-6 * 2^-3 */
    double q = ldexp(1.0, lead - 3);
    double r = nearbyint(a / q) * q;   /* default rounding mode: to nearest, ties to even */
    if (r > 448.0) r = 448.0;
    return copysign(r, x);
}

double orc_e4m3(double x) { return e4m3(x); }

/* dense() in the FP8 reading: inputs and per-row-scaled weights rounded to E4M3 */
static void dense_e4m3(const float *Wm, const float *b, int n_out, int n_in, const double *x, double *y)
{
    double xq[512];
    for (int c = 0; c < n_in; ++c) xq[c] = e4m3((double)(float)x[c]);
    for (int r = 0; r < n_out; ++r) {
        const float *row = Wm + (int64_t)r * n_in;
        float amax = 0.0f;
        for (int c = 0; c < n_in; ++c) amax = fmaxf(amax, fabsf(row[c]));
        const float s = amax > 0.0f ? amax / 448.0f : 1.0f;
        double acc = 0.0;
        for (int c = 0; c < n_in; ++c) acc += e4m3((double)(row[c] / s)) * xq[c];
        y[r] = (double)b[r] + (double)s * acc;
    }
}

/* Nearest BF16 value (8 significant bits: a = m 2^e with m in [0.5, 1) is
 * rounded to a multiple of 2^(e-8)), ties to even; the magnitudes here stay
 * far inside the format's normal range. */
static double bf16r(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(fabs(x), &e);
    const double q = ldexp(1.0, e - 8);
    return copysign(nearbyint(fabs(x) / q) * q, x);
}

double orc_bf16(double x) { return bf16r(x); }

/* dense() in the BF16 reading: inputs, weights and bias rounded to BF16 */
static void dense_bf16(const float *Wm, const float *b, int n_out, int n_in, const double *x, double *y)
{
    double xq[512];
    for (int c = 0; c < n_in; ++c) xq[c] = bf16r(x[c]);
    for (int r = 0; r < n_out; ++r) {
        double acc = bf16r((double)b[r]);
        for (int c = 0; c < n_in; ++c) acc += bf16r((double)Wm[(int64_t)r * n_in + c]) * xq[c];
        y[r] = acc;
    }
}

static double softplus(double s) { return s > 30.0 ? s : log1p(exp(s)); }
static double sigm(double s) { return 1.0 / (1.0 + exp(-s)); }

/* cache of one forward evaluation, for the backward pass */
typedef struct {
    double pe_x[ORC_PE_POS];
    double in_c[256 + ORC_PE_DIR];  /* [feat; F(d)] */
    double z[8][256];               /* pre-activations of layer 1..H */
    double zh[257];                 /* head output [s; feat] */
    double zc[256];                 /* colour layer pre-activation */
    double zo[3];
    double sigma, rgb[3];
} orc_cache;

/* Evaluates the field's MLP at world point p (field-local x = scale*p +
 * offset) and world direction d.  out = (sigma, r, g, b). */
static void mlp_forward(const float *w, const orc_arch *A, const double *aff, const double *p,
                        const double *d, orc_cache *c)
{
    int W = A->W, H = A->H;
    double xl[3];
    for (int a = 0; a < 3; ++a) xl[a] = aff[a] * p[a] + aff[3 + a];
    encode(xl, 10, c->pe_x);
    const float *q = w;
    double h[256];
    void (*mat)(const float *, const float *, int, int, const double *, double *) =
        A->quant == 1 ? dense_e4m3 : (A->quant == 2 ? dense_bf16 : dense);
    mat(q, q + W * ORC_PE_POS, W, ORC_PE_POS, c->pe_x, c->z[0]);
    q += W * ORC_PE_POS + W;
    for (int r = 0; r < W; ++r) h[r] = c->z[0][r] > 0.0 ? c->z[0][r] : 0.0;
    for (int k = 1; k < H; ++k) {
        mat(q, q + W * W, W, W, h, c->z[k]);
        q += W * W + W;
        for (int r = 0; r < W; ++r) h[r] = c->z[k][r] > 0.0 ? c->z[k][r] : 0.0;
    }
    mat(q, q + (1 + W) * W, 1 + W, W, h, c->zh);
    q += (1 + W) * W + (1 + W);
    double s = c->zh[0];
    c->sigma = A->sigma_scale * (A->act == 1 ? (s > 0.0 ? s : 0.0) : softplus(s));
    for (int r = 0; r < W; ++r) c->in_c[r] = c->zh[1 + r];
    encode(d, 4, c->in_c + W);
    mat(q, q + W * (W + ORC_PE_DIR), W, W + ORC_PE_DIR, c->in_c, c->zc);
    q += W * (W + ORC_PE_DIR) + W;
    double g[256];
    for (int r = 0; r < W; ++r) g[r] = c->zc[r] > 0.0 ? c->zc[r] : 0.0;
    dense(q, q + 3 * W, 3, W, g, c->zo);
    for (int r = 0; r < 3; ++r) c->rgb[r] = sigm(c->zo[r]);
}

/* Public single-sample evaluation.  w: FP32 weights of one field in storage
 * order; aff = (scale[3], offset[3]); out = (sigma, r, g, b). */
void orc_mlp(const float *w, int W, int H, int act, double sigma_scale, int quant, const double *aff,
             const double *p, const double *d, double *out)
{
    orc_arch A = {W, H, act, sigma_scale, quant};
    orc_cache c;
    mlp_forward(w, &A, aff, p, d, &c);
    out[0] = c.sigma;
    out[1] = c.rgb[0]; out[2] = c.rgb[1]; out[3] = c.rgb[2];
}

/* positional encoding alone, for pins */
void orc_encode(const double *x, int L, double *out) { encode(x, L, out); }

/* Reverse mode through the MLP for one sample: adds d(loss)/d(weights) into
 * gw given d(loss)/d(sigma) and d(loss)/d(rgb). */
static void mlp_backward(const float *w, const orc_arch *A, const orc_cache *c, double dsigma,
                         const double *drgb, double *gw)
{
    int W = A->W, H = A->H;
    /* the BF16 reading rounds operands (see the header); otherwise identity */
    const int rb = A->quant == 2;
#define RQ(x) (rb ? bf16r(x) : (x))
    /* offsets of each layer in the flat parameter vector */
    int64_t off[16];
    int64_t o = 0;
    off[0] = o; o += (int64_t)W * ORC_PE_POS + W;
    for (int k = 1; k < H; ++k) { off[k] = o; o += (int64_t)W * W + W; }
    int64_t off_h = o; o += (int64_t)(1 + W) * W + (1 + W);
    int64_t off_c = o; o += (int64_t)W * (W + ORC_PE_DIR) + W;
    int64_t off_o = o;

    double h[8][256];               /* post-activation of layers 1..H (as the next layer reads them) */
    for (int k = 0; k < H; ++k)
        for (int r = 0; r < W; ++r) h[k][r] = RQ(c->z[k][r] > 0.0 ? c->z[k][r] : 0.0);
    double g[256];
    for (int r = 0; r < W; ++r) g[r] = c->zc[r] > 0.0 ? c->zc[r] : 0.0;

    /* output layer: rgb = sigmoid(zo) */
    double dzo[3];
    for (int r = 0; r < 3; ++r) dzo[r] = drgb[r] * c->rgb[r] * (1.0 - c->rgb[r]);
    const float *Wo = w + off_o;
    double dg[256];
    for (int i = 0; i < W; ++i) dg[i] = 0.0;
    for (int r = 0; r < 3; ++r) {
        for (int i = 0; i < W; ++i) {
            gw[off_o + (int64_t)r * W + i] += RQ(dzo[r]) * RQ(g[i]);
            dg[i] += (double)Wo[r * W + i] * dzo[r];
        }
        gw[off_o + 3 * W + r] += RQ(dzo[r]);
    }
    /* colour layer: g = relu(zc), zc = Wc [feat; F(d)] + bc */
    int Kc = W + ORC_PE_DIR;
    const float *Wc = w + off_c;
    double dfeat[256];
    for (int i = 0; i < W; ++i) dfeat[i] = 0.0;
    for (int r = 0; r < W; ++r) {
        double dz = RQ(c->zc[r] > 0.0 ? dg[r] : 0.0);
        if (dz == 0.0) continue;
        for (int i = 0; i < Kc; ++i) gw[off_c + (int64_t)r * Kc + i] += dz * RQ(c->in_c[i]);
        for (int i = 0; i < W; ++i) dfeat[i] += RQ((double)Wc[(int64_t)r * Kc + i]) * dz;
        gw[off_c + (int64_t)W * Kc + r] += dz;
    }
    /* head: [s; feat] = Wh h_H + bh; sigma = scale * softplus(s) */
    double s = c->zh[0];
    double dz_h[257];
    dz_h[0] = RQ(dsigma * A->sigma_scale * (A->act == 1 ? (s > 0.0 ? 1.0 : 0.0) : sigm(s)));
    for (int i = 0; i < W; ++i) dz_h[1 + i] = RQ(dfeat[i]);
    const float *Wh = w + off_h;
    double dh[256];
    for (int i = 0; i < W; ++i) dh[i] = 0.0;
    for (int r = 0; r < 1 + W; ++r) {
        double dz = dz_h[r];
        if (dz == 0.0) continue;
        for (int i = 0; i < W; ++i) {
            gw[off_h + (int64_t)r * W + i] += dz * h[H - 1][i];
            dh[i] += RQ((double)Wh[(int64_t)r * W + i]) * dz;
        }
        gw[off_h + (int64_t)(1 + W) * W + r] += dz;
    }
    /* hidden layers H..2 */
    for (int k = H - 1; k >= 1; --k) {
        const float *Wk = w + off[k];
        double dprev[256];
        for (int i = 0; i < W; ++i) dprev[i] = 0.0;
        for (int r = 0; r < W; ++r) {
            double dz = RQ(c->z[k][r] > 0.0 ? dh[r] : 0.0);
            if (dz == 0.0) continue;
            for (int i = 0; i < W; ++i) {
                gw[off[k] + (int64_t)r * W + i] += dz * h[k - 1][i];
                dprev[i] += RQ((double)Wk[(int64_t)r * W + i]) * dz;
            }
            gw[off[k] + (int64_t)W * W + r] += dz;
        }
        for (int i = 0; i < W; ++i) dh[i] = dprev[i];
    }
    /* layer 1 */
    for (int r = 0; r < W; ++r) {
        double dz = RQ(c->z[0][r] > 0.0 ? dh[r] : 0.0);
        if (dz == 0.0) continue;
        for (int i = 0; i < ORC_PE_POS; ++i) gw[off[0] + (int64_t)r * ORC_PE_POS + i] += dz * RQ(c->pe_x[i]);
        gw[off[0] + (int64_t)W * ORC_PE_POS + r] += dz;
    }
#undef RQ
}

/* ------------------------------------------------------------------ */
/* volume rendering with early termination: Eq. 4 and Eq. 5             */
/* ------------------------------------------------------------------ */

/* For samples i = 0..n-1 with densities sigma[i], colours rgb[3i..], depths
 * t[i], every interval delta:
 *   T_i = exp(-sum_{k<i} sigma_k delta),  w_i = T_i (1 - exp(-sigma_i delta)),
 * stopping after the first i with T_{i+1} < t_stop.
 * out = (C_r, C_g, C_b, D, opacity) with C = sum w_i c_i + T_end bg,
 * D = sum w_i t_i, opacity = sum w_i.  Returns the number of samples used;
 * *margin = min over used i of |ln(T_{i+1} / t_stop)|. */
static int composite(int n, const double *sigma, const double *rgb, const double *t, double delta,
                     double t_stop, const double *bg, double *out, double *margin, double *w_out,
                     double *T_end_out)
{
    double C[3] = {0, 0, 0}, D = 0.0, acc = 0.0, tau = 0.0, mg = INFINITY;
    int used = 0;
    for (int i = 0; i < n; ++i) {
        double Ti = exp(-tau);
        double wi = Ti * (1.0 - exp(-sigma[i] * delta));
        if (w_out) w_out[i] = wi;
        for (int c = 0; c < 3; ++c) C[c] += wi * rgb[3 * i + c];
        D += wi * t[i];
        acc += wi;
        tau += sigma[i] * delta;
        used = i + 1;
        double Tn = exp(-tau);
        double m = fabs(log(Tn / t_stop));
        if (m < mg) mg = m;
        if (Tn < t_stop) break;
    }
    double Te = exp(-tau);
    for (int c = 0; c < 3; ++c) out[c] = C[c] + Te * bg[c];
    out[3] = D;
    out[4] = acc;
    if (margin) *margin = mg;
    if (T_end_out) *T_end_out = Te;
    return used;
}

int orc_composite(int n, const double *sigma, const double *rgb, const double *t, double delta,
                  double t_stop, const double *bg, double *out, double *margin)
{
    return composite(n, sigma, rgb, t, delta, t_stop, bg, out, margin, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* whole rays                                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    orc_grid g;
    orc_arch A;
    int64_t P;
    const float *weights;   /* [F][P], or field after field at woff[f] when widths vary */
    const int32_t *widths;  /* NULL: every field has width A.W */
    int64_t *woff;          /* start of field f's weights (widths != NULL) */
    const float *affine;    /* [F][6] */
    const double *cams;     /* [n_views][16] */
    int n_views;
    double delta, t_stop, bg[3];
    int n_max;
} orc_scene;

static void ray_of(const orc_scene *S, const uint32_t *rays, int64_t r, const int64_t *starts,
                   double *o, double *d)
{
    int64_t view, pix;
    if (rays) {
        view = rays[2 * r];
        pix = rays[2 * r + 1];
    } else {
        view = 0;
        while (view + 1 < S->n_views && r >= starts[view + 1]) ++view;
        pix = r - starts[view];
    }
    const double *cam = S->cams + 16 * view;
    int64_t width = (int64_t)cam[1];
    double u = (double)(pix % width), v = (double)(pix / width);
    orc_ray(cam, u + 0.5, v + 0.5, o, d);
}

/* The MLP at every given kept sample (j_k, field_k) of the ray o + t d,
 * t_k = (j_k + 1/2) delta, then Eq. 4-5 over them in ray order; fills
 * per-sample caches if given (sized n).  Returns the number composited. */
static int shade_ray(const orc_scene *S, const double *o, const double *d, int n, const int32_t *js,
                     const int32_t *fields, double *out, double *margin, orc_cache *caches, double *w_buf,
                     double *T_end)
{
    double sig[1024], rgb[3 * 1024], tt[1024];
    orc_cache local;
    for (int k = 0; k < n; ++k) {
        double t = ((double)js[k] + 0.5) * S->delta;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        int f = fields[k];
        orc_cache *c = caches ? &caches[k] : &local;
        orc_arch A = S->A;
        if (S->widths) A.W = S->widths[f];
        mlp_forward(S->weights + (S->widths ? S->woff[f] : (int64_t)f * S->P), &A, (const double[6]){
                        S->affine[6 * f + 0], S->affine[6 * f + 1], S->affine[6 * f + 2],
                        S->affine[6 * f + 3], S->affine[6 * f + 4], S->affine[6 * f + 5]},
                    p, d, c);
        sig[k] = c->sigma;
        rgb[3 * k + 0] = c->rgb[0]; rgb[3 * k + 1] = c->rgb[1]; rgb[3 * k + 2] = c->rgb[2];
        tt[k] = t;
    }
    return composite(n, sig, rgb, tt, S->delta, S->t_stop, S->bg, out, margin, w_buf, T_end);
}

/* per-ray forward: the march, then shade_ray over its kept samples */
static int render_ray(const orc_scene *S, const double *o, const double *d, double *out,
                      int *n_kept, int *ties, double *margin, int32_t *js, int32_t *fields,
                      orc_cache *caches, double *w_buf, double *T_end)
{
    int nt = 0;
    int n = march_ray(&S->g, o, d, S->delta, S->n_max, js, fields, &nt);
    int used = shade_ray(S, o, d, n, js, fields, out, margin, caches, w_buf, T_end);
    if (n_kept) *n_kept = n;
    if (ties) *ties = nt;
    return used;
}

static int setup_scene(orc_scene *S, const int32_t *dims, const double *origin, double vox,
                       const int32_t *label, const float *weights, const float *affine, int W, int H,
                       int act, double sigma_scale, int quant, const double *cams, int n_views,
                       double delta, int n_max, double t_stop, const double *bg)
{
    if (n_max > 1024 || W > 256 || H > 8 || H < 1) return -1;
    S->g = (orc_grid){{dims[0], dims[1], dims[2]}, {origin[0], origin[1], origin[2]}, vox, label};
    S->A = (orc_arch){W, H, act, sigma_scale, quant};
    S->P = orc_param_count(W, H);
    S->weights = weights;
    S->widths = NULL;
    S->woff = NULL;
    S->affine = affine;
    S->cams = cams;
    S->n_views = n_views;
    S->delta = delta;
    S->t_stop = t_stop;
    S->bg[0] = bg[0]; S->bg[1] = bg[1]; S->bg[2] = bg[2];
    S->n_max = n_max;
    return 0;
}

/* Per-field weight offsets when every field has its own width (widths !=
 * NULL: field f's parameters follow field f-1's).  0, or -1 on a bad width
 * or a failed allocation. */
static int scene_widths(orc_scene *S, const int32_t *widths, int n_fields, int64_t **woff_out)
{
    *woff_out = NULL;
    if (!widths) return 0;
    int64_t *woff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_fields > 0 ? n_fields : 1));
    if (!woff) return -1;
    int64_t o = 0;
    for (int f = 0; f < n_fields; ++f) {
        if (widths[f] < 1 || widths[f] > 256) { free(woff); return -1; }
        woff[f] = o;
        o += orc_param_count(widths[f], S->A.H);
    }
    S->widths = widths;
    S->woff = woff;
    *woff_out = woff;
    return 0;
}

static int view_starts(const double *cams, int n_views, int64_t *starts)
{
    if (n_views > 256) return -1;
    starts[0] = 0;
    for (int v = 0; v < n_views; ++v) starts[v + 1] = starts[v] + (int64_t)cams[16 * v + 1] * (int64_t)cams[16 * v + 2];
    return 0;
}

/* Renders rays (view, pixel) pairs, or every pixel of every view in order
 * when rays == NULL.  Per ray: rgb[3], depth, opacity, number of kept
 * samples, number composited before termination, near-tie count of the
 * march, termination margin.  widths (NULL: every field has width W) gives
 * each of the n_fields fields its own width, the weights then lying field
 * after field.  Returns 0, or -1 on bad sizes. */
int orc_render(const int32_t *dims, const double *origin, double vox, const int32_t *label,
               const float *weights, const float *affine, int W, int H, int act, double sigma_scale,
               int quant, const int32_t *widths, int n_fields, const double *cams, int n_views,
               const uint32_t *rays, int64_t n_rays, double delta, int n_max, double t_stop,
               const double *bg, double *rgb, double *depth, double *opacity, int32_t *n_kept,
               int32_t *n_used, int32_t *ties, double *margin)
{
    orc_scene S;
    int64_t *woff = NULL, starts[257];
    if (setup_scene(&S, dims, origin, vox, label, weights, affine, W, H, act, sigma_scale, quant, cams,
                    n_views, delta, n_max, t_stop, bg) ||
        view_starts(cams, n_views, starts) || scene_widths(&S, widths, n_fields, &woff))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3], d[3], out[5], mg = INFINITY;
        int32_t js[1024], fs[1024];
        int nk = 0, nt = 0;
        ray_of(&S, rays, r, starts, o, d);
        int used = render_ray(&S, o, d, out, &nk, &nt, &mg, js, fs, NULL, NULL, NULL);
        rgb[3 * r + 0] = out[0]; rgb[3 * r + 1] = out[1]; rgb[3 * r + 2] = out[2];
        if (depth) depth[r] = out[3];
        if (opacity) opacity[r] = out[4];
        if (n_kept) n_kept[r] = nk;
        if (n_used) n_used[r] = used;
        if (ties) ties[r] = nt;
        if (margin) margin[r] = mg;
    }
    free(woff);
    return 0;
}

/* Eq. 4-5 over a GIVEN set of kept samples per ray instead of the oracle's
 * own march: ray r composites samples (rec_j[r][k], rec_field[r][k]) for
 * k < rec_count[r] (rows rec_stride apart), each through its field's MLP at
 * t = (j + 1/2) delta, with early termination as orc_render.  This is the
 * plain composite of another march's sample records (a renderer's, say),
 * so that its colours can be checked on its own sample set where its march
 * legitimately differs from the oracle's at near-ties.  Outputs as
 * orc_render (no kept count or tie count).  Returns 0, or -1 on bad sizes,
 * a negative sample index or a field id outside [0, n_fields). */
int orc_render_records(const int32_t *dims, const double *origin, double vox, const int32_t *label,
                       const float *weights, const float *affine, int W, int H, int act, double sigma_scale,
                       int quant, const int32_t *widths, int n_fields, const double *cams, int n_views,
                       const uint32_t *rays, int64_t n_rays, double delta, double t_stop, const double *bg,
                       const int32_t *rec_count, const int32_t *rec_j, const int32_t *rec_field, int rec_stride,
                       double *rgb, double *depth, double *opacity, int32_t *n_used, double *margin)
{
    orc_scene S;
    int64_t *woff = NULL, starts[257];
    if (rec_stride < 1 || rec_stride > 1024) return -1;
    for (int64_t r = 0; r < n_rays; ++r) {
        if (rec_count[r] < 0 || rec_count[r] > rec_stride) return -1;
        for (int k = 0; k < rec_count[r]; ++k)
            if (rec_j[r * rec_stride + k] < 0 || rec_field[r * rec_stride + k] < 0 ||
                rec_field[r * rec_stride + k] >= n_fields)
                return -1;
    }
    if (setup_scene(&S, dims, origin, vox, label, weights, affine, W, H, act, sigma_scale, quant, cams,
                    n_views, delta, rec_stride, t_stop, bg) ||
        view_starts(cams, n_views, starts) || scene_widths(&S, widths, n_fields, &woff))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3], d[3], out[5], mg = INFINITY;
        ray_of(&S, rays, r, starts, o, d);
        int used = shade_ray(&S, o, d, rec_count[r], rec_j + r * rec_stride, rec_field + r * rec_stride, out, &mg,
                             NULL, NULL, NULL);
        rgb[3 * r + 0] = out[0]; rgb[3 * r + 1] = out[1]; rgb[3 * r + 2] = out[2];
        if (depth) depth[r] = out[3];
        if (opacity) opacity[r] = out[4];
        if (n_used) n_used[r] = used;
        if (margin) margin[r] = mg;
    }
    free(woff);
    return 0;
}

/* Near-tie certificate of single samples: for query q, sample q_j[q] of ray
 * q_ray[q] (an index into rays, or a global pixel index when rays == NULL),
 * the distance in voxel units from its point o + (j + 1/2) delta d to the
 * nearest face of its voxel whose two sides differ in state (empty, outside
 * the grid, or another field); INFINITY when no face of the voxel does.  A
 * sample nearer such a face than the rounding error of another
 * implementation's coordinates may legitimately land on either side.
 * Returns 0, or -1 on bad sizes. */
int orc_sample_tie_distance(const int32_t *dims, const double *origin, double vox, const int32_t *label,
                            const double *cams, int n_views, const uint32_t *rays, int64_t n_queries,
                            const int64_t *q_ray, const int32_t *q_j, double delta, double *dist)
{
    orc_scene S;
    static const float dummy_w[1] = {0};
    static const double zero_bg[3] = {0, 0, 0};
    int64_t starts[257];
    if (setup_scene(&S, dims, origin, vox, label, dummy_w, dummy_w, 1, 1, 0, 1.0, 0, cams, n_views,
                    delta, 1, 1e-4, zero_bg) ||
        view_starts(cams, n_views, starts))
        return -1;
    for (int64_t q = 0; q < n_queries; ++q) {
        double o[3], d[3], gc[3];
        int64_t iv[3];
        ray_of(&S, rays, q_ray[q], starts, o, d);
        double t = ((double)q_j[q] + 0.5) * delta;
        for (int a = 0; a < 3; ++a) {
            gc[a] = (o[a] + t * d[a] - S.g.origin[a]) / S.g.vox;
            iv[a] = (int64_t)floor(gc[a]);
        }
        int32_t s = state_at(&S.g, iv);
        double best = INFINITY;
        for (int a = 0; a < 3; ++a)
            for (int step = -1; step <= 1; step += 2) {
                int64_t nb[3] = {iv[0], iv[1], iv[2]};
                nb[a] += step;
                if (state_at(&S.g, nb) == s) continue;
                double fr = gc[a] - (double)iv[a];
                double dd = step < 0 ? fr : 1.0 - fr;
                if (dd < best) best = dd;
            }
        dist[q] = best;
    }
    return 0;
}

/* Marches rays only (no MLP): per ray the kept sample indices and fields,
 * row r of js/fields holding up to n_max entries. */
int orc_march_rays(const int32_t *dims, const double *origin, double vox, const int32_t *label,
                   const double *cams, int n_views, const uint32_t *rays, int64_t n_rays,
                   double delta, int n_max, int32_t *count, int32_t *js, int32_t *fields,
                   int32_t *ties)
{
    orc_scene S;
    static const float dummy_w[1] = {0};
    static const double zero_bg[3] = {0, 0, 0};
    if (setup_scene(&S, dims, origin, vox, label, dummy_w, dummy_w, 1, 1, 0, 1.0, 0, cams, n_views,
                    delta, n_max, 1e-4, zero_bg))
        return -1;
    int64_t starts[257];
    if (n_views > 256) return -1;
    starts[0] = 0;
    for (int v = 0; v < n_views; ++v) starts[v + 1] = starts[v] + (int64_t)cams[16 * v + 1] * (int64_t)cams[16 * v + 2];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3], d[3];
        int nt = 0;
        ray_of(&S, rays, r, starts, o, d);
        count[r] = march_ray(&S.g, o, d, delta, n_max, js + r * n_max, fields + r * n_max, &nt);
        if (ties) ties[r] = nt;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* fine-tuning loss and its gradient                                    */
/* ------------------------------------------------------------------ */

static uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

/* Sum over rays of sum_c (C_c - target_c)^2 divided by loss_norm (3 * n for
 * the mean over a batch of n rays).  When grad != NULL it receives, in
 * the [F][P] storage order, d(loss)/d(weights) (overwritten).  *signature
 * hashes every ReLU sign and termination index, so that a finite-difference
 * step can be checked not to cross a kink.  Returns the loss, NAN on error. */
double orc_loss_grad(const int32_t *dims, const double *origin, double vox, const int32_t *label,
                     const float *weights, const float *affine, int n_fields, int W, int H, int act,
                     double sigma_scale, const double *cams, int n_views, const uint32_t *rays,
                     int64_t n_rays, double delta, int n_max, double t_stop, const double *bg,
                     const float *target, double loss_norm, double *grad, uint64_t *signature,
                     double *rgb_out)
{
    orc_scene S;
    if (setup_scene(&S, dims, origin, vox, label, weights, affine, W, H, act, sigma_scale, 0, cams,
                    n_views, delta, n_max, t_stop, bg))
        return NAN;
    int64_t starts[257];
    if (n_views > 256) return NAN;
    starts[0] = 0;
    for (int v = 0; v < n_views; ++v) starts[v + 1] = starts[v] + (int64_t)cams[16 * v + 1] * (int64_t)cams[16 * v + 2];

    /* phase 1, per ray: forward, loss, d(loss)/d(sigma_i) and d(loss)/d(c_i) */
    int32_t *cnt = (int32_t *)calloc((size_t)n_rays, sizeof(int32_t));
    int32_t *s_j = (int32_t *)malloc((size_t)n_rays * n_max * sizeof(int32_t));
    int32_t *s_f = (int32_t *)malloc((size_t)n_rays * n_max * sizeof(int32_t));
    double *s_g = (double *)malloc((size_t)n_rays * n_max * 4 * sizeof(double));
    uint64_t *rh = (uint64_t *)calloc((size_t)n_rays, sizeof(uint64_t));
    double loss = 0.0;
    int fail = !(cnt && s_j && s_f && s_g && rh);
    if (!fail) {
#pragma omp parallel reduction(+ : loss)
        {
            orc_cache *caches = (orc_cache *)malloc((size_t)n_max * sizeof(orc_cache));
            double *wb = (double *)malloc((size_t)n_max * sizeof(double));
            double *Tn = (double *)malloc((size_t)n_max * sizeof(double));
#pragma omp for schedule(dynamic, 16)
            for (int64_t r = 0; r < n_rays; ++r) {
                double o[3], d[3], out[5], mg, Te;
                int nk, nt;
                int32_t *js = s_j + r * n_max, *fs = s_f + r * n_max;
                ray_of(&S, rays, r, starts, o, d);
                int used = render_ray(&S, o, d, out, &nk, &nt, &mg, js, fs, caches, wb, &Te);
                double dC[3];
                for (int c = 0; c < 3; ++c) {
                    double e = out[c] - (double)target[3 * r + c];
                    loss += e * e / loss_norm;
                    dC[c] = 2.0 * e / loss_norm;
                    if (rgb_out) rgb_out[3 * r + c] = out[c];
                }
                /* T_{i+1} = exp(-sum_{k<=i} sigma_k delta) */
                double tau = 0.0;
                for (int i = 0; i < used; ++i) {
                    tau += caches[i].sigma * S.delta;
                    Tn[i] = exp(-tau);
                }
                /* dC/dc_i = w_i;
                 * dC/dsigma_i = delta (T_{i+1} c_i - sum_{i<j<=I} w_j c_j - T_end bg) */
                double suffix[3] = {0, 0, 0};
                uint64_t h = mix64(0, (uint64_t)used);
                for (int i = used - 1; i >= 0; --i) {
                    const orc_cache *c = &caches[i];
                    double ds = 0.0;
                    for (int ch = 0; ch < 3; ++ch)
                        ds += S.delta * (Tn[i] * c->rgb[ch] - suffix[ch] - Te * S.bg[ch]) * dC[ch];
                    double *gg = s_g + (r * n_max + i) * 4;
                    gg[0] = ds;
                    for (int ch = 0; ch < 3; ++ch) gg[1 + ch] = wb[i] * dC[ch];
                    for (int ch = 0; ch < 3; ++ch) suffix[ch] += wb[i] * c->rgb[ch];
                    for (int k = 0; k < H; ++k)
                        for (int q = 0; q < W; ++q) h = mix64(h, c->z[k][q] > 0.0);
                    for (int q = 0; q < W; ++q) h = mix64(h, c->zc[q] > 0.0);
                }
                cnt[r] = used;
                rh[r] = mix64(h, (uint64_t)r);
            }
            free(caches);
            free(wb);
            free(Tn);
        }
    }
    uint64_t sig = 0;
    for (int64_t r = 0; r < n_rays && !fail; ++r) sig ^= rh[r] * 0x100000001b3ULL + (uint64_t)r;
    if (signature) *signature = sig;

    /* phase 2, per field: backpropagate every used sample of the field */
    if (grad && !fail) {
        int64_t P = S.P;
        memset(grad, 0, (size_t)n_fields * P * sizeof(double));
        int64_t total = 0;
        for (int64_t r = 0; r < n_rays; ++r) total += cnt[r];
        int64_t *fcount = (int64_t *)calloc((size_t)n_fields + 1, sizeof(int64_t));
        int64_t *order = (int64_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int64_t));
        if (!fcount || !order) {
            fail = 1;
        } else {
            for (int64_t r = 0; r < n_rays; ++r)
                for (int i = 0; i < cnt[r]; ++i) fcount[s_f[r * n_max + i] + 1]++;
            for (int f = 0; f < n_fields; ++f) fcount[f + 1] += fcount[f];
            int64_t *cur = (int64_t *)malloc((size_t)n_fields * sizeof(int64_t));
            for (int f = 0; f < n_fields; ++f) cur[f] = fcount[f];
            for (int64_t r = 0; r < n_rays; ++r)
                for (int i = 0; i < cnt[r]; ++i) order[cur[s_f[r * n_max + i]]++] = r * n_max + i;
            free(cur);
#pragma omp parallel for schedule(dynamic, 1)
            for (int f = 0; f < n_fields; ++f) {
                orc_cache c;
                const float *wf = S.weights + (int64_t)f * P;
                const double aff[6] = {affine[6 * f + 0], affine[6 * f + 1], affine[6 * f + 2],
                                       affine[6 * f + 3], affine[6 * f + 4], affine[6 * f + 5]};
                for (int64_t q = fcount[f]; q < fcount[f + 1]; ++q) {
                    int64_t idx = order[q];
                    int64_t r = idx / n_max;
                    double o[3], d[3];
                    ray_of(&S, rays, r, starts, o, d);
                    double t = ((double)s_j[idx] + 0.5) * S.delta;
                    double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                    mlp_forward(wf, &S.A, aff, p, d, &c);
                    const double *gg = s_g + idx * 4;
                    mlp_backward(wf, &S.A, &c, gg[0], gg + 1, grad + (int64_t)f * P);
                }
            }
        }
        free(fcount);
        free(order);
    }
    free(cnt); free(s_j); free(s_f); free(s_g); free(rh);
    return fail ? NAN : loss;
}

/* Rays (of a list) whose kept samples include field f: only their loss
 * terms change when f's weights change. */
int orc_rays_touching(const int32_t *dims, const double *origin, double vox, const int32_t *label,
                      const double *cams, int n_views, const uint32_t *rays, int64_t n_rays,
                      double delta, int n_max, int field, uint8_t *mask)
{
    orc_grid g = {{dims[0], dims[1], dims[2]}, {origin[0], origin[1], origin[2]}, vox, label};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3], d[3];
        int32_t js[1024], fs[1024];
        const double *cam = cams + 16 * rays[2 * r];
        int64_t width = (int64_t)cam[1];
        int64_t pix = rays[2 * r + 1];
        orc_ray(cam, (double)(pix % width) + 0.5, (double)(pix / width) + 0.5, o, d);
        int n = march_ray(&g, o, d, delta, n_max, js, fs, NULL);
        uint8_t m = 0;
        for (int k = 0; k < n; ++k) m |= (fs[k] == field);
        mask[r] = m;
    }
    (void)n_views;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adam (Sec. "Training Details and Parameters": beta1 = 0.9,           */
/* beta2 = 0.99, exponentially decaying learning rate)                  */
/* ------------------------------------------------------------------ */

/* One Adam step of the (FP32-stored) weights w with gradient g, moments m
 * and v updated in place, everything computed in FP64: m <- b1 m + (1-b1) g,
 * v <- b2 v + (1-b2) g^2, w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void orc_adam(int64_t n, double *w, double *m, double *v, const double *g, double lr, double b1, double b2,
              double eps, int t)
{
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------------ */
/* Progressive probabilistic occupancy (Eq. 6, Alg. 1 stage I)          */
/* ------------------------------------------------------------------ */
/*
 * Reading of Eq. 6 taken here (the paper gives the log-odds recursion, the
 * clamp [-2, 3.5], the 0.97 threshold, and that the measurement comes from
 * a rendered depth map and an uncertainty obtained by normalising the
 * weights of Eq. 5; it builds on Octomap's ray insertion):
 *   - a pixel with opacity A = sum w_i (the normaliser of the weights) and
 *     depth D = sum w_i t_i measures its ray's end point at
 *     e = o + (D / A) d; pixels with A < a_min carry no measurement;
 *   - per scan (one camera), every voxel whose interior the segment [o, e)
 *     crosses is observed free, the voxel holding e is observed occupied,
 *     occupied wins over free, and each voxel takes at most one update per
 *     scan: L += logit(p_hit(A)) with p_hit(A) = 1/2 + (p_hit - 1/2) A (the
 *     largest A among the rays ending in it), or L += logit(p_miss);
 *   - L is clamped to [l_min, l_max] after every update; a voxel is occupied
 *     iff L > logit(p_occ).
 * The segment's voxels are found by their definition: every parameter at
 * which the segment crosses a voxel plane is listed and sorted, and the
 * voxel of each interval's midpoint is taken (intervals shorter than 1e-9
 * voxel are reported as near-ties, where an incremental traversal may
 * legitimately differ).
 */

static double logit_of(double p) { return log(p / (1.0 - p)); }

static int dcmp(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Voxels (linear indices x-fastest) crossed by the open segment between
 * parameters 0 and t_end of o + t d, inside the grid.  Returns the count
 * written to out (at most cap), or -1 on overflow; *ties counts intervals
 * shorter than 1e-9 voxel. */
static int64_t segment_voxels(const int32_t *dims, const double *origin, double vox, const double *o,
                              const double *d, double t_end, int64_t *out, int64_t cap, int *ties)
{
    /* crossing parameters of every voxel plane between the two ends */
    double len = 0.0;
    for (int a = 0; a < 3; ++a) len += d[a] * d[a];
    len = sqrt(len);
    int64_t n_t = 0, cap_t = 4;
    for (int a = 0; a < 3; ++a) cap_t += (int64_t)(fabs(d[a]) * t_end / vox) + 4;
    double *ts = (double *)malloc(sizeof(double) * (size_t)cap_t);
    if (!ts) return -1;
    ts[n_t++] = 0.0;
    ts[n_t++] = t_end;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        const double u0 = (o[a] - origin[a]) / vox, u1 = (o[a] + t_end * d[a] - origin[a]) / vox;
        const double lo = fmin(u0, u1), hi = fmax(u0, u1);
        for (double k = ceil(lo); k <= hi && n_t < cap_t; k += 1.0) {
            const double t = (origin[a] + k * vox - o[a]) / d[a];
            if (t > 0.0 && t < t_end) ts[n_t++] = t;
        }
    }
    qsort(ts, (size_t)n_t, sizeof(double), dcmp);
    int64_t n = 0;
    for (int64_t i = 0; i + 1 < n_t; ++i) {
        const double ta = ts[i], tb = ts[i + 1];
        if (tb - ta <= 0.0) continue;
        if ((tb - ta) * len < 1e-9 * vox) { if (ties) ++*ties; continue; }
        const double tm = 0.5 * (ta + tb);
        int64_t c[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            c[a] = (int64_t)floor((o[a] + tm * d[a] - origin[a]) / vox);
            if (c[a] < 0 || c[a] >= dims[a]) inside = 0;
        }
        if (!inside) continue;
        const int64_t v = (c[2] * dims[1] + c[1]) * dims[0] + c[0];
        if (n > 0 && out[n - 1] == v) continue;
        if (n >= cap) { free(ts); return -1; }
        out[n++] = v;
    }
    free(ts);
    return n;
}

/* One scan per camera, applied in camera order.  logit: double[n_voxels]
 * (in/out); depth, opacity: per pixel of every view in order; params =
 * (p_hit, p_miss, l_min, l_max, p_occ, a_min); bits (may be NULL): u32 words
 * x-fastest, bit i of word w = voxel 32 w + i, set iff occupied.  ties
 * (may be NULL) gets the number of near-tie intervals met.  Returns 0, or
 * -1 on bad input. */
int orc_occupancy_update(const int32_t *dims, const double *origin, double vox, double *logit,
                         const double *cams, int n_views, const float *depth, const float *opacity,
                         const double *params, uint32_t *bits, int64_t *ties_out)
{
    const double p_hit = params[0], p_miss = params[1], l_min = params[2], l_max = params[3];
    const double p_occ = params[4], a_min = params[5];
    const int64_t nv = (int64_t)dims[0] * dims[1] * dims[2];
    double *conf = (double *)malloc(sizeof(double) * (size_t)nv);
    uint8_t *miss = (uint8_t *)malloc((size_t)nv);
    const int64_t cap = 4 * (int64_t)(dims[0] + dims[1] + dims[2]) + 16;
    int64_t ties_total = 0;
    if (!conf || !miss) { free(conf); free(miss); return -1; }
    int64_t pix0 = 0;
    for (int v = 0; v < n_views; ++v) {
        const double *cam = cams + 16 * v;
        const int64_t W = (int64_t)cam[1], H = (int64_t)cam[2];
        for (int64_t i = 0; i < nv; ++i) { conf[i] = 0.0; miss[i] = 0; }
        int64_t scan_ties = 0;
#pragma omp parallel reduction(+ : scan_ties)
        {
            int64_t *vox_list = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 256)
            for (int64_t p = 0; p < W * H; ++p) {
                const double A = (double)opacity[pix0 + p];
                if (!(A >= a_min) || !vox_list) continue;
                double o[3], d[3];
                orc_ray(cam, (double)(p % W) + 0.5, (double)(p / W) + 0.5, o, d);
                const double t_end = (double)depth[pix0 + p] / A;
                int nt = 0;
                const int64_t n = segment_voxels(dims, origin, vox, o, d, t_end, vox_list, cap, &nt);
                scan_ties += nt;
                for (int64_t k = 0; k < n; ++k) {
#pragma omp atomic write
                    miss[vox_list[k]] = 1;
                }
                int64_t c[3];
                int inside = 1;
                for (int a = 0; a < 3; ++a) {
                    c[a] = (int64_t)floor((o[a] + t_end * d[a] - origin[a]) / vox);
                    if (c[a] < 0 || c[a] >= dims[a]) inside = 0;
                }
                if (inside) {
                    const int64_t e = (c[2] * dims[1] + c[1]) * dims[0] + c[0];
#pragma omp critical(orc_occ_hit)
                    if (A > conf[e]) conf[e] = A;
                }
            }
            free(vox_list);
        }
        ties_total += scan_ties;
        for (int64_t i = 0; i < nv; ++i) {
            double upd = 0.0;
            if (conf[i] > 0.0) upd = logit_of(0.5 + (p_hit - 0.5) * conf[i]);
            else if (miss[i]) upd = logit_of(p_miss);
            else continue;
            double L = logit[i] + upd;
            logit[i] = L < l_min ? l_min : (L > l_max ? l_max : L);
        }
        pix0 += W * H;
    }
    if (bits) {
        const double thr = logit_of(p_occ);
        for (int64_t w = 0; w < nv / 32; ++w) bits[w] = 0;
        for (int64_t i = 0; i < nv; ++i)
            if (logit[i] > thr) bits[i >> 5] |= 1u << (i & 31);
    }
    if (ties_out) *ties_out = ties_total;
    free(conf);
    free(miss);
    return 0;
}

/* the segment traversal alone, for pins */
int64_t orc_segment_voxels(const int32_t *dims, const double *origin, double vox, const double *o, const double *d,
                           double t_end, int64_t *out, int64_t cap)
{
    return segment_voxels(dims, origin, vox, o, d, t_end, out, cap, NULL);
}

/* ------------------------------------------------------------------ */
/* Adaptive assignment of occupied voxels to networks (Alg. 1 stage II) */
/* ------------------------------------------------------------------ */
/*
 * Readings taken (the algorithm leaves them open): the "minimum coordinate"
 * is the lexicographic (z, y, x) minimum, i.e. the smallest linear index
 * (x fastest); the s - 1 "nearest neighbours" are the unassigned occupied
 * voxels of smallest squared distance to the anchor (voxel units), ties
 * broken by the smaller linear index; s = S / n (integer division) and the
 * last network takes every voxel still unassigned.
 */

static void swap_u64(uint64_t *a, uint64_t *b) { uint64_t t = *a; *a = *b; *b = t; }

/* rearranges a[0..n) so that a[k] is the k-th smallest (0-based), smaller
 * ones before it */
static void quickselect_u64(uint64_t *a, int64_t n, int64_t k)
{
    int64_t lo = 0, hi = n - 1;
    uint64_t seed = 88172645463325252ull;
    while (lo < hi) {
        seed ^= seed << 13; seed ^= seed >> 7; seed ^= seed << 17;
        const int64_t pi = lo + (int64_t)(seed % (uint64_t)(hi - lo + 1));
        const uint64_t pivot = a[pi];
        swap_u64(&a[pi], &a[hi]);
        int64_t st = lo;
        for (int64_t i = lo; i < hi; ++i)
            if (a[i] < pivot) swap_u64(&a[i], &a[st++]);
        swap_u64(&a[st], &a[hi]);
        if (st == k) return;
        if (st < k) lo = st + 1; else hi = st - 1;
    }
}

/* occupied voxels given by their linear indices in increasing order
 * (vox_idx[S], dims x-fastest); writes field[S].  Returns 0, or -1. */
int orc_assign_fields(const int32_t *dims, const int64_t *vox_idx, int64_t S, int n, int32_t *field)
{
    if (n < 1 || S < n) return -1;
    const int64_t s = S / n;
    uint8_t *done = (uint8_t *)calloc((size_t)S, 1);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)S);
    if (!done || !keys) { free(done); free(keys); return -1; }
    int64_t cursor = 0;                      /* every position before it is assigned */
    for (int k = 0; k < n; ++k) {
        while (cursor < S && done[cursor]) ++cursor;
        if (k == n - 1) {
            for (int64_t i = cursor; i < S; ++i)
                if (!done[i]) { field[i] = k; done[i] = 1; }
            break;
        }
        const int64_t a = cursor;            /* anchor: smallest unassigned linear index */
        const int64_t ax = vox_idx[a] % dims[0], ay = (vox_idx[a] / dims[0]) % dims[1],
                      az = vox_idx[a] / ((int64_t)dims[0] * dims[1]);
        int64_t m = 0;
        for (int64_t i = a; i < S; ++i) {
            if (done[i]) continue;
            const int64_t x = vox_idx[i] % dims[0], y = (vox_idx[i] / dims[0]) % dims[1],
                          z = vox_idx[i] / ((int64_t)dims[0] * dims[1]);
            const uint64_t d2 = (uint64_t)((x - ax) * (x - ax) + (y - ay) * (y - ay) + (z - az) * (z - az));
            keys[m++] = (d2 << 32) | (uint64_t)i;    /* position order = linear-index order */
        }
        /* the anchor (distance 0, smallest index) and its s - 1 nearest */
        if (s < m) quickselect_u64(keys, m, s - 1);
        const int64_t take = s < m ? s : m;
        for (int64_t q = 0; q < take; ++q) {
            const int64_t i = (int64_t)(keys[q] & 0xffffffffull);
            field[i] = k;
            done[i] = 1;
        }
    }
    free(done);
    free(keys);
    return 0;
}

/* ------------------------------------------------------------------ */
/* The global 360NeRF as a distillation teacher (network table of the   */
/* implementation details) and the distillation loss (Eq. 7)            */
/* ------------------------------------------------------------------ */
/*
 * Readings: the global position is the world point mapped by a global
 * affine (scene box onto [-1, 1]^3) and encoded with L = 10 (63 features),
 * the view direction with L = 4 (27) as in the tiny networks (this makes
 * the parameter count 595,844, the paper's "about 0.596M"); layers 1-7 are
 * ReLU, layer 8 has no activation, the density head is ReLU, the feature
 * head ReLU, layer 10 ReLU, layer 11 sigmoid; the skip connection feeds
 * [layer-4 output; F(x)] into layer 5.  Eq. 7 sums over a field's I samples
 * (sigma_k - sigma)^2 + |c_k - c|^2 and divides by I.
 */

#define ORC_T_W 256
#define ORC_T_C 128

int64_t orc_teacher_param_count(void)
{
    const int64_t W = ORC_T_W;
    return (W * ORC_PE_POS + W) + 3 * (W * W + W) + (W * (W + ORC_PE_POS) + W) + 3 * (W * W + W) + (W + 1) +
           (W * W + W) + (ORC_T_C * (W + ORC_PE_DIR) + ORC_T_C) + (3 * ORC_T_C + 3);
}

/* dense() with inputs and weights rounded to BF16 and the bias not (the
 * teacher's BF16 reading of its layers whose bias is added in FP32) */
static void dense_bf16_fb(const float *Wm, const float *b, int n_out, int n_in, const double *x, double *y)
{
    double xq[512];
    for (int c = 0; c < n_in; ++c) xq[c] = bf16r(x[c]);
    for (int r = 0; r < n_out; ++r) {
        double acc = (double)b[r];
        for (int c = 0; c < n_in; ++c) acc += bf16r((double)Wm[(int64_t)r * n_in + c]) * xq[c];
        y[r] = acc;
    }
}

/* The teacher at one point.  quant == 2 is the BF16 reading (the library's
 * tensor-core teacher): every layer but the density head and layer 11 takes
 * its inputs and weights rounded to BF16; layers 1, 5 and 10 (whose input
 * has a spare column for it) their bias too, the others an unrounded bias;
 * the density head (on layer 8's unrounded output) and layer 11 stay FP64
 * on the FP32 weights; sums in FP64. */
static void teacher_forward(const float *w, const double *aff, const double *p, const double *d, double *out,
                            int quant)
{
    const int W = ORC_T_W;
    void (*mat_b)(const float *, const float *, int, int, const double *, double *) = quant == 2 ? dense_bf16 : dense;
    void (*mat_f)(const float *, const float *, int, int, const double *, double *) =
        quant == 2 ? dense_bf16_fb : dense;
    double xg[3], pe[ORC_PE_POS], h[ORC_T_W + ORC_PE_POS], z[ORC_T_W], ped[ORC_PE_DIR];
    for (int a = 0; a < 3; ++a) xg[a] = aff[a] * p[a] + aff[3 + a];
    encode(xg, 10, pe);
    encode(d, 4, ped);
    const float *q = w;
    mat_b(q, q + W * ORC_PE_POS, W, ORC_PE_POS, pe, z);                 /* layer 1 */
    q += W * ORC_PE_POS + W;
    for (int r = 0; r < W; ++r) h[r] = z[r] > 0.0 ? z[r] : 0.0;
    for (int l = 2; l <= 4; ++l) {                                       /* layers 2-4 */
        mat_f(q, q + W * W, W, W, h, z);
        q += W * W + W;
        for (int r = 0; r < W; ++r) h[r] = z[r] > 0.0 ? z[r] : 0.0;
    }
    for (int k = 0; k < ORC_PE_POS; ++k) h[W + k] = pe[k];               /* skip: [h4; F(x)] */
    mat_b(q, q + W * (W + ORC_PE_POS), W, W + ORC_PE_POS, h, z);         /* layer 5 */
    q += W * (W + ORC_PE_POS) + W;
    for (int r = 0; r < W; ++r) h[r] = z[r] > 0.0 ? z[r] : 0.0;
    for (int l = 6; l <= 8; ++l) {                                       /* layers 6-8 (8: linear) */
        mat_f(q, q + W * W, W, W, h, z);
        q += W * W + W;
        for (int r = 0; r < W; ++r) h[r] = (l < 8) ? (z[r] > 0.0 ? z[r] : 0.0) : z[r];
    }
    double s;
    dense(q, q + W, 1, W, h, &s);                                        /* layer 9, density */
    q += W + 1;
    out[0] = s > 0.0 ? s : 0.0;
    double f[ORC_T_W + ORC_PE_DIR];
    mat_f(q, q + W * W, W, W, h, z);                                     /* layer 9, feature */
    q += W * W + W;
    for (int r = 0; r < W; ++r) f[r] = z[r] > 0.0 ? z[r] : 0.0;
    for (int k = 0; k < ORC_PE_DIR; ++k) f[W + k] = ped[k];
    double g[ORC_T_C], zo[3];
    mat_b(q, q + ORC_T_C * (W + ORC_PE_DIR), ORC_T_C, W + ORC_PE_DIR, f, g);   /* layer 10 */
    q += ORC_T_C * (W + ORC_PE_DIR) + ORC_T_C;
    for (int r = 0; r < ORC_T_C; ++r) g[r] = g[r] > 0.0 ? g[r] : 0.0;
    dense(q, q + 3 * ORC_T_C, 3, ORC_T_C, g, zo);                        /* layer 11 */
    for (int c = 0; c < 3; ++c) out[1 + c] = sigm(zo[c]);
}

/* out[n][4] = (sigma, r, g, b) of the teacher at points p[n][3], directions
 * d[n][3]; quant 0: FP64, 2: the BF16 reading above */
void orc_teacher_eval(const float *w, const double *aff, int64_t n, const double *p, const double *d, double *out,
                      int quant)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) teacher_forward(w, aff, p + 3 * i, d + 3 * i, out + 4 * i, quant);
}

/* Eq. 7 summed over the fields: loss = sum_i [(sigma_s - sigma_t)^2 +
 * |c_s - c_t|^2] / I over the n samples (field[i] = the sample's field,
 * target[i] = the teacher's (sigma, r, g, b)); grad[F][P] (zeroed here)
 * receives d loss / d student weights.  Returns the loss. */
double orc_distill_loss_grad(const float *weights, const float *affine, int n_fields, int W, int H, int act,
                             double sigma_scale, int64_t n, const double *p, const double *d, const int32_t *field,
                             const double *target, double I, double *grad)
{
    orc_arch A = {W, H, act, sigma_scale, 0};
    const int64_t P = orc_param_count(W, H);
    for (int64_t i = 0; i < P * n_fields; ++i) grad[i] = 0.0;
    double loss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const int f = field[i];
        const double aff[6] = {affine[6 * f], affine[6 * f + 1], affine[6 * f + 2],
                               affine[6 * f + 3], affine[6 * f + 4], affine[6 * f + 5]};
        orc_cache c;
        mlp_forward(weights + (int64_t)f * P, &A, aff, p + 3 * i, d + 3 * i, &c);
        const double ds = c.sigma - target[4 * i];
        const double dc[3] = {c.rgb[0] - target[4 * i + 1], c.rgb[1] - target[4 * i + 2], c.rgb[2] - target[4 * i + 3]};
        loss += (ds * ds + dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]) / I;
        const double drgb[3] = {2.0 * dc[0] / I, 2.0 * dc[1] / I, 2.0 * dc[2] / I};
        mlp_backward(weights + (int64_t)f * P, &A, &c, 2.0 * ds / I, drgb, grad + (int64_t)f * P);
    }
    return loss;
}

/* The adjoint of the fields' MLPs at n points for given per-sample output
 * gradients dl[n][4] = d loss / d (sigma, r, g, b): grad[F][P] (zeroed here)
 * = sum_i J_i^T dl_i.  margin[i] (may be NULL) receives the smallest
 * |pre-activation| over the sample's ReLU units: below ~1e-4 an FP32
 * evaluation may take the other branch (a near-kink).  quant 0: FP64;
 * quant 2: the BF16 reading of the forward pass and its adjoint. */
void orc_mlp_grad_points(const float *weights, const float *affine, int n_fields, int W, int H, int act,
                         double sigma_scale, int quant, int64_t n, const double *p, const double *d,
                         const int32_t *field, const double *dl, double *grad, double *margin)
{
    orc_arch A = {W, H, act, sigma_scale, quant};
    const int64_t P = orc_param_count(W, H);
    for (int64_t i = 0; i < P * n_fields; ++i) grad[i] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const int f = field[i];
        const double aff[6] = {affine[6 * f], affine[6 * f + 1], affine[6 * f + 2],
                               affine[6 * f + 3], affine[6 * f + 4], affine[6 * f + 5]};
        orc_cache c;
        mlp_forward(weights + (int64_t)f * P, &A, aff, p + 3 * i, d + 3 * i, &c);
        mlp_backward(weights + (int64_t)f * P, &A, &c, dl[4 * i], dl + 4 * i + 1, grad + (int64_t)f * P);
        if (margin) {
            double m = INFINITY;
            for (int k = 0; k < H; ++k)
                for (int r = 0; r < W; ++r) m = fmin(m, fabs(c.z[k][r]));
            for (int r = 0; r < W; ++r) m = fmin(m, fabs(c.zc[r]));
            if (act == 1) m = fmin(m, fabs(c.zh[0]));
            margin[i] = m;
        }
    }
}
