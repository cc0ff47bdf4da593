// The global 360NeRF (network table of the implementation details) as the
// distillation teacher of the local fields (Eq. 7): 8 fully connected layers
// of width 256 with a skip of F(x) into layer 5, a density head, a feature
// head, and a 128-wide colour layer on [feature; F(d)].  Its layers are
// plain dense GEMMs over the sample batch (K up to 319, N = 256), run as
// cuBLAS GEMMs in FP32 or, on request, on the tensor cores with TF32
// operands and FP32 accumulation; the encodings, bias + activation
// epilogues and the output heads are this file's kernels, in FP32.
//
// Activations live row-major per sample in two ping-pong buffers whose
// trailing columns hold the encodings the skip and the colour layer read:
//   A: [n][320]  columns 0..255 activations, 256..318 F(x), 319 zero
//   B: [n][288]  columns 0..255 activations, 256..282 F(d), 283..287 zero
#include <cublas_v2.h>

#include "internal.cuh"

namespace roam {

namespace {

constexpr int kTW = 256, kTC = 128;
constexpr int kLdA = 320, kLdB = 288;

__global__ void k_teacher_encode(int64_t n, const float *__restrict__ p, const float *__restrict__ d, TeacherAffine aff,
                                 float *__restrict__ A, float *__restrict__ B)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float x[3], dv[3];
        for (int a = 0; a < 3; ++a) {
            x[a] = fmaf(aff.v[a], p[3 * i + a], aff.v[3 + a]);
            dv[a] = d[3 * i + a];
        }
        float *pa = A + i * kLdA + kTW;
        float *pb = B + i * kLdB + kTW;
        for (int a = 0; a < 3; ++a) { pa[a] = x[a]; pb[a] = dv[a]; }
        for (int k = 0; k < 10; ++k)
            for (int a = 0; a < 3; ++a) {
                float s, c;
                sincospif(x[a] * (float)(1 << k), &s, &c);
                pa[3 + 6 * k + a] = s;
                pa[6 + 6 * k + a] = c;
            }
        pa[63] = 0.f;
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) {
                float s, c;
                sincospif(dv[a] * (float)(1 << k), &s, &c);
                pb[3 + 6 * k + a] = s;
                pb[6 + 6 * k + a] = c;
            }
        for (int q = 27; q < 32; ++q) pb[q] = 0.f;
    }
}

// Y[i][0..N) += b, then ReLU when relu; N and ld multiples of 4: one float4
// per thread, a block of rows per CTA (threadIdx.y)
__global__ void k_bias_act(int64_t n, int N, int ld, float *__restrict__ Y, const float *__restrict__ b, int relu)
{
    const int c4 = threadIdx.x;                       // float4 column, blockDim.x = N / 4
    const float4 bb = reinterpret_cast<const float4 *>(b)[c4];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < n; i += (int64_t)gridDim.x * blockDim.y) {
        float4 *y = reinterpret_cast<float4 *>(Y + i * ld) + c4;
        float4 v = *y;
        v.x += bb.x; v.y += bb.y; v.z += bb.z; v.w += bb.w;
        if (relu) {
            v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
        }
        *y = v;
    }
}

// the layers of the API layout: output width, input width
constexpr int kTLayers = 12;
__host__ __device__ constexpr int t_out(int l)
{
    return l == 8 ? 1 : (l == 10 ? kTC : (l == 11 ? 3 : kTW));
}
__host__ __device__ constexpr int t_in(int l)
{
    return l == 0 ? kPeX : (l == 4 ? kTW + kPeX : (l == 10 ? kTW + kPeD : (l == 11 ? kTC : kTW)));
}
__host__ __device__ constexpr int round4i(int x) { return (x + 3) & ~3; }

// API layout -> every layer's matrix with its rows padded to a multiple of
// 4 floats (zeros), bias after it (16-byte aligned operands for the GEMMs)
__global__ void k_teacher_pad(const float *__restrict__ w, float *__restrict__ wp)
{
    int64_t src = 0, dst = 0;
    for (int l = 0; l < kTLayers; ++l) {
        const int N = t_out(l), K = t_in(l), Kp = round4i(K);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)N * Kp + N;
             e += (int64_t)gridDim.x * blockDim.x) {
            float v = 0.f;
            if (e < (int64_t)N * Kp) {
                const int r = (int)(e / Kp), k = (int)(e % Kp);
                if (k < K) v = w[src + (int64_t)r * K + k];
            } else {
                v = w[src + (int64_t)N * K + (e - (int64_t)N * Kp)];
            }
            wp[dst + e] = v;
        }
        src += (int64_t)N * K + N;
        dst += round4i((int)((int64_t)N * Kp + N));
    }
}

// out[i] = (relu(s + b_s), sigmoid(z + b_o))
__global__ void k_teacher_out(int64_t n, const float *__restrict__ s, const float *__restrict__ bs,
                              const float *__restrict__ z, const float *__restrict__ bo, float4 *__restrict__ out)
{
    const float b0 = bs[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float sg = fmaxf(s[i] + b0, 0.f);
        float c[3];
        for (int k = 0; k < 3; ++k) c[k] = 1.f / (1.f + expf(-(z[3 * i + k] + bo[k])));
        out[i] = make_float4(sg, c[0], c[1], c[2]);
    }
}

// C[n][N] (ldc) = X[n][K] (ldx) W^T, W row-major [N][K]: column-major
// C^T = W X^T with W read transposed
cublasStatus_t dense(cublasHandle_t h, int64_t n, int N, int K, const float *W, const float *X, int ldx, float *C,
                     int ldc)
{
    const float one = 1.f, zero = 0.f;
    return cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, N, (int)n, K, &one, W, K, X, ldx, &zero, C, ldc);
}

}  // namespace

int64_t teacher_padded_floats()
{
    int64_t t = 0;
    for (int l = 0; l < kTLayers; ++l) t += round4i(t_out(l) * round4i(t_in(l)) + t_out(l));
    return t;
}

void launch_teacher_pad(const float *w, float *wp, cudaStream_t s) { k_teacher_pad<<<512, 256, 0, s>>>(w, wp); }

int64_t teacher_param_count()
{
    return ((int64_t)kTW * kPeX + kTW) + 3 * ((int64_t)kTW * kTW + kTW) + ((int64_t)kTW * (kTW + kPeX) + kTW) +
           3 * ((int64_t)kTW * kTW + kTW) + (kTW + 1) + ((int64_t)kTW * kTW + kTW) +
           ((int64_t)kTC * (kTW + kPeD) + kTC) + (3 * kTC + 3);
}

size_t teacher_workspace_floats(int64_t n) { return (size_t)n * (kLdA + kLdB + 1 + 3); }

// w: device FP32 parameters padded by launch_teacher_pad (each layer's rows
// padded to a multiple of 4 floats with zeros, then its bias)
int teacher_eval(void *handle, const float *w, TeacherAffine aff, int64_t n, const float *p, const float *d,
                 float4 *out, float *ws, bool tf32, cudaStream_t s)
{
    cublasHandle_t h = static_cast<cublasHandle_t>(handle);
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return 1;
    if (cublasSetMathMode(h, tf32 ? CUBLAS_TF32_TENSOR_OP_MATH : CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS)
        return 1;
    float *A = ws, *B = A + (size_t)n * kLdA, *sig = B + (size_t)n * kLdB, *z = sig + n;
    const int grid = 1024;
    k_teacher_encode<<<grid, 256, 0, s>>>(n, p, d, aff, A, B);
    const float *q = w;
    int st = 0;
    // K: the layer's input width; the GEMM runs over it rounded up to 4 (the
    // padded weight columns and the activation columns there are zero)
    auto layer = [&](int N, int K, const float *X, int ldx, float *Y, int ldy, int relu) {
        const int Kp = round4i(K);
        st |= dense(h, n, N, Kp, q, X, ldx, Y, ldy) != CUBLAS_STATUS_SUCCESS;
        const dim3 blk((unsigned)(N / 4), (unsigned)(256 / (N / 4)));
        k_bias_act<<<grid, blk, 0, s>>>(n, N, ldy, Y, q + (int64_t)N * Kp, relu);
        q += round4i(N * Kp + N);
    };
    layer(kTW, kPeX, A + kTW, kLdA, B, kLdB, 1);          // layer 1 on F(x)
    layer(kTW, kTW, B, kLdB, A, kLdA, 1);                 // layer 2
    layer(kTW, kTW, A, kLdA, B, kLdB, 1);                 // layer 3
    layer(kTW, kTW, B, kLdB, A, kLdA, 1);                 // layer 4 (A keeps F(x) after it)
    layer(kTW, kTW + kPeX, A, kLdA, B, kLdB, 1);          // layer 5 on [layer 4; F(x)]
    layer(kTW, kTW, B, kLdB, A, kLdA, 1);                 // layer 6
    layer(kTW, kTW, A, kLdA, B, kLdB, 1);                 // layer 7
    layer(kTW, kTW, B, kLdB, A, kLdA, 0);                 // layer 8, linear
    // density head: N = 1
    st |= dense(h, n, 1, kTW, q, A, kLdA, sig, 1) != CUBLAS_STATUS_SUCCESS;
    const float *b_sig = q + kTW;
    q += round4i(kTW + 1);
    layer(kTW, kTW, A, kLdA, B, kLdB, 1);                 // feature head (B keeps F(d) after it)
    layer(kTC, kTW + kPeD, B, kLdB, A, kLdA, 1);          // layer 10 on [feature; F(d)]
    st |= dense(h, n, 3, kTC, q, A, kLdA, z, 3) != CUBLAS_STATUS_SUCCESS;   // layer 11
    const float *b_out = q + 3 * kTC;
    k_teacher_out<<<grid, 256, 0, s>>>(n, sig, b_sig, z, b_out, out);
    return st;
}

}  // namespace roam
