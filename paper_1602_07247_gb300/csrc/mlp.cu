// Learned proposal: a multilayer perceptron that maps sum-normalised signals
// to (x, y, ln E) (the role of the neural-network reconstruction of
// Sec. 5.1.3), trained on the GPU by the kernels below.
//
//   u = s / S,  z1 = W1 u + b1,  h1 = GELU(z1),  z2 = W2 h1 + b2,
//   h2 = GELU(z2),  o = W3 h2 + b3,   GELU(x) = 0.5 x (1 + erf(x / sqrt 2)).
//
// Targets: (x / xy_scale, y / xy_scale, (ln E - loge_mean) / loge_std); loss:
// mean squared error; optimiser: Adam on FP32 master weights.  With bf16 = 1
// every matrix-product operand is rounded to BF16 and products accumulate in
// FP32 (mixed precision); with bf16 = 0 everything is FP32.
//
// With bf16 = 1 and input and hidden widths that are multiples of 8 and at
// most 256, every product of the hidden layers runs on the tensor cores
// (tcgen05, umma.cu): the forward products with bias and GELU fused (z kept
// for the backward pass), the backward product dZ1 = (dZ2 W2) GELU'(z1)
// fused likewise, and the weight gradients dW = dZ^T X with the batch as the
// contraction (from transposed BF16 copies the epilogues write).  The 3-wide
// output layer and its gradients, and the FP32 mode, use the tiled SIMT kernel
// below (64 x 64 output tile per block, 4 x 4 per thread, K staged through
// shared memory in steps of 16).  All sums are taken in a fixed order, so
// training is bitwise reproducible.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "internal.cuh"

struct ants_mlp {
    ants_ctx *ctx = nullptr;
    int device = 0;
    int n_in = 0, H = 0;
    ants_mlp_config cfg{};
    size_t n_par = 0;
    float *d_par = nullptr;  // FP32 master weights
    float *d_m = nullptr, *d_v = nullptr;
    int adam_t = 0;
    // BF16 copies of W1 [Hp][Ip] and W2 [Hp][Hp] and FP32 biases [Hp] for
    // tensor-core inference, zero-padded to multiples of 8 (Ip, Hp); refreshed
    // on use
    __nv_bfloat16 *d_w1b = nullptr, *d_w2b = nullptr;
    float *d_bpad = nullptr;  // b1 [Hp], b2 [Hp]
    bool bf16_stale = true;
    __nv_bfloat16 *d_w2tb = nullptr;  // W2 transposed [H][H] (tensor-core training only)
};

namespace ants {

namespace {

struct Offsets {
    size_t W1, b1, W2, b2, W3, b3, total;
};

Offsets offsets(int n_in, int H)
{
    Offsets o;
    o.W1 = 0;
    o.b1 = o.W1 + (size_t)H * n_in;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (size_t)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + 3 * (size_t)H;
    o.total = o.b3 + 3;
    return o;
}

__device__ __forceinline__ float rbf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

// C[m][n] = sum_k opA(m,k) opB(k,n) + beta C[m][n]
// opA(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  opB(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
template <bool TA, bool TB, bool BF>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                   const float *__restrict__ B, int ldb, float *__restrict__ C,
                                                   int ldc, float beta)
{
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int l = threadIdx.x; l < 1024; l += 256) {
            int mm, kk;
            if (TA) { mm = l & 63; kk = l >> 6; }   // A[k][m]: m contiguous
            else { kk = l & 15; mm = l >> 4; }      // A[m][k]: k contiguous
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.0f;
            if (m < M && k < K) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            As[kk][mm] = BF ? rbf16(v) : v;
        }
        for (int l = threadIdx.x; l < 1024; l += 256) {
            int nn, kk;
            if (TB) { kk = l & 15; nn = l >> 4; }   // B[n][k]: k contiguous
            else { nn = l & 63; kk = l >> 6; }      // B[k][n]: n contiguous
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.0f;
            if (n < N && k < K) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            Bs[kk][nn] = BF ? rbf16(v) : v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (beta != 0.0f) v = fmaf(beta, C[(size_t)m * ldc + n], v);
            C[(size_t)m * ldc + n] = v;
        }
    }
}

// u = s / S for rows idx[r] (idx nullable: rows r) -> U [n][n_in]; one warp per row
__global__ void normalize_rows(const float *__restrict__ sig, const long *__restrict__ idx, long n, int n_in,
                               float *__restrict__ U)
{
    const long r = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const long src = idx ? idx[r] : r;
    const float *s = sig + src * n_in;
    float S = 0.0f;
    for (int i = lane; i < n_in; i += 32) S += s[i];
    for (int o = 16; o; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    const float inv = S > 0.0f ? 1.0f / S : 0.0f;
    for (int i = lane; i < n_in; i += 32) U[r * n_in + i] = s[i] * inv;
}

// Z += b (row-broadcast); Hout = GELU(Z)  (Z keeps the pre-activation)
__global__ void bias_gelu(float *__restrict__ Z, long n, int H, const float *__restrict__ b, float *__restrict__ Hout)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * H) return;
    const float z = Z[t] + b[t % H];
    Z[t] = z;
    Hout[t] = gelu(z);
}

__global__ void bias_add(float *__restrict__ Z, long n, int H, const float *__restrict__ b)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * H) return;
    Z[t] += b[t % H];
}

// dZ *= GELU'(Z)
__global__ void gelu_backward(float *__restrict__ dZ, const float *__restrict__ Z, long n)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dZ[t] *= gelu_grad(Z[t]);
}

// targets from truth rows idx[r]: (x / s, y / s, (ln E - mu) / sd)
__global__ void make_targets(const float *__restrict__ truth, const long *__restrict__ idx, long n,
                             ants_mlp_config cfg, float *__restrict__ T)
{
    const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const long s = idx ? idx[r] : r;
    const float *t = truth + s * 4;
    T[r * 3] = t[0] / cfg.xy_scale;
    T[r * 3 + 1] = t[1] / cfg.xy_scale;
    T[r * 3 + 2] = (logf(t[3]) - cfg.loge_mean) / cfg.loge_std;
}

// dO = 2 (O - T) / (n 3); per-block partial sums of (O - T)^2 / (n 3)
__global__ void mse_grad(const float *__restrict__ O, const float *__restrict__ T, long n, float *__restrict__ dO,
                         float *__restrict__ part)
{
    __shared__ float red[256];
    const float scale = 1.0f / (3.0f * (float)n);
    float acc = 0.0f;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < 3 * n; t += (long)gridDim.x * blockDim.x) {
        const float d = O[t] - T[t];
        if (dO) dO[t] = 2.0f * d * scale;
        acc += d * d * scale;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out[j] = sum_r X[r][j]: block (32, 8) per 32 columns; thread (c, t) adds
// rows t, t+8, ... in order, then a fixed tree over t (reproducible)
__global__ void column_sums(const float *__restrict__ X, long n, int N, float *__restrict__ out)
{
    __shared__ float red[8][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.0f;
    if (j < N)
        for (long r = threadIdx.y; r < n; r += 8) acc += X[r * N + j];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    for (int o = 4; o; o >>= 1) {
        if ((int)threadIdx.y < o) red[threadIdx.y][threadIdx.x] += red[threadIdx.y + o][threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.y == 0 && j < N) out[j] = red[0][threadIdx.x];
}

void launch_column_sums(const float *X, long n, int N, float *out, cudaStream_t s)
{
    column_sums<<<(unsigned)((N + 31) / 32), dim3(32, 8), 0, s>>>(X, n, N, out);
}

__global__ void adam_kernel(size_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// decode network outputs to start positions: (o0 s, o1 s, 0) and E
__global__ void decode_outputs(const float *__restrict__ O, long n, ants_mlp_config cfg, float *__restrict__ xyz,
                               float *__restrict__ E)
{
    const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    xyz[3 * r] = O[3 * r] * cfg.xy_scale;
    xyz[3 * r + 1] = O[3 * r + 1] * cfg.xy_scale;
    xyz[3 * r + 2] = 0.0f;
    if (E) E[r] = expf(fmaf(O[3 * r + 2], cfg.loge_std, cfg.loge_mean));
}

unsigned blocks_for(long n, int t) { return (unsigned)((n + t - 1) / t); }

// y[r][c] = bf16(x[r][c]) for c < cols, 0 for cols <= c < ld (rows of ld)
__global__ void to_bf16_pad(const float *__restrict__ x, long rows, int cols, int ld, __nv_bfloat16 *__restrict__ y)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * ld) return;
    const long r = i / ld;
    const int c = (int)(i - r * ld);
    y[i] = c < cols ? __float2bfloat16_rn(x[r * cols + c]) : __float2bfloat16_rn(0.0f);
}

__global__ void copy_pad(const float *__restrict__ x, int n, int ld, float *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ld) y[i] = i < n ? x[i] : 0.0f;
}

// U[r][i] = s[r][i] / S_r for i < n_in, 0 up to the row stride ld
__global__ void normalize_rows_pad(const float *__restrict__ sig, long n, int n_in, int ld, float *__restrict__ U)
{
    const long r = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *s = sig + r * n_in;
    float S = 0.0f;
    for (int i = lane; i < n_in; i += 32) S += s[i];
    for (int o = 16; o; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    const float inv = S > 0.0f ? 1.0f / S : 0.0f;
    for (int i = lane; i < ld; i += 32) U[r * ld + i] = i < n_in ? s[i] * inv : 0.0f;
}

// o[r][k] = sum_i bf16(h[r][i]) bf16(W3[k][i]) + b3[k] (h rows of ld); one warp per row
__global__ void output_layer(const __nv_bfloat16 *__restrict__ h, long n, int H, int ld, const float *__restrict__ W3,
                             const float *__restrict__ b3, float *__restrict__ O)
{
    const long r = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int i = lane; i < H; i += 32) {
        const float hv = __bfloat162float(h[r * ld + i]);
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] = fmaf(hv, rbf16(W3[k * H + i]), acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float v = acc[k];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) O[r * 3 + k] = v + b3[k];
    }
}

// XT[c][r] = bf16(X[r][c]) for r < n and 0 for n <= r < ldT (X [n][cols] FP32);
// 32 x 32 tiles through shared memory, block (32, 8)
__global__ void transpose_bf16(const float *__restrict__ X, long n, int cols, int ldT, __nv_bfloat16 *__restrict__ XT)
{
    __shared__ float tile[32][33];
    const long r0 = (long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32, tx = threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const long r = r0 + k;
        const int c = c0 + tx;
        tile[k][tx] = (r < n && c < cols) ? X[r * cols + c] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k;
        const long r = r0 + tx;
        if (c < cols && r < ldT) XT[(size_t)c * ldT + r] = __float2bfloat16_rn(tile[tx][k]);
    }
}

// BF16 copies of the hidden weights for the tensor cores: W1 [H][I], W2 [H][H]
// and W2 transposed
__global__ void weights_to_bf16(const float *__restrict__ W1, const float *__restrict__ W2, int H, int I,
                                __nv_bfloat16 *__restrict__ w1b, __nv_bfloat16 *__restrict__ w2b,
                                __nv_bfloat16 *__restrict__ w2tb)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long n1 = (long)H * I;
    if (t < n1) {
        w1b[t] = __float2bfloat16_rn(W1[t]);
    } else if (t < n1 + (long)H * H) {
        const long u = t - n1;
        const int r = (int)(u / H), c = (int)(u - (long)r * H);
        const __nv_bfloat16 v = __float2bfloat16_rn(W2[u]);
        w2b[u] = v;
        w2tb[(size_t)c * H + r] = v;
    }
}

// dZ2[b][i] = (sum_k bf16(dO[b][k]) bf16(W3[k][i])) GELU'(Z2[b][i])
__global__ void output_backward(const float *__restrict__ dO, const float *__restrict__ W3,
                                const float *__restrict__ Z2, long n, int H, float *__restrict__ dZ2)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * H) return;
    const long b = t / H;
    const int i = (int)(t - b * H);
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc = fmaf(rbf16(dO[b * 3 + k]), rbf16(W3[k * H + i]), acc);
    dZ2[t] = acc * gelu_grad(Z2[t]);
}

// gW3[k][i] = sum_b bf16(dO[b][k]) h2[b][i] (h2 BF16 [n][H]); one block per i,
// partial sums per thread in a fixed order, then a fixed tree
__global__ void output_weight_grad(const float *__restrict__ dO, const __nv_bfloat16 *__restrict__ h2, long n, int H,
                                   float *__restrict__ gW3)
{
    __shared__ float red[3][256];
    const int i = blockIdx.x;
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (long b = threadIdx.x; b < n; b += blockDim.x) {
        const float h = __bfloat162float(h2[b * H + i]);
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] = fmaf(rbf16(dO[b * 3 + k]), h, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) gW3[threadIdx.x * H + i] = red[threadIdx.x][0];
}

// C = opA(A) opB(B) (+ beta C), dispatching on transposes and precision
int gemm(bool ta, bool tb, bool bf, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
         int ldc, float beta, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return ANTS_OK;
    dim3 grid((N + 63) / 64, (M + 63) / 64);
#define ANTS_GEMM(TA_, TB_, BF_) gemm_kernel<TA_, TB_, BF_><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, beta)
    if (!ta && !tb) { if (bf) ANTS_GEMM(false, false, true); else ANTS_GEMM(false, false, false); }
    else if (!ta && tb) { if (bf) ANTS_GEMM(false, true, true); else ANTS_GEMM(false, true, false); }
    else if (ta && !tb) { if (bf) ANTS_GEMM(true, false, true); else ANTS_GEMM(true, false, false); }
    else { if (bf) ANTS_GEMM(true, true, true); else ANTS_GEMM(true, true, false); }
#undef ANTS_GEMM
    count_launch();
    return ANTS_OK;
}

// activations of one batch of up to cap rows
struct Acts {
    float *U, *Z1, *H1, *Z2, *H2, *O;
};

size_t acts_floats(long cap, int n_in, int H) { return (size_t)cap * (n_in + 4 * (size_t)H + 3); }

Acts carve(float *base, long cap, int n_in, int H)
{
    Acts a;
    a.U = base;
    a.Z1 = a.U + (size_t)cap * n_in;
    a.H1 = a.Z1 + (size_t)cap * H;
    a.Z2 = a.H1 + (size_t)cap * H;
    a.H2 = a.Z2 + (size_t)cap * H;
    a.O = a.H2 + (size_t)cap * H;
    return a;
}

// forward pass of n rows (idx nullable) whose activations go to `a`
void forward_batch(const ants_mlp *M, const float *par, const float *sig, const long *idx, long n, bool bf,
                   const Acts &a, cudaStream_t s)
{
    const Offsets o = offsets(M->n_in, M->H);
    const int H = M->H, I = M->n_in;
    normalize_rows<<<blocks_for(n, 8), 256, 0, s>>>(sig, idx, n, I, a.U);
    gemm(false, true, bf, (int)n, H, I, a.U, I, par + o.W1, I, a.Z1, H, 0.0f, s);
    bias_gelu<<<blocks_for(n * H, 256), 256, 0, s>>>(a.Z1, n, H, par + o.b1, a.H1);
    gemm(false, true, bf, (int)n, H, H, a.H1, H, par + o.W2, H, a.Z2, H, 0.0f, s);
    bias_gelu<<<blocks_for(n * H, 256), 256, 0, s>>>(a.Z2, n, H, par + o.b2, a.H2);
    gemm(false, true, bf, (int)n, 3, H, a.H2, H, par + o.W3, H, a.O, 3, 0.0f, s);
    bias_add<<<blocks_for(n * 3, 256), 256, 0, s>>>(a.O, n, 3, par + o.b3);
    count_launch(5);
}

// gradient of the batch loss into g (same layout as the parameters); dO set
void backward_batch(const ants_mlp *M, const float *par, long n, bool bf, const Acts &a, float *dO, float *dA,
                    float *dB, float *g, cudaStream_t s)
{
    const Offsets o = offsets(M->n_in, M->H);
    const int H = M->H, I = M->n_in;
    // output layer
    gemm(true, false, bf, 3, H, (int)n, dO, 3, a.H2, H, g + o.W3, H, 0.0f, s);
    launch_column_sums(dO, n, 3, g + o.b3, s);
    gemm(false, false, bf, (int)n, H, 3, dO, 3, par + o.W3, H, dA, H, 0.0f, s);  // dH2
    gelu_backward<<<blocks_for(n * H, 256), 256, 0, s>>>(dA, a.Z2, n * H);        // dZ2
    // second hidden layer
    gemm(true, false, bf, H, H, (int)n, dA, H, a.H1, H, g + o.W2, H, 0.0f, s);
    launch_column_sums(dA, n, H, g + o.b2, s);
    gemm(false, false, bf, (int)n, H, H, dA, H, par + o.W2, H, dB, H, 0.0f, s);  // dH1
    gelu_backward<<<blocks_for(n * H, 256), 256, 0, s>>>(dB, a.Z1, n * H);        // dZ1
    // first hidden layer
    gemm(true, false, bf, H, I, (int)n, dB, H, a.U, I, g + o.W1, I, 0.0f, s);
    launch_column_sums(dB, n, H, g + o.b1, s);
    count_launch(5);
}

// ---- tensor-core training (BF16 operands) ---------------------------------

// the shapes the tensor-core products take: widths multiples of 8, at most 256
bool tc_trainable(const ants_mlp *M) { return M->n_in % 8 == 0 && M->H % 8 == 0 && M->n_in <= 256 && M->H <= 256; }

long round8(long n) { return (n + 7) & ~7L; }

// buffers of one batch of up to cap rows (FP32 and BF16 parts 256-byte aligned)
struct TcActs {
    float *U, *Z1, *Z2, *O, *dZ2, *dZ1;
    __nv_bfloat16 *UT, *H1, *H1T, *H2, *dZ2T, *dZ1T;
};

size_t tc_bytes(long cap, int I, int H)
{
    const long ldT = round8(cap);
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return r((size_t)cap * I * 4) + 4 * r((size_t)cap * H * 4) + r((size_t)cap * 3 * 4) + r((size_t)I * ldT * 2) +
           2 * r((size_t)cap * H * 2) + 3 * r((size_t)H * ldT * 2);
}

TcActs tc_carve(unsigned char *base, long cap, int I, int H)
{
    const long ldT = round8(cap);
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    TcActs a;
    unsigned char *p = base;
    auto f = [&](size_t n) { float *q = (float *)p; p += r(n * 4); return q; };
    auto h = [&](size_t n) { __nv_bfloat16 *q = (__nv_bfloat16 *)p; p += r(n * 2); return q; };
    a.U = f((size_t)cap * I);
    a.Z1 = f((size_t)cap * H);
    a.Z2 = f((size_t)cap * H);
    a.dZ2 = f((size_t)cap * H);
    a.dZ1 = f((size_t)cap * H);
    a.O = f((size_t)cap * 3);
    a.UT = h((size_t)I * ldT);
    a.H1 = h((size_t)cap * H);
    a.H2 = h((size_t)cap * H);
    a.H1T = h((size_t)H * ldT);
    a.dZ2T = h((size_t)H * ldT);
    a.dZ1T = h((size_t)H * ldT);
    return a;
}

// BF16 weight copies from the FP32 masters (allocated on first use)
int tc_refresh_weights(ants_mlp *M, cudaStream_t s)
{
    const Offsets o = offsets(M->n_in, M->H);
    const int H = M->H, I = M->n_in;
    if (!M->d_w1b) {
        ANTS_CUDA_TRY(cudaMalloc(&M->d_w1b, (size_t)H * I * sizeof(__nv_bfloat16)), "bf16 weights");
        ANTS_CUDA_TRY(cudaMalloc(&M->d_w2b, (size_t)H * H * sizeof(__nv_bfloat16)), "bf16 weights");
        ANTS_CUDA_TRY(cudaMalloc(&M->d_bpad, 2 * (size_t)H * sizeof(float)), "padded biases");
    }
    if (!M->d_w2tb) ANTS_CUDA_TRY(cudaMalloc(&M->d_w2tb, (size_t)H * H * sizeof(__nv_bfloat16)), "bf16 weights");
    const long n = (long)H * I + (long)H * H;
    weights_to_bf16<<<blocks_for(n, 256), 256, 0, s>>>(M->d_par + o.W1, M->d_par + o.W2, H, I, M->d_w1b, M->d_w2b,
                                                        M->d_w2tb);
    count_launch();
    // the inference path's padded copies are these (widths already multiples of 8), biases aside
    M->bf16_stale = true;
    return ANTS_OK;
}

// forward of n rows (idx nullable) on the tensor cores into a.O; with
// want_bwd the transposed copies the weight gradients need are written too
int tc_forward(ants_ctx *ctx, const ants_mlp *M, const float *sig, const long *idx, long n, bool want_bwd,
               const TcActs &a, cudaStream_t s)
{
    const Offsets o = offsets(M->n_in, M->H);
    const int H = M->H, I = M->n_in;
    const int ldT = (int)round8(n);
    normalize_rows<<<blocks_for(n, 8), 256, 0, s>>>(sig, idx, n, I, a.U);
    count_launch();
    if (want_bwd) {
        transpose_bf16<<<dim3((unsigned)((ldT + 31) / 32), (unsigned)((I + 31) / 32)), dim3(32, 8), 0, s>>>(
            a.U, n, I, ldT, a.UT);
        count_launch();
    }
    int rc = mma_train_forward(ctx, a.U, true, M->d_w1b, M->d_par + o.b1, (int)n, H, I, a.Z1, a.H1,
                               want_bwd ? a.H1T : nullptr, ldT, s);
    if (rc != ANTS_OK) return rc;
    rc = mma_train_forward(ctx, a.H1, false, M->d_w2b, M->d_par + o.b2, (int)n, H, H, a.Z2, a.H2, nullptr, ldT, s);
    if (rc != ANTS_OK) return rc;
    output_layer<<<blocks_for(n, 8), 256, 0, s>>>(a.H2, n, H, H, M->d_par + o.W3, M->d_par + o.b3, a.O);
    count_launch();
    return ANTS_OK;
}

// gradient of the batch loss into g (parameter layout), from dO [n][3]
int tc_backward(ants_ctx *ctx, const ants_mlp *M, long n, const TcActs &a, const float *dO, float *g,
                cudaStream_t s)
{
    const Offsets o = offsets(M->n_in, M->H);
    const int H = M->H, I = M->n_in;
    const int ldT = (int)round8(n);
    output_weight_grad<<<H, 256, 0, s>>>(dO, a.H2, n, H, g + o.W3);
    launch_column_sums(dO, n, 3, g + o.b3, s);
    output_backward<<<blocks_for(n * H, 256), 256, 0, s>>>(dO, M->d_par + o.W3, a.Z2, n, H, a.dZ2);
    transpose_bf16<<<dim3((unsigned)((ldT + 31) / 32), (unsigned)((H + 31) / 32)), dim3(32, 8), 0, s>>>(
        a.dZ2, n, H, ldT, a.dZ2T);
    launch_column_sums(a.dZ2, n, H, g + o.b2, s);
    count_launch(5);
    int rc = mma_f32(ctx, a.dZ2T, a.H1T, H, H, ldT, g + o.W2, s);
    if (rc != ANTS_OK) return rc;
    rc = mma_gelu_backward(ctx, a.dZ2, M->d_w2tb, a.Z1, (int)n, H, H, a.dZ1, a.dZ1T, ldT, s);
    if (rc != ANTS_OK) return rc;
    launch_column_sums(a.dZ1, n, H, g + o.b1, s);
    count_launch();
    return mma_f32(ctx, a.dZ1T, a.UT, H, I, ldT, g + o.W1, s);
}

struct Buf {
    void *p = nullptr;
    ~Buf() { cudaFree(p); }
    int alloc(size_t bytes, const char *what)
    {
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e != cudaSuccess) return fail(ANTS_E_OOM, "cudaMalloc(%s, %zu): %s", what, bytes, cudaGetErrorString(e));
        return ANTS_OK;
    }
    float *f() const { return (float *)p; }
};

#define MLP_TRY(x)                       \
    do {                                 \
        int _rc = (x);                   \
        if (_rc != ANTS_OK) return _rc;  \
    } while (0)

// sum of per-block partials in a fixed order on the host
float host_sum(const float *d_part, int n, cudaStream_t s, int *rc)
{
    std::vector<float> h(n);
    cudaError_t e = cudaMemcpyAsync(h.data(), d_part, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *rc = cuda_fail(e, "mlp: loss readback");
        return 0.0f;
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += h[i];
    *rc = ANTS_OK;
    return (float)acc;
}

constexpr int kLossBlocks = 64;

}  // namespace

// BF16 inference on the tensor cores: the same roundings as the BF16 training
// path (operands rounded to BF16, FP32 accumulation), in fewer passes
int mlp_forward_tc(ants_ctx *ctx, const ants_mlp *Mc, const float *sig, long n, float *O, cudaStream_t s)
{
    ants_mlp *M = const_cast<ants_mlp *>(Mc);
    const Offsets o = offsets(M->n_in, M->H);
    const int H = M->H, I = M->n_in;
    const int Hp = (H + 7) & ~7, Ip = (I + 7) & ~7;  // 16-byte rows for the tensor-core operands
    if (Ip > 256 || Hp > 256)
        return fail(ANTS_E_UNIMPLEMENTED, "BF16 inference: inputs and hidden width must be <= 256 (%d, %d)", I, H);
    if (!M->d_w1b) {
        ANTS_CUDA_TRY(cudaMalloc(&M->d_w1b, (size_t)Hp * Ip * sizeof(__nv_bfloat16)), "bf16 weights");
        ANTS_CUDA_TRY(cudaMalloc(&M->d_w2b, (size_t)Hp * Hp * sizeof(__nv_bfloat16)), "bf16 weights");
        ANTS_CUDA_TRY(cudaMalloc(&M->d_bpad, 2 * (size_t)Hp * sizeof(float)), "padded biases");
        M->bf16_stale = true;
    }
    if (M->bf16_stale) {
        // padded rows of W carry zero weights and zero bias, so their GELU is 0
        to_bf16_pad<<<blocks_for((long)Hp * Ip, 256), 256, 0, s>>>(M->d_par + o.W1, H, I, Ip, M->d_w1b);
        to_bf16_pad<<<blocks_for((long)Hp * Hp, 256), 256, 0, s>>>(M->d_par + o.W2, H, H, Hp, M->d_w2b);
        if (Hp > H) {
            ANTS_CUDA_TRY(cudaMemsetAsync(M->d_w1b + (size_t)H * Ip, 0, (size_t)(Hp - H) * Ip * 2, s), "pad");
            ANTS_CUDA_TRY(cudaMemsetAsync(M->d_w2b + (size_t)H * Hp, 0, (size_t)(Hp - H) * Hp * 2, s), "pad");
        }
        copy_pad<<<1, 256, 0, s>>>(M->d_par + o.b1, H, Hp, M->d_bpad);
        copy_pad<<<1, 256, 0, s>>>(M->d_par + o.b2, H, Hp, M->d_bpad + Hp);
        count_launch(4);
        M->bf16_stale = false;
    }
    const long chunk = 1L << 17;
    const long cap = n < chunk ? n : chunk;
    const size_t bytes = (size_t)cap * Ip * sizeof(float) + 2 * (size_t)cap * Hp * sizeof(__nv_bfloat16) + 256;
    unsigned char *base = (unsigned char *)ctx_scratch(ctx, 0, bytes);
    if (!base) return ANTS_E_OOM;
    float *U = (float *)base;
    __nv_bfloat16 *H1 = (__nv_bfloat16 *)(base + (size_t)cap * Ip * sizeof(float));
    __nv_bfloat16 *H2 = H1 + (size_t)cap * Hp;
    for (long off = 0; off < n; off += chunk) {
        const long m = n - off < chunk ? n - off : chunk;
        normalize_rows_pad<<<blocks_for(m, 8), 256, 0, s>>>(sig + off * I, m, I, Ip, U);
        count_launch();
        int rc = mma_bias_gelu(ctx, U, true, M->d_w1b, M->d_bpad, (int)m, Hp, Ip, H1, s);
        if (rc != ANTS_OK) return rc;
        rc = mma_bias_gelu(ctx, H1, false, M->d_w2b, M->d_bpad + Hp, (int)m, Hp, Hp, H2, s);
        if (rc != ANTS_OK) return rc;
        output_layer<<<blocks_for(m, 8), 256, 0, s>>>(H2, m, H, Hp, M->d_par + o.W3, M->d_par + o.b3, O + off * 3);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ANTS_OK : cuda_fail(e, "mlp tensor-core forward");
}

// forward of n rows (device signals) into raw outputs O [n][3]; chunked
int mlp_forward(ants_ctx *ctx, const ants_mlp *M, const float *sig, long n, bool bf, float *O, cudaStream_t s)
{
    if (bf) return mlp_forward_tc(ctx, M, sig, n, O, s);
    const long chunk = 1L << 16;
    const long cap = n < chunk ? n : chunk;
    float *base = (float *)ctx_scratch(ctx, 0, acts_floats(cap, M->n_in, M->H) * sizeof(float));
    if (!base) return ANTS_E_OOM;
    Acts a = carve(base, cap, M->n_in, M->H);
    for (long off = 0; off < n; off += chunk) {
        const long m = n - off < chunk ? n - off : chunk;
        Acts b = a;
        b.O = O + off * 3;  // write outputs in place
        forward_batch(M, M->d_par, sig + off * M->n_in, nullptr, m, bf, b, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp forward launch");
    return ANTS_OK;
}

int mlp_n_in(const ants_mlp *M) { return M ? M->n_in : -1; }

int mlp_decode(const ants_mlp *M, const float *O, long n, float *xyz, float *E, cudaStream_t s)
{
    decode_outputs<<<blocks_for(n, 256), 256, 0, s>>>(O, n, M->cfg, xyz, E);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ANTS_OK : cuda_fail(e, "decode launch");
}

}  // namespace ants

using namespace ants;

static int check_mlp(const ants_mlp *M, const char *fn)
{
    if (!M || !M->d_par) return fail(ANTS_E_ARG, "%s: NULL network", fn);
    return ANTS_OK;
}

extern "C" {

ANTS_API int ants_mlp_create(ants_ctx *ctx, int n_in, const ants_mlp_config *cfg, uint64_t seed, ants_mlp **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_mlp_create: out is NULL");
    *out = nullptr;
    if (!ctx || !cfg) return fail(ANTS_E_ARG, "ants_mlp_create: NULL ctx or config");
    if (n_in < 1 || n_in > 1024) return fail(ANTS_E_ARG, "ants_mlp_create: n_in %d not in [1, 1024]", n_in);
    if (cfg->n_hidden < 4 || cfg->n_hidden > 1024)
        return fail(ANTS_E_ARG, "ants_mlp_create: n_hidden %d not in [4, 1024]", cfg->n_hidden);
    if (!(cfg->xy_scale > 0.0f) || !(cfg->loge_std > 0.0f) || !std::isfinite(cfg->loge_mean))
        return fail(ANTS_E_ARG, "ants_mlp_create: xy_scale and loge_std must be > 0");
    ants_mlp *M = new (std::nothrow) ants_mlp();
    if (!M) return fail(ANTS_E_OOM, "ants_mlp_create: out of host memory");
    M->ctx = ctx;
    M->device = ctx->device;
    M->n_in = n_in;
    M->H = cfg->n_hidden;
    M->cfg = *cfg;
    const Offsets o = offsets(n_in, M->H);
    M->n_par = o.total;
    // He-normal hidden weights, Xavier-normal output weights, zero biases
    std::vector<float> p(o.total, 0.0f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (size_t i = 0; i < (size_t)M->H * n_in; ++i) p[o.W1 + i] = (float)(nd(rng) * std::sqrt(2.0 / n_in));
    for (size_t i = 0; i < (size_t)M->H * M->H; ++i) p[o.W2 + i] = (float)(nd(rng) * std::sqrt(2.0 / M->H));
    for (size_t i = 0; i < 3 * (size_t)M->H; ++i) p[o.W3 + i] = (float)(nd(rng) * std::sqrt(2.0 / (M->H + 3)));
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_par, o.total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&M->d_m, o.total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&M->d_v, o.total * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(M->d_par, p.data(), o.total * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->d_m, 0, o.total * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(M->d_v, 0, o.total * sizeof(float));
    if (e != cudaSuccess) {
        ants_mlp_free(M);
        return cuda_fail(e, "ants_mlp_create");
    }
    *out = M;
    return ANTS_OK;
}

ANTS_API void ants_mlp_free(ants_mlp *M)
{
    if (!M) return;
    cudaSetDevice(M->device);
    cudaFree(M->d_par);
    cudaFree(M->d_m);
    cudaFree(M->d_v);
    cudaFree(M->d_w1b);
    cudaFree(M->d_w2b);
    cudaFree(M->d_w2tb);
    cudaFree(M->d_bpad);
    delete M;
    (void)cudaGetLastError();
}

ANTS_API int ants_mlp_shape(const ants_mlp *M, int *n_in, int *n_hidden, long *n_params)
{
    begin_call();
    MLP_TRY(check_mlp(M, "ants_mlp_shape"));
    if (n_in) *n_in = M->n_in;
    if (n_hidden) *n_hidden = M->H;
    if (n_params) *n_params = (long)M->n_par;
    return ANTS_OK;
}

ANTS_API int ants_mlp_set_params(ants_mlp *M, const float *params_host, long count)
{
    begin_call();
    MLP_TRY(check_mlp(M, "ants_mlp_set_params"));
    if (!params_host || count != (long)M->n_par)
        return fail(ANTS_E_ARG, "ants_mlp_set_params: need %zu parameters", M->n_par);
    ANTS_CUDA_TRY(cudaSetDevice(M->ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaMemcpy(M->d_par, params_host, M->n_par * sizeof(float), cudaMemcpyHostToDevice), "upload");
    ANTS_CUDA_TRY(cudaMemset(M->d_m, 0, M->n_par * sizeof(float)), "memset");
    ANTS_CUDA_TRY(cudaMemset(M->d_v, 0, M->n_par * sizeof(float)), "memset");
    M->adam_t = 0;
    M->bf16_stale = true;
    return ANTS_OK;
}

ANTS_API int ants_mlp_get_params(const ants_mlp *M, float *params_host, long count)
{
    begin_call();
    MLP_TRY(check_mlp(M, "ants_mlp_get_params"));
    if (!params_host || count < (long)M->n_par)
        return fail(ANTS_E_ARG, "ants_mlp_get_params: need room for %zu parameters", M->n_par);
    ANTS_CUDA_TRY(cudaSetDevice(M->ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaMemcpy(params_host, M->d_par, M->n_par * sizeof(float), cudaMemcpyDeviceToHost), "download");
    return ANTS_OK;
}

ANTS_API int ants_mlp_forward(ants_ctx *ctx, const ants_mlp *M, const float *signals_dev, long n_events,
                              int n_sensors, int bf16, float *out_dev, float *start_xyz_dev, float *E_dev,
                              void *stream)
{
    begin_call();
    ANTS_NVTX("ants_mlp_forward");
    MLP_TRY(check_mlp(M, "ants_mlp_forward"));
    if (!ctx || M->ctx != ctx) return fail(ANTS_E_ARG, "ants_mlp_forward: network belongs to another context");
    if (n_sensors != M->n_in)
        return fail(ANTS_E_SHAPE, "ants_mlp_forward: n_sensors %d but the network takes %d", n_sensors, M->n_in);
    if (n_events < 0) return fail(ANTS_E_ARG, "ants_mlp_forward: n_events < 0");
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev || !out_dev) return fail(ANTS_E_ARG, "ants_mlp_forward: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    MLP_TRY(mlp_forward(ctx, M, signals_dev, n_events, bf16 != 0, out_dev, s));
    if (start_xyz_dev || E_dev) {
        if (!start_xyz_dev) return fail(ANTS_E_ARG, "ants_mlp_forward: E_dev needs start_xyz_dev");
        MLP_TRY(mlp_decode(M, out_dev, n_events, start_xyz_dev, E_dev, s));
    }
    return ANTS_OK;
}

ANTS_API int ants_mlp_loss_grad(ants_ctx *ctx, const ants_mlp *M, const float *signals_dev, const float *truth_dev,
                                long n_events, int n_sensors, int bf16, float *loss_host, float *grads_host)
{
    begin_call();
    ANTS_NVTX("ants_mlp_loss_grad");
    MLP_TRY(check_mlp(M, "ants_mlp_loss_grad"));
    if (!ctx || M->ctx != ctx) return fail(ANTS_E_ARG, "ants_mlp_loss_grad: network belongs to another context");
    if (n_sensors != M->n_in) return fail(ANTS_E_SHAPE, "ants_mlp_loss_grad: n_sensors %d", n_sensors);
    if (n_events < 1 || n_events > (1L << 20)) return fail(ANTS_E_ARG, "ants_mlp_loss_grad: n_events out of range");
    if (!signals_dev || !truth_dev) return fail(ANTS_E_ARG, "ants_mlp_loss_grad: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = ctx->stream[0];
    const int H = M->H;
    const bool tc = bf16 != 0 && tc_trainable(M);  // BF16 products on the tensor cores
    Buf acts, tgt, dO, dA, dB, g, part;
    if (tc) {
        MLP_TRY(acts.alloc(tc_bytes(n_events, M->n_in, H), "activations"));
    } else {
        MLP_TRY(acts.alloc(acts_floats(n_events, M->n_in, H) * sizeof(float), "activations"));
        MLP_TRY(dA.alloc((size_t)n_events * H * sizeof(float), "dA"));
        MLP_TRY(dB.alloc((size_t)n_events * H * sizeof(float), "dB"));
    }
    MLP_TRY(tgt.alloc(n_events * 3 * sizeof(float), "targets"));
    MLP_TRY(dO.alloc(n_events * 3 * sizeof(float), "dO"));
    MLP_TRY(g.alloc(M->n_par * sizeof(float), "grads"));
    MLP_TRY(part.alloc(kLossBlocks * sizeof(float), "loss"));
    if (tc) {
        const TcActs a = tc_carve((unsigned char *)acts.p, n_events, M->n_in, H);
        // the BF16 copies are caches of the parameters, which stay unchanged
        MLP_TRY(tc_refresh_weights(const_cast<ants_mlp *>(M), s));
        MLP_TRY(tc_forward(ctx, M, signals_dev, nullptr, n_events, true, a, s));
        make_targets<<<blocks_for(n_events, 256), 256, 0, s>>>(truth_dev, nullptr, n_events, M->cfg, tgt.f());
        mse_grad<<<kLossBlocks, 256, 0, s>>>(a.O, tgt.f(), n_events, dO.f(), part.f());
        MLP_TRY(tc_backward(ctx, M, n_events, a, dO.f(), g.f(), s));
    } else {
        Acts a = carve(acts.f(), n_events, M->n_in, H);
        forward_batch(M, M->d_par, signals_dev, nullptr, n_events, bf16 != 0, a, s);
        make_targets<<<blocks_for(n_events, 256), 256, 0, s>>>(truth_dev, nullptr, n_events, M->cfg, tgt.f());
        mse_grad<<<kLossBlocks, 256, 0, s>>>(a.O, tgt.f(), n_events, dO.f(), part.f());
        backward_batch(M, M->d_par, n_events, bf16 != 0, a, dO.f(), dA.f(), dB.f(), g.f(), s);
    }
    count_launch(2);
    ANTS_CUDA_TRY(cudaGetLastError(), "mlp loss_grad launch");
    int rc;
    float loss = host_sum(part.f(), kLossBlocks, s, &rc);
    if (rc != ANTS_OK) return rc;
    if (loss_host) *loss_host = loss;
    if (grads_host)
        ANTS_CUDA_TRY(cudaMemcpy(grads_host, g.p, M->n_par * sizeof(float), cudaMemcpyDeviceToHost), "grads");
    return ANTS_OK;
}

ANTS_API int ants_mlp_train(ants_ctx *ctx, ants_mlp *M, const float *signals_dev, const float *truth_dev,
                            long n_events, int n_sensors, const ants_train_params *tp, ants_train_report *report)
{
    begin_call();
    ANTS_NVTX("ants_mlp_train");
    MLP_TRY(check_mlp(M, "ants_mlp_train"));
    if (!ctx || M->ctx != ctx || !tp) return fail(ANTS_E_ARG, "ants_mlp_train: bad ctx or params");
    if (n_sensors != M->n_in) return fail(ANTS_E_SHAPE, "ants_mlp_train: n_sensors %d", n_sensors);
    if (!signals_dev || !truth_dev) return fail(ANTS_E_ARG, "ants_mlp_train: NULL buffer");
    if (tp->batch < 1 || tp->batch > 65536 || tp->epochs < 1 || !(tp->lr > 0.0f) || !(tp->monitor_frac > 0.0f) ||
        !(tp->monitor_frac < 1.0f) || tp->patience < 1)
        return fail(ANTS_E_ARG, "ants_mlp_train: bad training parameters");
    const long n_mon = (long)(tp->monitor_frac * (double)n_events);
    const long n_tr = n_events - n_mon;
    if (n_mon < 1 || n_tr < tp->batch) return fail(ANTS_E_ARG, "ants_mlp_train: too few events");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = ctx->stream[0];
    const int H = M->H, B = tp->batch;
    const bool bf = tp->bf16 != 0;
    const bool tc = bf && tc_trainable(M);  // BF16 products on the tensor cores
    const long mon_chunk = 8192;
    const long cap = std::max<long>(B, std::min(n_mon, mon_chunk));
    Buf acts, tgt, dO, dA, dB, g, part, best, idx;
    if (tc) {
        MLP_TRY(acts.alloc(tc_bytes(cap, M->n_in, H), "activations"));
    } else {
        MLP_TRY(acts.alloc(acts_floats(cap, M->n_in, H) * sizeof(float), "activations"));
        MLP_TRY(dA.alloc((size_t)cap * H * sizeof(float), "dA"));
        MLP_TRY(dB.alloc((size_t)cap * H * sizeof(float), "dB"));
    }
    MLP_TRY(tgt.alloc(cap * 3 * sizeof(float), "targets"));
    MLP_TRY(dO.alloc(cap * 3 * sizeof(float), "dO"));
    MLP_TRY(g.alloc(M->n_par * sizeof(float), "grads"));
    MLP_TRY(part.alloc(kLossBlocks * sizeof(float), "loss"));
    MLP_TRY(best.alloc(M->n_par * sizeof(float), "best"));
    MLP_TRY(idx.alloc((size_t)n_events * sizeof(long), "index"));
    Acts a{};
    TcActs ta{};
    if (tc) {
        ta = tc_carve((unsigned char *)acts.p, cap, M->n_in, H);
        MLP_TRY(tc_refresh_weights(M, s));
    } else {
        a = carve(acts.f(), cap, M->n_in, H);
    }
    float *const out_rows = tc ? ta.O : a.O;  // network outputs of the current batch
    std::vector<long> perm(n_tr);
    for (long i = 0; i < n_tr; ++i) perm[i] = i;
    std::mt19937_64 rng(tp->seed);
    std::vector<long> mon(n_mon);
    for (long i = 0; i < n_mon; ++i) mon[i] = n_tr + i;
    long *d_idx = (long *)idx.p;
    long *d_mon = d_idx + n_tr;
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_mon, mon.data(), n_mon * sizeof(long), cudaMemcpyHostToDevice, s), "upload");
    float best_mse = INFINITY, last_train = 0.0f;
    int best_epoch = -1, epochs_run = 0, since_best = 0;
    for (int ep = 0; ep < tp->epochs; ++ep) {
        // Fisher-Yates shuffle of the training rows
        for (long i = n_tr - 1; i > 0; --i) std::swap(perm[i], perm[(long)(rng() % (unsigned long long)(i + 1))]);
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_idx, perm.data(), n_tr * sizeof(long), cudaMemcpyHostToDevice, s), "upload");
        for (long off = 0; off + B <= n_tr; off += B) {
            const long *bidx = d_idx + off;
            if (tc) MLP_TRY(tc_forward(ctx, M, signals_dev, bidx, B, true, ta, s));
            else forward_batch(M, M->d_par, signals_dev, bidx, B, bf, a, s);
            make_targets<<<blocks_for(B, 256), 256, 0, s>>>(truth_dev, bidx, B, M->cfg, tgt.f());
            mse_grad<<<kLossBlocks, 256, 0, s>>>(out_rows, tgt.f(), B, dO.f(), part.f());
            if (tc) MLP_TRY(tc_backward(ctx, M, B, ta, dO.f(), g.f(), s));
            else backward_batch(M, M->d_par, B, bf, a, dO.f(), dA.f(), dB.f(), g.f(), s);
            M->adam_t += 1;
            const float c1 = 1.0f - powf(tp->beta1, (float)M->adam_t), c2 = 1.0f - powf(tp->beta2, (float)M->adam_t);
            adam_kernel<<<blocks_for((long)M->n_par, 256), 256, 0, s>>>(M->n_par, M->d_par, g.f(), M->d_m, M->d_v,
                                                                        tp->lr, tp->beta1, tp->beta2, tp->eps, c1, c2);
            count_launch(3);
            if (tc) MLP_TRY(tc_refresh_weights(M, s));
            if (off + 2 * B > n_tr) {  // loss of the last batch of the epoch
                int rc;
                last_train = host_sum(part.f(), kLossBlocks, s, &rc);
                if (rc != ANTS_OK) return rc;
            }
        }
        ANTS_CUDA_TRY(cudaGetLastError(), "mlp train launch");
        // monitor subset (Sec. 5.1.3: training stops when it stops improving)
        double mse = 0.0;
        for (long off = 0; off < n_mon; off += mon_chunk) {
            const long m = std::min(mon_chunk, n_mon - off);
            if (tc) MLP_TRY(tc_forward(ctx, M, signals_dev, d_mon + off, m, false, ta, s));
            else forward_batch(M, M->d_par, signals_dev, d_mon + off, m, bf, a, s);
            make_targets<<<blocks_for(m, 256), 256, 0, s>>>(truth_dev, d_mon + off, m, M->cfg, tgt.f());
            mse_grad<<<kLossBlocks, 256, 0, s>>>(out_rows, tgt.f(), m, nullptr, part.f());
            count_launch(2);
            int rc;
            const float chunk_mse = host_sum(part.f(), kLossBlocks, s, &rc);
            if (rc != ANTS_OK) return rc;
            mse += (double)chunk_mse * (double)m / (double)n_mon;
        }
        ++epochs_run;
        if (mse < best_mse * (1.0 - 1e-3)) {
            best_mse = (float)mse;
            best_epoch = ep;
            since_best = 0;
            ANTS_CUDA_TRY(cudaMemcpyAsync(best.p, M->d_par, M->n_par * sizeof(float), cudaMemcpyDeviceToDevice, s),
                          "keep best");
        } else if (++since_best >= tp->patience) {
            break;
        }
    }
    ANTS_CUDA_TRY(cudaMemcpyAsync(M->d_par, best.p, M->n_par * sizeof(float), cudaMemcpyDeviceToDevice, s),
                  "restore best");
    M->bf16_stale = true;
    ANTS_CUDA_TRY(cudaStreamSynchronize(s), "mlp train");
    MLP_TRY(check_bounds(ctx, s));
    if (report) {
        report->epochs_run = epochs_run;
        report->best_epoch = best_epoch;
        report->best_monitor_mse = best_mse;
        report->last_train_mse = last_train;
    }
    return ANTS_OK;
}

// --- save / load: "ANTSMLP1", n_in, n_hidden, config, adam_t, params -------------

ANTS_API int ants_mlp_save(const ants_mlp *M, const char *path)
{
    begin_call();
    MLP_TRY(check_mlp(M, "ants_mlp_save"));
    if (!path) return fail(ANTS_E_ARG, "ants_mlp_save: NULL path");
    std::vector<float> p(M->n_par);
    ANTS_CUDA_TRY(cudaSetDevice(M->ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaMemcpy(p.data(), M->d_par, M->n_par * sizeof(float), cudaMemcpyDeviceToHost), "download");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ANTS_E_IO, "ants_mlp_save: cannot open %s", path);
    const char magic[8] = {'A', 'N', 'T', 'S', 'M', 'L', 'P', '1'};
    int32_t hdr[3] = {M->n_in, M->H, M->adam_t};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 3, f) == 3 &&
              fwrite(&M->cfg, sizeof(ants_mlp_config), 1, f) == 1 && fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? ANTS_OK : fail(ANTS_E_IO, "ants_mlp_save: write to %s failed", path);
}

ANTS_API int ants_mlp_load(ants_ctx *ctx, const char *path, ants_mlp **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_mlp_load: out is NULL");
    *out = nullptr;
    if (!ctx || !path) return fail(ANTS_E_ARG, "ants_mlp_load: NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ANTS_E_IO, "ants_mlp_load: cannot open %s", path);
    char magic[8];
    int32_t hdr[3];
    ants_mlp_config cfg;
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "ANTSMLP1", 8) == 0 &&
              fread(hdr, sizeof(int32_t), 3, f) == 3 && fread(&cfg, sizeof(cfg), 1, f) == 1;
    if (!ok || hdr[0] < 1 || hdr[0] > 1024 || hdr[1] != cfg.n_hidden) {
        fclose(f);
        return fail(ANTS_E_IO, "ants_mlp_load: %s is not a network file", path);
    }
    const Offsets o = offsets(hdr[0], hdr[1]);
    std::vector<float> p(o.total);
    ok = fread(p.data(), sizeof(float), p.size(), f) == p.size();
    fclose(f);
    if (!ok) return fail(ANTS_E_IO, "ants_mlp_load: %s is truncated", path);
    ants_mlp *M = nullptr;
    int rc = ants_mlp_create(ctx, hdr[0], &cfg, 0, &M);
    if (rc != ANTS_OK) return rc;
    rc = ants_mlp_set_params(M, p.data(), (long)p.size());
    if (rc != ANTS_OK) {
        ants_mlp_free(M);
        return rc;
    }
    M->adam_t = hdr[2];
    *out = M;
    return ANTS_OK;
}

}  // extern "C"
