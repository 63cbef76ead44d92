// BF16 tensor-core products with fused epilogues.
//
//   C[m][n] = sum_k A[m][k] B[n][k]      (A [M][K], B [N][K], both K-contiguous)
//
// Block tile 64 (m) x 128 (n), 8 warps of 32 x 32, K staged through shared
// memory 64 at a time; mma.sync.m16n8k16 (BF16 x BF16 -> FP32).  A may be FP32
// in global memory (rounded to BF16 while it is staged) or BF16.  One block
// owns a 64-row band of C and walks all of N, so row-wise epilogues see every
// column of their rows:
//   EPI_TOPK       running top-K (value desc, index asc) per row, written as
//                  K (score, column) pairs per row -- the global-grid
//                  candidate search of the precision form;
//   EPI_BIAS_GELU  GELU(C + bias[n]) stored as BF16 -- a hidden layer of the
//                  proposal network.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace ants {

namespace {

constexpr int kTM = 64, kTN = 128, kKC = 64, kPad = 8;
constexpr int kThreads = 256;
constexpr int kMaxTop = 8;

enum { EPI_TOPK = 0, EPI_BIAS_GELU = 1 };

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

struct MmaArgs {
    int M, N, K;
    const void *A;  // [M][K] FP32 or BF16
    const __nv_bfloat16 *B;  // [N][K]
    // EPI_TOPK
    int topk;
    float *top_val;  // [M][topk]
    int *top_idx;    // [M][topk]
    // EPI_BIAS_GELU
    const float *bias;     // [N]
    __nv_bfloat16 *out;    // [M][N]
};

// insert (v, c) into a descending list of length k (ties: lower column first)
__device__ __forceinline__ void top_insert(float *val, int *idx, int k, float v, int c)
{
    if (!(v > val[k - 1] || (v == val[k - 1] && c < idx[k - 1]))) return;
    int p = k - 1;
    while (p > 0 && (v > val[p - 1] || (v == val[p - 1] && c < idx[p - 1]))) {
        val[p] = val[p - 1];
        idx[p] = idx[p - 1];
        --p;
    }
    val[p] = v;
    idx[p] = c;
}

template <int EPI, bool A_F32>
__global__ void __launch_bounds__(kThreads) mma_tn_kernel(MmaArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem);       // [kTM][kKC + kPad]
    __nv_bfloat16 *Bs = As + kTM * (kKC + kPad);                         // [kTN][kKC + kPad]
    float *Cs = reinterpret_cast<float *>(Bs + kTN * (kKC + kPad));      // [kTM][kTN + 4] (top-K)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps
    const int g = lane >> 2, t4 = lane & 3;
    const int m0 = blockIdx.x * kTM;
    constexpr int LDS = kKC + kPad;

    // top-K state: 4 threads per row, each over a quarter of every column chunk
    float tv[kMaxTop];
    int ti[kMaxTop];
    const int trow = tid >> 2, tq = tid & 3;
    if (EPI == EPI_TOPK)
        for (int j = 0; j < kMaxTop; ++j) {
            tv[j] = -INFINITY;
            ti[j] = 0x7fffffff;
        }

    for (int n0 = 0; n0 < a.N; n0 += kTN) {
        float acc[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
        for (int k0 = 0; k0 < a.K; k0 += kKC) {
            // stage A (64 x 64) and B (128 x 64), zero outside the matrices
            for (int l = tid; l < kTM * kKC / 2; l += kThreads) {
                const int r = l / (kKC / 2), c2 = (l % (kKC / 2)) * 2;
                const int m = m0 + r, k = k0 + c2;
                __nv_bfloat162 v = __floats2bfloat162_rn(0.0f, 0.0f);
                if (m < a.M && k < a.K) {
                    if (A_F32) {
                        const float *Af = static_cast<const float *>(a.A) + (size_t)m * a.K + k;
                        v = __floats2bfloat162_rn(Af[0], k + 1 < a.K ? Af[1] : 0.0f);
                    } else {
                        const __nv_bfloat16 *Ab = static_cast<const __nv_bfloat16 *>(a.A) + (size_t)m * a.K + k;
                        v = __halves2bfloat162(Ab[0], k + 1 < a.K ? Ab[1] : __float2bfloat16_rn(0.0f));
                    }
                }
                *reinterpret_cast<__nv_bfloat162 *>(As + r * LDS + c2) = v;
            }
            for (int l = tid; l < kTN * kKC / 2; l += kThreads) {
                const int r = l / (kKC / 2), c2 = (l % (kKC / 2)) * 2;
                const int n = n0 + r, k = k0 + c2;
                __nv_bfloat162 v = __floats2bfloat162_rn(0.0f, 0.0f);
                if (n < a.N && k < a.K) {
                    const __nv_bfloat16 *Bb = a.B + (size_t)n * a.K + k;
                    v = __halves2bfloat162(Bb[0], k + 1 < a.K ? Bb[1] : __float2bfloat16_rn(0.0f));
                }
                *reinterpret_cast<__nv_bfloat162 *>(Bs + r * LDS + c2) = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kKC; kk += 16) {
                uint32_t af[2][4], bfr[4][2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const __nv_bfloat16 *p = As + (wm * 32 + i * 16 + g) * LDS + kk + 2 * t4;
                    af[i][0] = *reinterpret_cast<const uint32_t *>(p);
                    af[i][1] = *reinterpret_cast<const uint32_t *>(p + 8 * LDS);
                    af[i][2] = *reinterpret_cast<const uint32_t *>(p + 8);
                    af[i][3] = *reinterpret_cast<const uint32_t *>(p + 8 * LDS + 8);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const __nv_bfloat16 *p = Bs + (wn * 32 + j * 8 + g) * LDS + kk + 2 * t4;
                    bfr[j][0] = *reinterpret_cast<const uint32_t *>(p);
                    bfr[j][1] = *reinterpret_cast<const uint32_t *>(p + 8);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
            }
            __syncthreads();
        }
        // ---- epilogue for this column chunk ---------------------------------
        if (EPI == EPI_BIAS_GELU) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m = m0 + wm * 32 + i * 16 + g + 8 * h;
                        const int n = n0 + wn * 32 + j * 8 + 2 * t4;
                        if (m >= a.M) continue;
                        if (n < a.N) a.out[(size_t)m * a.N + n] = __float2bfloat16_rn(gelu_f(acc[i][j][2 * h] + a.bias[n]));
                        if (n + 1 < a.N)
                            a.out[(size_t)m * a.N + n + 1] =
                                __float2bfloat16_rn(gelu_f(acc[i][j][2 * h + 1] + a.bias[n + 1]));
                    }
        } else {
            constexpr int LDC = kTN + 4;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int r = wm * 32 + i * 16 + g + 8 * h;
                        const int c = wn * 32 + j * 8 + 2 * t4;
                        Cs[r * LDC + c] = acc[i][j][2 * h];
                        Cs[r * LDC + c + 1] = acc[i][j][2 * h + 1];
                    }
            __syncthreads();
            // thread (trow, tq) scans columns tq, tq+4, ... of its row
            for (int c = tq; c < kTN && n0 + c < a.N; c += 4) top_insert(tv, ti, a.topk, Cs[trow * LDC + c], n0 + c);
            __syncthreads();
        }
    }
    if (EPI == EPI_TOPK) {
        // merge the four partial lists of each row through shared memory
        float *mv = Cs;                                            // [kTM][4][kMaxTop]
        int *mi = reinterpret_cast<int *>(Cs + kTM * 4 * kMaxTop);  // [kTM][4][kMaxTop]
        for (int j = 0; j < a.topk; ++j) {
            mv[(trow * 4 + tq) * kMaxTop + j] = tv[j];
            mi[(trow * 4 + tq) * kMaxTop + j] = ti[j];
        }
        __syncthreads();
        if (tq == 0) {
            for (int q = 1; q < 4; ++q)
                for (int j = 0; j < a.topk; ++j)
                    top_insert(tv, ti, a.topk, mv[(trow * 4 + q) * kMaxTop + j], mi[(trow * 4 + q) * kMaxTop + j]);
            const int m = m0 + trow;
            if (m < a.M)
                for (int j = 0; j < a.topk; ++j) {
                    a.top_val[(size_t)m * a.topk + j] = tv[j];
                    a.top_idx[(size_t)m * a.topk + j] = ti[j];
                }
        }
    }
}

size_t smem_bytes(int epi)
{
    size_t ab = (size_t)(kTM + kTN) * (kKC + kPad) * sizeof(__nv_bfloat16);
    size_t c = epi == EPI_TOPK ? (size_t)kTM * (kTN + 4) * sizeof(float) : 0;
    return ab + c;
}

template <int EPI, bool AF>
int launch(const MmaArgs &a, cudaStream_t s)
{
    const size_t smem = smem_bytes(EPI);
    cudaError_t e = cudaFuncSetAttribute(mma_tn_kernel<EPI, AF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mma)");
    const unsigned blocks = (unsigned)((a.M + kTM - 1) / kTM);
    mma_tn_kernel<EPI, AF><<<blocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mma launch");
    count_launch();
    return ANTS_OK;
}

}  // namespace

int mma_topk(const void *A, bool a_f32, const __nv_bfloat16 *B, int M, int N, int K, int topk, float *val, int *idx,
             cudaStream_t s)
{
    if (topk < 1 || topk > kMaxTop) return fail(ANTS_E_ARG, "top-K: K must be in [1, %d]", kMaxTop);
    if (M <= 0) return ANTS_OK;
    MmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.B = B;
    a.topk = topk;
    a.top_val = val;
    a.top_idx = idx;
    return a_f32 ? launch<EPI_TOPK, true>(a, s) : launch<EPI_TOPK, false>(a, s);
}

int mma_bias_gelu(const void *A, bool a_f32, const __nv_bfloat16 *B, const float *bias, int M, int N, int K,
                  __nv_bfloat16 *out, cudaStream_t s)
{
    if (M <= 0) return ANTS_OK;
    MmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.B = B;
    a.bias = bias;
    a.out = out;
    return a_f32 ? launch<EPI_BIAS_GELU, true>(a, s) : launch<EPI_BIAS_GELU, false>(a, s);
}

}  // namespace ants
